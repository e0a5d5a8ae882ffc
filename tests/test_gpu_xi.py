"""The variance-optimal sampling law xi** (Thm 3.1) on the GPU, through the C ABI, against the oracle.

mlmc_plan computes q_k = sqrt(E||A_{:,k}||^2 E||B_{k,:}||^2) and their running sums on the device
in the oracle's summation order; a slot draws the smallest k with u Q_{n-1} < Q_k and carries the
weight Q_{n-1} / q_k.

Bars:
  * indices: bit-exact (the same FP64 decision on both sides; a tie within one ulp of a
    cumulative sum would be the only way to differ);
  * FP64 samples: |D - D_oracle| <= 1e-12 * mag (mag includes the 1 / xi weights); level means
    within 1e-12 of the mean magnitude, M2 within 1e-11 relative; the estimate's N_l equal;
  * FP32 samples: tau_32(c) = (c + 8) 2^-24 + 2^-16 of mag, plus 2^-24 for the FP32 weights;
  * BF16 (tensor cores; the weight Q_{n-1} / q_k, rounded to FP32, multiplies each entry of B before
    its bfloat16 rounding): tau_bf16(c) = 2^-7 + 2^-15 + (c + 8) 2^-23 of mag plus 2^-22 for the
    FP32 weight and its product, per sample and for level means over the same samples.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
SEEDS = dict(seed_A=5, seed_B=6, seed_idx=7, problem_id=2)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def tau32(c):
    return (c + 9) * 2.0**-24 + 2.0**-16


def _params(m, n, p, dtype, zero_col=None, seed=3):
    rng = np.random.default_rng(seed)
    scale = np.linspace(0.2, 2.0, n)   # columns of unequal size, so xi** is far from uniform
    M = rng.uniform(-1, 1, (m, n)) * scale
    S = rng.uniform(0.1, 1, (m, n)) * scale
    Mp = rng.uniform(-1, 1, (n, p))
    Sp = rng.uniform(0.1, 1, (n, p))
    if zero_col is not None:
        M[:, zero_col] = 0.0
        S[:, zero_col] = 0.0
    return [x.astype(dtype) for x in (M, S, Mp, Sp)]


def _plan(params, precision, c0, L, **kw):
    tdt = torch.float64 if params[0].dtype == np.float64 else torch.float32
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(DEV, tdt) for x in params]
    return binding.Plan([binding.ProblemSpec(*ts, **SEEDS)], c0=c0, L=L, ratio=2, precision=precision,
                        sampling="optimal", **kw)


def _orc(params):
    return oracle.Problem(*[x.astype(np.float64) for x in params], sampling="optimal", **SEEDS)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_indices_match_oracle(precision):
    params = _params(24, 700, 16, np.float64 if precision == "fp64" else np.float32, zero_col=13)
    orc = _orc(params)
    with _plan(params, precision, 4, 3) as plan:
        for (l, s, t0, count) in [(0, 0, 0, 4), (1, 5, 0, 8), (3, 2**40 + 9, 3, 29), (2, 77, 0, 16)]:
            got = plan.debug_indices(0, l, s, t0, count).cpu().numpy()
            want = [oracle.index_xi(orc, l, s, t) for t in range(t0, t0 + count)]
            assert list(got) == want, (l, s)
            assert 13 not in got


CASES = [
    # m, n, p, c0, L, (level, sample) pairs
    (24, 700, 16, 4, 3, [(0, 0), (1, 3), (3, 9)]),
    (70, 300, 130, 1, 4, [(0, 1), (2, 8), (4, 2)]),   # two column tiles, odd slot counts
]


@pytest.mark.parametrize("m,n,p,c0,L,picks", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_samples_match_oracle(m, n, p, c0, L, picks, precision):
    params = _params(m, n, p, np.float64 if precision == "fp64" else np.float32)
    orc = _orc(params)
    lv = oracle.Levels(c0, 2, L)
    with _plan(params, precision, c0, L) as plan:
        for l, s in picks:
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, _, _, mag = oracle.sample(orc, lv, l, s)
            tol = 1e-12 if precision == "fp64" else tau32(lv.cl(l))
            err = np.abs(D - Dref) / mag
            assert np.all(err <= tol), (l, s, err.max(), tol)


def test_nonlinear_f_with_xi_matches_oracle():
    params = _params(24, 700, 16, np.float64)
    orc = _orc(params)
    lv = oracle.Levels(4, 2, 3)
    with _plan(params, "fp64", 4, 3, f="abs_step") as plan:
        for l, s in [(0, 0), (2, 5), (3, 1)]:
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, Pf, Pc, mag = oracle.sample(orc, lv, l, s, fkind=oracle.F_ABS_STEP)
            band = 1e-9 * mag
            far = (np.abs(Pf - 2.0) > band) & ((np.abs(Pc - 2.0) > band) | (l == 0))
            assert np.all(np.abs(D - Dref)[far] <= 1e-12 * mag[far])


def test_level_statistics_and_estimate_match_oracle_fp64():
    params = _params(16, 400, 12, np.float64)
    orc = _orc(params)
    lv = oracle.Levels(4, 2, 3)
    with _plan(params, "fp64", 4, 3) as plan:
        for l, N in enumerate([120, 60, 33, 17]):
            plan.level_stats(0, l, 0, N)
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 0, N)
            assert n_got == N
            assert np.all(np.abs(mean.cpu().numpy() - mref) <= 1e-12 * magm)
            assert abs(M2 - M2ref) <= 1e-11 * M2ref
    eps = 0.1 * np.linalg.norm(params[0] @ params[2])
    Yref, Lref, Nref, Vref, _ = oracle.estimate_f(orc, lv, eps, pilot=32)
    with _plan(params, "fp64", 4, 3, pilot_n=32) as plan:
        (Y,), (rep,) = plan.estimate([eps])
        assert rep["N"] == list(Nref)
        np.testing.assert_allclose(rep["V"], Vref, rtol=1e-11)


def test_xi_lowers_the_level_zero_variance():
    params = _params(16, 400, 12, np.float64)
    ts = [torch.from_numpy(x).to(DEV) for x in params]
    V = {}
    for law in ("uniform", "optimal"):
        with binding.Plan([binding.ProblemSpec(*ts, **SEEDS)], c0=4, L=0, precision="fp64", sampling=law) as plan:
            plan.level_stats(0, 0, 0, 4000)
            n, _, M2 = plan.get_level_stats(0, 0)
            V[law] = M2 / (n - 1)
    assert V["optimal"] < V["uniform"]


def test_unsupported_combinations():
    params = _params(8, 64, 8, np.float32)
    ts = [torch.from_numpy(x).to(DEV) for x in params]
    with pytest.raises(binding.MLMCError) as e:
        binding.Plan([binding.ProblemSpec(*ts)], c0=4, L=2, precision="fp8", sampling="optimal")
    assert e.value.status == 6
    with binding.Plan([binding.ProblemSpec(*ts)], c0=4, L=2, precision="fp32", sampling="optimal") as plan:
        for l in range(3):
            plan.level_stats(0, l, 0, 8)
        plan.telescoping_sum()
        with pytest.raises(binding.MLMCError) as e:
            plan.backward([torch.zeros(8, 8, device=DEV, dtype=torch.float64)])
        assert e.value.status == 6


def tau_bf16(c):
    return 2.0**-7 + 2.0**-15 + (c + 8) * 2.0**-23 + 2.0**-22


BF16_CASES = [
    # m, n, p, c0, L, f, (level, sample) pairs
    (24, 700, 16, 4, 3, "identity", [(0, 0), (1, 3), (3, 9)]),        # c_l < 32: partial sub-blocks
    (70, 300, 130, 1, 4, "identity", [(0, 1), (2, 8), (4, 2)]),       # two column tiles, odd slot counts
    (200, 2000, 300, 32, 2, "identity", [(0, 4), (2, 11)]),           # the CTA pair (256 x 256 tiles)
    (64, 1024, 64, 16, 3, "abs_step", [(0, 2), (1, 5), (3, 1)]),      # the targeted-function form
]


@pytest.mark.parametrize("m,n,p,c0,L,f,picks", BF16_CASES)
def test_bf16_samples_and_levels_match_oracle(m, n, p, c0, L, f, picks):
    params = _params(m, n, p, np.float32)
    if f != "identity":
        # entries of AB of order one around the jump of f at 2
        k = 2.0 / np.sqrt(n)
        params = [(params[0] * k + 2.0 / n).astype(np.float32), (params[1] * k).astype(np.float32),
                  params[2], params[3]]
    orc = _orc(params)
    lv = oracle.Levels(c0, 2, L)
    fkind = oracle.F_ABS_STEP if f != "identity" else oracle.F_IDENTITY
    near = 0
    with _plan(params, "bf16", c0, L, f=f) as plan:
        for l, s in picks:
            c = lv.cl(l)
            D = plan.debug_sample(0, l, s).cpu().numpy().astype(np.float64)
            Dref, Pf, Pc, mag = oracle.sample(orc, lv, l, s, fkind=fkind)
            ok = np.ones(D.shape, dtype=bool)
            if f != "identity":
                band = tau_bf16(c) * mag
                ok = (np.abs(Pf - 2.0) > band) & ((np.abs(Pc - 2.0) > band) | (l == 0))
                near += int((~ok).sum())
            err = np.abs(D - Dref)[ok] / mag[ok]
            assert np.all(err <= tau_bf16(c)), (l, s, err.max(), tau_bf16(c))
        if f == "identity":
            for l in range(min(L, 2) + 1):
                plan.level_stats(0, l, 0, 40)
                n_got, mean, _ = plan.get_level_stats(0, l)
                mref, _, magm = oracle.level_stats(orc, lv, l, 0, 40)
                assert n_got == 40
                assert np.all(np.abs(mean.cpu().numpy() - mref) <= tau_bf16(lv.cl(l)) * magm), l
    assert near <= 0.25 * m * p * len(picks)


def test_bf16_xi_lowers_variance_and_estimates():
    """BF16 under xi** against BF16 under the uniform law on the same problem: a smaller level-0
    variance, and an estimate within five predicted RMSEs of M M'."""
    params = _params(48, 2048, 40, np.float32)
    ts = [torch.from_numpy(x).to(DEV) for x in params]
    mu = params[0].astype(np.float64) @ params[2].astype(np.float64)
    eps = 0.02 * float(np.linalg.norm(mu))
    V0 = {}
    for law in ("uniform", "optimal"):
        with binding.Plan([binding.ProblemSpec(*ts, **SEEDS)], c0=16, L=3, precision="bf16", sampling=law,
                          pilot_n=128) as plan:
            (Y,), (rep,) = plan.estimate([eps])
            V0[law] = rep["V"][0]
            assert np.linalg.norm(Y.cpu().numpy() - mu) <= 5 * rep["rmse_pred"]
    assert V0["optimal"] < V0["uniform"], V0
