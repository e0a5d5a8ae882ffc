"""Targeted function f and adaptive L (Alg. 2) on the GPU, through the C ABI, against the oracle.

f(x) = |x| H(2 - x) (the paper's matrix example, H(0) = 1) is applied to the fine and the coarse
estimate of each sample apart: D = f(P_l) - f(P_{l-1}), by the CUDA-core kernel (FP64, FP32) and by
the tensor-core kernel (BF16 operands; the fine and coarse sums in two tensor-memory accumulators).

Bars:
  * FP64: |D - D_oracle| <= 1e-12 * mag entrywise, where mag bounds the rounding of P_l and
    P_{l-1} (f is 1-Lipschitz away from its jump); entries whose P_l or P_{l-1} lies within
    1e-9 * mag of the jump at 2 are excluded (there the two sides may take different branches);
  * FP32: the same with tau_32(c) = (c + 8) 2^-24 + 2^-16 in place of 1e-12, and the band widened
    to tau_32(c) * mag (the branch is decided in FP32 on the GPU and in FP64 in the oracle);
  * adaptive FP64 estimate: the same finest level and N_l as the oracle's Alg. 2, V_l within
    1e-11 relative, the estimate within 1e-12 of the summed level magnitudes;
  * BF16: against the plain oracle |D - D_oracle| <= tau_bf16(c) * mag away from the jump (band
    tau_bf16(c) * mag), tau_bf16(c) = 2^-7 + 2^-15 + (c + 8) 2^-23 (both operands rounded to
    bfloat16, FP32 generation and accumulation; f is 1-Lipschitz away from its jump, and mag bounds
    the fine and the coarse sums together); against the oracle's bf16 emulation at least 90 % of
    those entries within tau_acc(c) * mag, tau_acc(c) = (c + 8) 2^-23 + 2^-16 (terms whose FP32 and
    FP64 values round to different bfloat16 neighbours are the exception).  Level statistics: the
    mean within 64 2^-24 mean|D| of the mean of the kernel's own samples (FP32 running sums of at
    most 64 samples per chunk), M2 within 1e-4 relative of theirs (FP32 Welford terms).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def tau32(c):
    return (c + 8) * 2.0**-24 + 2.0**-16


def _plan(M, S, Mp, Sp, dtype, precision, c0, L, seeds=(3, 4, 5, 1), **kw):
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype) for x in (M, S, Mp, Sp)]
    spec = binding.ProblemSpec(*ts, seed_A=seeds[0], seed_B=seeds[1], seed_idx=seeds[2], problem_id=seeds[3])
    return binding.Plan([spec], c0=c0, L=L, ratio=2, precision=precision, f="abs_step", **kw)


CASES = [
    # m, n, p, c0, L, (level, sample) pairs; entries scaled so that AB straddles the jump at 2
    (64, 1024, 64, 16, 3, [(0, 0), (1, 3), (3, 9)]),
    (37, 1000, 53, 4, 3, [(0, 1), (2, 8), (3, 2)]),     # ragged tiles
    (130, 300, 70, 1, 4, [(0, 0), (1, 2), (4, 7)]),      # c0 = 1, odd slot counts
]


def _params(m, n, p, dtype):
    pp = make_params(m, n, p, seed_A=3, seed_B=4, seed_idx=5, problem_id=1, dtype=dtype)
    # scale so that the entries of AB are O(1) around the jump of f
    k = 2.0 / math.sqrt(n)
    return (pp.M * k + 2.0 / n).astype(dtype), (pp.S * k).astype(dtype), pp.Mp.astype(dtype), pp.Sp.astype(dtype)


@pytest.mark.parametrize("m,n,p,c0,L,picks", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_samples_match_oracle(m, n, p, c0, L, picks, precision):
    dtype = np.float64 if precision == "fp64" else np.float32
    M, S, Mp, Sp = _params(m, n, p, dtype)
    orc = oracle.Problem(M.astype(np.float64), S.astype(np.float64), Mp.astype(np.float64), Sp.astype(np.float64),
                         seed_A=3, seed_B=4, seed_idx=5, problem_id=1)
    lv = oracle.Levels(c0, 2, L)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    near = 0
    with _plan(M, S, Mp, Sp, tdt, precision, c0, L) as plan:
        for l, s in picks:
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, Pf, Pc, mag = oracle.sample(orc, lv, l, s, fkind=oracle.F_ABS_STEP)
            tol = 1e-12 if precision == "fp64" else tau32(lv.cl(l))
            band = (1e-9 if precision == "fp64" else tol) * mag
            far = (np.abs(Pf - 2.0) > band) & ((np.abs(Pc - 2.0) > band) | (l == 0))
            near += int((~far).sum())
            err = np.abs(D - Dref)[far] / mag[far]
            assert np.all(err <= tol), (l, s, err.max(), tol)
            assert np.mean(np.abs(Dref) > 0) > 0.3   # f is not trivially zero here
    assert near <= 0.01 * m * p * len(picks)


def tau_bf16(c):
    return 2.0**-7 + 2.0**-15 + (c + 8) * 2.0**-23


def tau_acc(c):
    return (c + 8) * 2.0**-23 + 2.0**-16


BF16_CASES = [
    (64, 1024, 64, 16, 3, [(0, 0), (1, 3), (3, 9)]),
    (37, 1000, 53, 4, 3, [(0, 1), (2, 8), (3, 2)]),       # ragged tiles; c_l = 4 .. 32: partial sub-blocks
    (130, 300, 70, 1, 4, [(0, 0), (1, 2), (4, 7)]),        # c0 = 1, odd slot counts, two row tiles
    (64, 4096, 200, 64, 3, [(0, 2), (3, 5)]),              # 128-column tiles, c_l up to 512
]


@pytest.mark.parametrize("m,n,p,c0,L,picks", BF16_CASES)
def test_bf16_samples_match_oracle(m, n, p, c0, L, picks):
    M, S, Mp, Sp = _params(m, n, p, np.float32)
    orc = oracle.Problem(M.astype(np.float64), S.astype(np.float64), Mp.astype(np.float64), Sp.astype(np.float64),
                         seed_A=3, seed_B=4, seed_idx=5, problem_id=1)
    lv = oracle.Levels(c0, 2, L)
    near = total = 0
    with _plan(M, S, Mp, Sp, torch.float32, "bf16", c0, L) as plan:
        for l, s in picks:
            c = lv.cl(l)
            D = plan.debug_sample(0, l, s).cpu().numpy().astype(np.float64)
            Dref, Pf, Pc, mag = oracle.sample(orc, lv, l, s, fkind=oracle.F_ABS_STEP)
            Demu, _, _, _ = oracle.sample(orc, lv, l, s, quant=oracle.QUANT_BF16, fkind=oracle.F_ABS_STEP)
            band = tau_bf16(c) * mag
            far = (np.abs(Pf - 2.0) > band) & ((np.abs(Pc - 2.0) > band) | (l == 0))
            near += int((~far).sum())
            total += m * p
            plain = np.abs(D - Dref)[far] / mag[far]
            assert np.all(plain <= tau_bf16(c)), (l, s, plain.max(), tau_bf16(c))
            emu = np.abs(D - Demu)[far] / mag[far]
            assert np.mean(emu <= tau_acc(c)) >= 0.9, (l, s, np.mean(emu <= tau_acc(c)))
            assert np.mean(np.abs(Dref) > 0) > 0.3   # f is not trivially zero here
    assert near <= 0.25 * total, (near, total)   # the bf16 band is wide: most entries still checked


def test_bf16_level_statistics():
    m, n, p = 64, 1024, 64
    M, S, Mp, Sp = _params(m, n, p, np.float32)
    orc = oracle.Problem(M.astype(np.float64), S.astype(np.float64), Mp.astype(np.float64), Sp.astype(np.float64),
                         seed_A=3, seed_B=4, seed_idx=5, problem_id=1)
    lv = oracle.Levels(16, 2, 3)
    with _plan(M, S, Mp, Sp, torch.float32, "bf16", 16, 3) as plan:
        for l, N in enumerate([150, 100, 70, 40]):
            plan.level_stats(0, l, 0, N)
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mean = mean.cpu().numpy()
            Ds = np.stack([plan.debug_sample(0, l, s).cpu().numpy().astype(np.float64) for s in range(N)])
            mu = Ds.mean(axis=0)
            M2own = float(((Ds - mu) ** 2).sum())
            assert n_got == N
            assert np.all(np.abs(mean - mu) <= 64 * 2.0**-24 * np.abs(Ds).mean(axis=0)), l
            assert abs(M2 - M2own) <= 1e-4 * M2own, (l, M2, M2own)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 0, N, quant=oracle.QUANT_BF16,
                                                   fkind=oracle.F_ABS_STEP)
            close = np.abs(mean - mref) <= tau_acc(lv.cl(l)) * magm
            assert close.mean() >= 0.9, (l, close.mean())
            assert abs(M2 - M2ref) <= 0.05 * M2ref, (l, M2, M2ref)


def test_bf16_adaptive_estimate_matches_emulating_oracle():
    M, S, Mp, Sp = _bias_params()
    M, S, Mp, Sp = (x.astype(np.float32) for x in (M, S, Mp, Sp))
    orc = oracle.Problem(*(x.astype(np.float64) for x in (M, S, Mp, Sp)), seed_A=21, seed_B=22, seed_idx=23)
    eps = 0.02
    Yref, Lref, Nref, _, _ = oracle.estimate_f(orc, oracle.Levels(16, 2, 8), eps, fkind=oracle.F_ABS_STEP,
                                               adaptive=True, pilot=64, quant=oracle.QUANT_BF16)
    with _plan(M, S, Mp, Sp, torch.float32, "bf16", 16, 8, seeds=(21, 22, 23, 0), pilot_n=64,
               adaptive_L=True) as plan:
        (Y,), (rep,) = plan.estimate([eps])
    # the same samples up to FP32 accumulation: the same finest level, N_l within a few percent
    assert rep["L"] == Lref and not rep["bias_unmet"]
    assert np.all(np.abs(np.array(rep["N"]) - Nref) <= 0.05 * Nref + 2), (rep["N"], list(Nref))
    assert np.linalg.norm(Y.cpu().numpy() - Yref) <= 0.5 * eps
    print(f"bf16 adaptive L = {rep['L']}, N_l = {rep['N']} (oracle {list(Nref)})")


def test_level_statistics_match_oracle_fp64():
    M, S, Mp, Sp = _params(48, 512, 40, np.float64)
    orc = oracle.Problem(M, S, Mp, Sp, seed_A=3, seed_B=4, seed_idx=5, problem_id=1)
    lv = oracle.Levels(8, 2, 3)
    with _plan(M, S, Mp, Sp, torch.float64, "fp64", 8, 3) as plan:
        for l, N in enumerate([200, 120, 70, 33]):
            plan.level_stats(0, l, 0, N)
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 0, N, fkind=oracle.F_ABS_STEP)
            assert n_got == N
            assert np.all(np.abs(mean.cpu().numpy() - mref) <= 1e-12 * magm), l
            assert abs(M2 - M2ref) <= 1e-11 * M2ref, (l, M2, M2ref)


def _bias_params():
    rng = np.random.default_rng(9)
    m, n, p = 2, 16, 2
    M = rng.uniform(0.2, 0.6, (m, n))
    S = np.full((m, n), 0.3)
    Mp = rng.uniform(0.05, 0.35, (n, p))
    Sp = np.full((n, p), 0.1)
    return M, S, Mp, Sp


def test_adaptive_L_matches_oracle_algorithm_2():
    M, S, Mp, Sp = _bias_params()
    orc = oracle.Problem(M, S, Mp, Sp, seed_A=21, seed_B=22, seed_idx=23)
    eps = 0.02
    Yref, Lref, Nref, Vref, means = oracle.estimate_f(orc, oracle.Levels(1, 2, 12), eps, fkind=oracle.F_ABS_STEP,
                                                      adaptive=True, pilot=64)
    with _plan(M, S, Mp, Sp, torch.float64, "fp64", 1, 12, seeds=(21, 22, 23, 0), pilot_n=64,
               adaptive_L=True) as plan:
        (Y,), (rep,) = plan.estimate([eps])
        assert rep["L"] == Lref and not rep["bias_unmet"]
        assert rep["N"] == list(Nref)
        np.testing.assert_allclose(rep["V"], Vref, rtol=1e-11)
        mags = np.zeros_like(Yref)
        for l in range(Lref + 1):
            mags += oracle.level_stats(orc, oracle.Levels(1, 2, 12), l, 0, int(Nref[l]),
                                       fkind=oracle.F_ABS_STEP)[2]
        assert np.all(np.abs(Y.cpu().numpy() - Yref) <= 1e-12 * mags)
    print(f"adaptive L = {Lref}, N_l = {list(Nref)}")


def test_adaptive_L_capped_reports_unmet_bias():
    M, S, Mp, Sp = _bias_params()
    with _plan(M, S, Mp, Sp, torch.float64, "fp64", 1, 4, seeds=(21, 22, 23, 0), pilot_n=64,
               adaptive_L=True) as plan:
        (_,), (rep,) = plan.estimate([0.02])
        assert rep["L"] == 4 and rep["bias_unmet"]


def test_adaptive_identity_bf16_stops_at_three_levels():
    pp = make_params(64, 1024, 64, seed_A=0, seed_B=1, dtype=np.float32)
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(DEV) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    eps = 0.05 * np.linalg.norm(pp.exact_mean())
    with binding.Plan([binding.ProblemSpec(*ts)], c0=16, L=5, precision="bf16", pilot_n=64,
                      adaptive_L=True) as plan:
        (Y,), (rep,) = plan.estimate([eps])
        assert rep["L"] == 2 and not rep["bias_unmet"]
        assert np.linalg.norm(Y.cpu().numpy() - pp.exact_mean()) <= 5 * rep["rmse_pred"]


def test_unsupported_combinations():
    pp = make_params(16, 64, 16, dtype=np.float32)
    ts = [torch.from_numpy(x).to(DEV) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    with pytest.raises(binding.MLMCError) as e:
        binding.Plan([binding.ProblemSpec(*ts)], c0=4, L=2, precision="fp8", f="abs_step")
    assert e.value.status == 6
    with pytest.raises(binding.MLMCError) as e:   # the targeted-function form takes 128-row tiles
        binding.Plan([binding.ProblemSpec(*ts)], c0=4, L=2, precision="bf16", f="abs_step", tile_override=2064)
    assert e.value.status == 1
    with binding.Plan([binding.ProblemSpec(*ts)], c0=4, L=2, precision="fp32", f="abs_step") as plan:
        for l in range(3):
            plan.level_stats(0, l, 0, 8)
        plan.telescoping_sum()
        with pytest.raises(binding.MLMCError) as e:
            plan.backward([torch.zeros(16, 16, device=DEV, dtype=torch.float64)])
        assert e.value.status == 6
