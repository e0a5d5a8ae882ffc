"""Parity of the CUDA-core level kernels (FP64, FP32) with the FP64 CPU oracle, through the C ABI.

Bars (derived from the arithmetic):
  * Philox words and sampled indices: bit-exact.
  * FP64: every entry of a sample D within 1e-12 * mag, where mag is the oracle's
    sum over the products entering D of |w| (|M| + |S Z|)(|M'| + |S' Z'|); level means within
    1e-12 * mean(mag); M2 within 1e-12 relative.
  * FP32: |D - D_oracle| <= tau_32(c) * mag with tau_32(c) = (c + 8) 2^-24 + 2^-16:
    sequential accumulation of c products (c u), one rounding each for A, w B and the FP32
    weight, and 2^-16 for the generated normals (|dZ| <= 2^-20 rho with rho <= 6.8).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu

C1 = dict(m=64, n=1024, p=64, c0=16, L=5)
C1_NL = [2000, 1000, 500, 250, 125, 62]   # 2000 * 2^-l, floored


def tau32(c):
    return (c + 8) * 2.0**-24 + 2.0**-16


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _plan(pp, precision, c0, L, R=2, dtype=torch.float64, **kw):
    dev = torch.device("cuda:0")
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev, dtype) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    spec = binding.ProblemSpec(*ts, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)
    return binding.Plan([spec], c0=c0, L=L, ratio=R, precision=precision, **kw)


def _orc(pp):
    return oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                          problem_id=pp.problem_id)


def test_philox_words_bit_exact():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0] * 4, [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [7, 0, 0, 0]]
    key[:4] = [[0, 0], [0xFFFFFFFF] * 2, [0xA4093822, 0x299F31D0], [1, 2]]
    dev = torch.device("cuda:0")
    out = binding.debug_philox(torch.from_numpy(ctr.view(np.int32)).to(dev),
                               torch.from_numpy(key.view(np.int32)).to(dev))
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    ref = np.array([oracle.philox4x32(c, k) for c, k in zip(ctr, key)])
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("n", [1, 3, 1024, 65536])
def test_indices_bit_exact(n):
    dev = torch.device("cuda:0")
    M = torch.zeros(4, n, dtype=torch.float32, device=dev)
    Mp = torch.zeros(n, 4, dtype=torch.float32, device=dev)
    spec = binding.ProblemSpec(M, M.clone(), Mp, Mp.clone(), seed_idx=9, problem_id=3)
    with binding.Plan([spec], c0=3, L=6, precision="fp32") as plan:
        for l, s in [(0, 0), (3, 17), (6, 2**40 + 5)]:
            c = 3 * 2**l
            got = plan.debug_indices(0, l, s, 0, c).cpu().numpy()
            ref = np.array([oracle.index(9, 3, l, s, t, n) for t in range(c)])
            np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2.0**-19)])
def test_normals_match_oracle(precision, tol):
    pp = make_params(64, 256, 48, seed_A=5, seed_B=6, problem_id=2)
    with _plan(pp, precision, 16, 3, dtype=torch.float64 if precision == "fp64" else torch.float32) as plan:
        for which, seed, rows in [(0, 5, 64), (1, 6, 48)]:
            for l, s, k in [(0, 0, 0), (2, 99, 255), (3, 2**33 + 7, 128)]:
                z = plan.debug_normals(0, which, l, s, k, 0, rows).cpu().numpy()
                ref = np.array([oracle.normal(seed, 2, l, s, r, k) for r in range(rows)])
                assert np.all(np.abs(z - ref) <= tol * np.maximum(np.abs(ref), 1.0)), np.max(np.abs(z - ref))


def test_fp64_samples_match_oracle_C1():
    pp = make_params(C1["m"], C1["n"], C1["p"], seed_A=0, seed_B=1)
    orc = _orc(pp)
    lv = oracle.Levels(C1["c0"], 2, C1["L"])
    worst = 0.0
    with _plan(pp, "fp64", C1["c0"], C1["L"]) as plan:
        for l in range(C1["L"] + 1):
            for s in (0, 1, 9, 61):
                D = plan.debug_sample(0, l, s).cpu().numpy()
                Dref, _, _, mag = oracle.sample(orc, lv, l, s)
                r = np.max(np.abs(D - Dref) / mag)
                worst = max(worst, r)
                assert r <= 1e-12, (l, s, r)
    print(f"fp64 C1 samples: max |D - D_oracle| / mag = {worst:.3e}")


def test_fp64_level_statistics_match_oracle_C1():
    """The full C1 workload: N_l = 2000 * 2^-l samples per level, FP64."""
    pp = make_params(C1["m"], C1["n"], C1["p"], seed_A=0, seed_B=1)
    orc = _orc(pp)
    lv = oracle.Levels(C1["c0"], 2, C1["L"])
    with _plan(pp, "fp64", C1["c0"], C1["L"]) as plan:
        for l, N in enumerate(C1_NL):
            plan.level_stats(0, l, 0, N)
        for l, N in enumerate(C1_NL):
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 0, N)
            assert n_got == N
            err = np.abs(mean.cpu().numpy() - mref) / magm
            assert err.max() <= 1e-12, (l, err.max())
            assert abs(M2 - M2ref) <= 1e-12 * M2ref, (l, M2, M2ref)


def test_fp32_samples_match_oracle_at_scale():
    """The large workload's shapes (256 x 65536 x 256, c_l = 64 * 2^l), sampled outputs."""
    m, n, p = 256, 65536, 256
    pp = make_params(m, n, p, seed_A=0, seed_B=1, dtype=np.float32)
    orc = _orc(pp)
    lv = oracle.Levels(64, 2, 8)
    worst = 0.0
    with _plan(pp, "fp32", 64, 8, dtype=torch.float32) as plan:
        for l, s in [(0, 0), (0, 12345), (1, 3), (4, 77), (8, 5)]:
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, _, _, mag = oracle.sample(orc, lv, l, s)
            r = np.abs(D - Dref) / mag
            c = lv.cl(l)
            worst = max(worst, float(r.max()) / tau32(c))
            assert np.all(r <= tau32(c)), (l, s, r.max(), tau32(c))
    print(f"fp32 large-shape samples: max error / bound = {worst:.3e}")


def test_fp32_level_statistics_match_oracle_small():
    pp = make_params(64, 1024, 64, seed_A=0, seed_B=1, dtype=np.float32)
    orc = _orc(pp)
    lv = oracle.Levels(16, 2, 3)
    with _plan(pp, "fp32", 16, 3, dtype=torch.float32) as plan:
        for l in range(4):
            plan.level_stats(0, l, 0, 40)
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 0, 40)
            assert n_got == 40
            assert np.all(np.abs(mean.cpu().numpy() - mref) <= tau32(lv.cl(l)) * magm)
            assert abs(M2 - M2ref) <= 4 * tau32(lv.cl(l)) * M2ref


@pytest.mark.parametrize("tile", [128064, 128128])
@pytest.mark.parametrize("m,n,p", [(200, 3000, 130), (129, 500, 257)])
def test_fp32_wide_tiles_ragged(m, n, p, tile):
    """The FP32 128 x 64 and 128 x 128 tiles (f = identity): several tiles with ragged edges in
    both directions, sampled D and level statistics over several chunks."""
    pp = make_params(m, n, p, seed_A=31, seed_B=32, seed_idx=33, problem_id=1, dtype=np.float32)
    orc = _orc(pp)
    lv = oracle.Levels(16, 2, 3)
    with _plan(pp, "fp32", 16, 3, dtype=torch.float32, tile_override=tile) as plan:
        for l, s in [(0, 0), (1, 70), (3, 5)]:
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, _, _, mag = oracle.sample(orc, lv, l, s)
            assert np.all(np.abs(D - Dref) <= tau32(lv.cl(l)) * mag), (l, s)
        for l in range(4):
            plan.level_stats(0, l, 10, 150)
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 10, 150)
            assert n_got == 150
            assert np.all(np.abs(mean.cpu().numpy() - mref) <= tau32(lv.cl(l)) * magm), l
            assert abs(M2 - M2ref) <= 4 * tau32(lv.cl(l)) * M2ref, (l, M2, M2ref)


@pytest.mark.parametrize("m,n,p,c0,R,L", [(37, 1000, 53, 3, 3, 3), (1, 50, 1, 1, 2, 4), (130, 17, 5, 5, 2, 2)])
def test_fp64_ragged_shapes_and_ratios(m, n, p, c0, R, L):
    pp = make_params(m, n, p, seed_A=11, seed_B=12, seed_idx=13, problem_id=4)
    orc = _orc(pp)
    lv = oracle.Levels(c0, R, L)
    with _plan(pp, "fp64", c0, L, R=R) as plan:
        for l in range(L + 1):
            for s in (0, 5, 8):
                D = plan.debug_sample(0, l, s).cpu().numpy()
                Dref, _, _, mag = oracle.sample(orc, lv, l, s)
                assert np.all(np.abs(D - Dref) <= 1e-12 * mag), (l, s)


def test_n_equal_one_differences_vanish():
    pp = make_params(8, 1, 8)
    orc = _orc(pp)
    lv = oracle.Levels(4, 2, 3)
    with _plan(pp, "fp64", 4, 3) as plan:
        for l in range(1, 4):
            D = plan.debug_sample(0, l, 3).cpu().numpy()
            _, _, _, mag = oracle.sample(orc, lv, l, 3)
            assert np.all(np.abs(D) <= 1e-13 * mag)


def test_split_calls_and_checkpoint_resume_are_bit_identical():
    pp = make_params(64, 1024, 64, seed_A=3, seed_B=4)
    with _plan(pp, "fp64", 16, 2) as one, _plan(pp, "fp64", 16, 2) as two, _plan(pp, "fp64", 16, 2) as three:
        one.level_stats(0, 2, 0, 192)
        two.level_stats(0, 2, 0, 64)
        two.level_stats(0, 2, 64, 128)
        N, s, q = two.get_level_state(0, 2)
        three.set_level_state(0, 2, N, s, q)   # resume in another plan from the checkpoint
        three.reset(0, 1)
        N1, s1, q1 = one.get_level_state(0, 2)
        N2, s2, q2 = two.get_level_state(0, 2)
        assert N1 == N2 == 192 and q1 == q2 and torch.equal(s1, s2)
        N3, s3, q3 = three.get_level_state(0, 2)
        assert N3 == 192 and q3 == q1 and torch.equal(s3, s1)
        # a split that is not at a multiple of 8 agrees up to rounding
        four = _plan(pp, "fp64", 16, 2)
        four.level_stats(0, 2, 0, 13)
        four.level_stats(0, 2, 13, 179)
        _, s4, q4 = four.get_level_state(0, 2)
        torch.testing.assert_close(s4, s1, rtol=1e-13, atol=1e-10)
        assert abs(q4 - q1) <= 1e-13 * q1
        four.close()


def test_estimate_matches_oracle_algorithm_2():
    pp = make_params(32, 512, 24, seed_A=7, seed_B=8)
    orc = _orc(pp)
    lv = oracle.Levels(8, 2, 3)
    eps = 0.2 * np.linalg.norm(pp.exact_mean())
    Yref, Nref, Vref, means = oracle.estimate(orc, lv, eps, pilot=32)
    with _plan(pp, "fp64", 8, 3, pilot_n=32) as plan:
        (Y,), (rep,) = plan.estimate([eps])
        assert rep["N"] == list(Nref)
        np.testing.assert_allclose(rep["V"], Vref, rtol=1e-11)
        mags = np.zeros_like(Yref)
        for l in range(4):
            mags += oracle.level_stats(orc, lv, l, 0, int(Nref[l]))[2]
        assert np.all(np.abs(Y.cpu().numpy() - Yref) <= 1e-12 * mags)
        # N_l were sized from the pilot variances; with the final V_l the predicted RMSE is
        # eps / sqrt(2) up to the sampling error of those variances
        assert rep["rmse_pred"] <= 1.2 * eps / np.sqrt(2)


def test_multi_problem_plan():
    pps = [make_params(40, 300, 20, seed_A=1, seed_B=2, problem_id=0),
           make_params(17, 900, 66, seed_A=1, seed_B=2, problem_id=1)]
    dev = torch.device("cuda:0")
    specs = [binding.ProblemSpec(*(torch.from_numpy(x).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)),
                                 seed_A=1, seed_B=2, seed_idx=2, problem_id=q, L=q + 1)
             for q, pp in enumerate(pps)]
    with binding.Plan(specs, c0=4, L=3, precision="fp64") as plan:
        for q, pp in enumerate(pps):
            orc = oracle.Problem(*pp.f64(), seed_A=1, seed_B=2, seed_idx=2, problem_id=q)
            lv = oracle.Levels(4, 2, q + 1)
            for l in range(q + 2):
                D = plan.debug_sample(q, l, 3).cpu().numpy()
                Dref, _, _, mag = oracle.sample(orc, lv, l, 3)
                assert np.all(np.abs(D - Dref) <= 1e-12 * mag)


def test_errors_are_reported_not_raised_in_c():
    pp = make_params(8, 16, 8)
    with _plan(pp, "fp64", 2, 2) as plan:
        with pytest.raises(binding.MLMCError) as e:
            plan.level_stats(0, 3, 0, 8)
        assert e.value.status == 1
        with pytest.raises(binding.MLMCError) as e:
            plan.backward([torch.zeros(8, 8, device="cuda:0", dtype=torch.float64)])
        assert e.value.status == 7
        plan.level_stats(0, 1, 0, 0)          # empty range: no-op
        assert plan.get_level_stats(0, 1)[0] == 0
        with pytest.raises(binding.MLMCError) as e:
            plan.estimate([-1.0])
        assert e.value.status == 1
    with pytest.raises(binding.MLMCError) as e:
        _plan(pp, "fp64", 0, 2)
    assert e.value.status == 1
