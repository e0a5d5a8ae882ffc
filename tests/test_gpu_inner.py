"""Parity of the inner-product kernel (m = p = 1, Sec. 2) with the FP64 oracle, through the C ABI.

FP64/FP32 plans of a problem with m = p = 1 run level_inner_kernel (one warp per sample).  Bars
as for the general CUDA-core kernel: FP64 |D - D_oracle| <= 1e-12 mag, FP32 <= tau_32(c) mag with
tau_32(c) = (c + 8) 2^-24 + 2^-16 (the lanes' partial sums add in a tree instead of in slot order,
which keeps the error of c products within c u); level means within the same bars of the mean
magnitude, M2 within 1e-12 (FP64) or 4 tau_32 (FP32) relative; a targeted function (|x| H(2 - x))
applied to the fine and coarse sums apart, samples whose sums lie within the bar of the jump at 2
left out; and Alg. 2 end to end gives the oracle's N_l (FP64).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu


def tau32(c):
    return (c + 8) * 2.0**-24 + 2.0**-16


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _plan(pp, precision, c0, L, R=2, **kw):
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev, dt) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    spec = binding.ProblemSpec(*ts, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)
    return binding.Plan([spec], c0=c0, L=L, ratio=R, precision=precision, **kw)


def _orc(pp):
    return oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                          problem_id=pp.problem_id)


CASES = [(50, 1, 2, 4, [(0, 0), (1, 3), (4, 17)]),          # c0 = 1: odd slot counts, n < c_L
         (65536, 64, 2, 8, [(0, 5), (3, 100), (8, 2)]),     # the headline's n and levels
         (1000, 3, 3, 3, [(0, 1), (2, 7), (3, 9)])]         # ratio 3


@pytest.mark.parametrize("n,c0,R,L,picks", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_inner_samples_and_levels_match_oracle(n, c0, R, L, picks, precision):
    dt = np.float64 if precision == "fp64" else np.float32
    pp = make_params(1, n, 1, seed_A=7, seed_B=8, seed_idx=9, problem_id=3, dtype=dt)
    orc = _orc(pp)
    lv = oracle.Levels(c0, R, L)
    with _plan(pp, precision, c0, L, R) as plan:
        for l, s in picks:
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, _, _, mag = oracle.sample(orc, lv, l, s)
            tol = 1e-12 if precision == "fp64" else tau32(lv.cl(l))
            assert np.all(np.abs(D - Dref) <= tol * mag), (l, s, float(np.abs(D - Dref).max() / mag.max()))
        for l in range(min(L, 3) + 1):
            N = 77
            plan.level_stats(0, l, 5, N)
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 5, N)
            tol = 1e-12 if precision == "fp64" else tau32(lv.cl(l))
            assert n_got == N
            assert np.all(np.abs(mean.cpu().numpy() - mref) <= tol * magm)
            bar = 1e-12 if precision == "fp64" else 4 * tau32(lv.cl(l))
            assert abs(M2 - M2ref) <= bar * M2ref, (l, M2, M2ref)


def test_inner_targeted_function_fp64():
    # a scaled so that a b straddles the jump of f at 2
    pp = make_params(1, 4096, 1, seed_A=11, seed_B=12, seed_idx=13, problem_id=0)
    pp.M[:] = pp.M * (2.0 / np.sqrt(4096)) + 2.0 / 4096
    pp.S[:] = pp.S * (2.0 / np.sqrt(4096))
    orc = _orc(pp)
    lv = oracle.Levels(16, 2, 4)
    near = 0
    with _plan(pp, "fp64", 16, 4, f="abs_step") as plan:
        for l in range(5):
            for s in range(20):
                D = plan.debug_sample(0, l, s).cpu().numpy()
                Dref, Pf, Pc, mag = oracle.sample(orc, lv, l, s, fkind=oracle.F_ABS_STEP)
                band = 1e-9 * mag
                far = (np.abs(Pf - 2.0) > band) & ((np.abs(Pc - 2.0) > band) | (l == 0))
                near += int((~far).sum())
                assert np.all(np.abs(D - Dref)[far] <= 1e-12 * mag[far]), (l, s)
    assert near <= 2


def test_inner_estimate_matches_oracle_algorithm_2():
    pp = make_params(1, 2048, 1, seed_A=21, seed_B=22, seed_idx=23, problem_id=0)
    eps = 0.02 * abs(float(pp.exact_mean()[0, 0])) + 0.5
    orc = _orc(pp)
    Yref, Nref, Vref, _ = oracle.estimate(orc, oracle.Levels(8, 2, 3), eps, pilot=64)
    with _plan(pp, "fp64", 8, 3, pilot_n=64) as plan:
        (Y,), (rep,) = plan.estimate([eps])
    assert list(rep["N"]) == list(Nref)
    assert abs(float(Y.cpu().numpy()[0, 0]) - float(Yref[0, 0])) <= 1e-10 * max(1.0, abs(float(Yref[0, 0])))
