"""Pins of the oracle's targeted function f (Sec. 3, f applied entrywise to each sketch) and of
Alg. 2's adaptive choice of the finest level L (Remark 3.5, Eq. L_num_bound_matrix).

No GPU.  The function is the one of the paper's matrix example (Sec. 5.2): f(x) = |x| H(2 - x)
with the Heaviside step H, H(0) = 1 (the paper leaves H(0) open).  The pins:
  * brute force: the draws of one realisation are rebuilt here from the oracle's already-pinned
    index and normal draws, the fine and coarse sketches are formed directly from their
    definition, and D must be f(P_l) - f(P_{l-1}) (not f(P_l - P_{l-1}), which the chosen
    case separates), and f(P_0) at level 0;
  * n = 1: every draw picks the only column, so P_l = P_{l-1} = A B (up to the rounding of
    summing c_l equal terms) and D_l = 0 for l >= 1 while D_0 = f(A B);
  * f = identity reproduces the pinned estimator of E[AB] bit for bit;
  * adaptive L: the loop stops at the first L >= 2 whose finest mean meets the bound.  Rounds are
    deterministic (fixed sample ids), so a run capped at L' < L reproduces the state of round L',
    whose finest mean must violate the bound, and the returned level must satisfy it.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def f_abs_step(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(2.0 - x >= 0.0, np.abs(x), 0.0)


def test_targeted_function_values():
    for x in (-3.5, -2.0, -0.25, 0.0, 0.7, 1.999, 2.0, 2.0000001, 7.0):
        assert oracle.f(oracle.F_ABS_STEP, x) == float(f_abs_step(x))
        assert oracle.f(oracle.F_IDENTITY, x) == x
    assert oracle.f(oracle.F_ABS_STEP, 2.0) == 2.0     # H(0) = 1


def _realisation(pr, l, s, c):
    """Indices and the sampled columns of A / rows of B of one realisation, from the draws."""
    idx = [oracle.index(pr.seeds[2], pr.seeds[3], l, s, t, pr.n) for t in range(c)]
    A = np.array([[pr.M[i, k] + pr.S[i, k] * oracle.normal(pr.seeds[0], pr.seeds[3], l, s, i, k)
                   for k in idx] for i in range(pr.m)])                       # m x c
    B = np.array([[pr.Mp[k, j] + pr.Sp[k, j] * oracle.normal(pr.seeds[1], pr.seeds[3], l, s, j, k)
                   for j in range(pr.p)] for k in idx])                       # c x p
    return idx, A, B


@pytest.mark.parametrize("l", [0, 1, 2])
def test_sample_f_brute_force(l):
    rng = np.random.default_rng(5)
    m, n, p = 3, 6, 2
    M = rng.uniform(-1, 1, (m, n))
    S = rng.uniform(0.1, 1, (m, n))
    Mp = rng.uniform(-1, 1, (n, p))
    Sp = rng.uniform(0.1, 1, (n, p))
    pr = oracle.Problem(M, S, Mp, Sp, seed_A=11, seed_B=12, seed_idx=13, problem_id=1)
    lv = oracle.Levels(2, 2, 3)
    separated = False
    for s in range(40):
        c = lv.cl(l)
        _, A, B = _realisation(pr, l, s, c)
        Pf = (n / c) * A @ B
        if l > 0:
            coarse = [t for t in range(c) if t % 2 == 1]   # slots t = jR - 1
            Pc = (n / (c // 2)) * A[:, coarse] @ B[coarse, :]
            want = f_abs_step(Pf) - f_abs_step(Pc)
            separated |= bool(np.any(np.abs(want - f_abs_step(Pf - Pc)) > 1e-6))
        else:
            Pc = np.zeros_like(Pf)
            want = f_abs_step(Pf)
        D, Pf_o, Pc_o, _ = oracle.sample(pr, lv, l, s, fkind=oracle.F_ABS_STEP)
        np.testing.assert_allclose(Pf_o, Pf, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Pc_o, Pc, rtol=1e-12, atol=1e-12)
        # f has a jump at 2: compare away from it
        far = (np.abs(Pf - 2.0) > 1e-9) & (np.abs(Pc - 2.0) > 1e-9)
        np.testing.assert_allclose(D[far], want[far], rtol=1e-12, atol=1e-12)
    if l > 0:
        assert separated   # the case tells f(P_l) - f(P_{l-1}) from f(P_l - P_{l-1})


def test_single_column_levels_cancel():
    rng = np.random.default_rng(6)
    m, p = 4, 3
    M, S = rng.uniform(-1, 1, (m, 1)), rng.uniform(0.1, 1, (m, 1))
    Mp, Sp = rng.uniform(-1, 1, (1, p)), rng.uniform(0.1, 1, (1, p))
    pr = oracle.Problem(M, S, Mp, Sp, seed_A=1, seed_B=2, seed_idx=3)
    lv = oracle.Levels(2, 2, 3)
    for s in range(5):
        _, A, B = _realisation(pr, 0, s, 1)
        D0 = oracle.sample(pr, lv, 0, s, fkind=oracle.F_ABS_STEP)[0]
        np.testing.assert_allclose(D0, f_abs_step(A @ B), rtol=1e-14, atol=0)
        for l in (1, 2, 3):
            D, Pf, _, _ = oracle.sample(pr, lv, l, s, fkind=oracle.F_ABS_STEP)
            # c_l equal products summed in FP64: c_l u of |P| at most
            assert np.all(np.abs(D) <= lv.cl(l) * 2.0**-52 * np.abs(Pf) + 1e-300)


def test_identity_is_the_estimator_of_EAB():
    rng = np.random.default_rng(7)
    m, n, p = 5, 40, 4
    M, S = rng.uniform(-1, 1, (m, n)), rng.uniform(0.1, 1, (m, n))
    Mp, Sp = rng.uniform(-1, 1, (n, p)), rng.uniform(0.1, 1, (n, p))
    pr = oracle.Problem(M, S, Mp, Sp)
    lv = oracle.Levels(4, 2, 3)
    eps = 0.1 * np.linalg.norm(M @ Mp)
    Y, Nl, V, means = oracle.estimate(pr, lv, eps, pilot=16)
    Y2, L2, Nl2, V2, means2 = oracle.estimate_f(pr, lv, eps, fkind=oracle.F_IDENTITY, adaptive=False, pilot=16)
    assert L2 == 3
    assert np.array_equal(Y, Y2) and np.array_equal(Nl, Nl2) and np.array_equal(V, V2)
    assert np.array_equal(means, means2)


def _bias_problem():
    # AB entries spread around the jump of f at 2, so E[f(P_l)] keeps changing with c_l
    rng = np.random.default_rng(9)
    m, n, p = 2, 16, 2
    M = rng.uniform(0.2, 0.6, (m, n))
    S = np.full((m, n), 0.3)
    Mp = rng.uniform(0.05, 0.35, (n, p))
    Sp = np.full((n, p), 0.1)
    return oracle.Problem(M, S, Mp, Sp, seed_A=21, seed_B=22, seed_idx=23)


def test_adaptive_L_stops_at_the_first_level_meeting_the_bound():
    pr = _bias_problem()
    R = 2
    eps = 0.02
    bound = (math.sqrt(R) + 1.0) * eps / math.sqrt(2.0)
    Y, L, Nl, V, means = oracle.estimate_f(pr, oracle.Levels(1, R, 12), eps, fkind=oracle.F_ABS_STEP,
                                           adaptive=True, pilot=64)
    assert 3 <= L < 12, L   # the case needs more than the minimum of three levels
    assert np.linalg.norm(means[L]) < bound
    np.testing.assert_allclose(Y, means.sum(axis=0), rtol=1e-12, atol=1e-15)
    for Lcap in range(2, L):
        Yc, Lc, Nc, Vc, mc = oracle.estimate_f(pr, oracle.Levels(1, R, Lcap), eps, fkind=oracle.F_ABS_STEP,
                                               adaptive=True, pilot=64)
        assert Lc == Lcap
        assert np.linalg.norm(mc[Lcap]) >= bound, (Lcap, np.linalg.norm(mc[Lcap]), bound)
    # the allocation of the last round: at least the pilot, the variance target met up to the
    # pilot floor and the variances' change after the top-up
    assert np.all(Nl >= 64)
    assert float(np.sum(V / Nl)) <= 1.5 * eps**2 / 2


def test_adaptive_identity_stops_at_three_levels():
    # f = identity: E[D_l] = 0 for l >= 1, so the finest mean is sampling noise below the bound
    rng = np.random.default_rng(10)
    m, n, p = 4, 64, 3
    M, S = rng.uniform(-1, 1, (m, n)), rng.uniform(0.1, 1, (m, n))
    Mp, Sp = rng.uniform(-1, 1, (n, p)), rng.uniform(0.1, 1, (n, p))
    pr = oracle.Problem(M, S, Mp, Sp)
    eps = 0.05 * np.linalg.norm(M @ Mp)
    Y, L, Nl, V, means = oracle.estimate_f(pr, oracle.Levels(2, 2, 8), eps, adaptive=True, pilot=32)
    assert L == 2
