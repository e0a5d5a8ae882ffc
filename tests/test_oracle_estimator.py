"""Pins of the oracle's estimator against the mathematics the paper fixes.

* Brute force over every index sequence (n <= 8, c <= 4) for a frozen realisation:
  the sketch of Eq. (matrixsketch) is unbiased for AB and its squared Frobenius error is
  (1/c)(n sum_k ||A_:k||^2 ||B_k:||^2 - ||AB||^2) (Thm 3.2 conditioned on A, B); the
  coupled difference of Alg. 1 has mean 0 and second moment (1/c_{l-1} - 1/c_l) times
  the same bracket.
* The coupling of Alg. 1: the coarse estimate reuses the draws r_{jR} of the fine one.
* Closed-form single-sample variances V_l of the Gaussian laws (Thm 3.2 with the
  expectation over A and B taken exactly) against the oracle's V_l.
* Unbiasedness of the estimator: E[Yhat] = E[A] E[B] = M M' (Eq. hatY), E[D_l] = 0 for l >= 1.
* Special cases: n = 1 (every sketch is exact, D_l = 0) and S = 0 (deterministic A, B).
* The N_l allocation of Remark 3.6 against a numerical constrained minimiser.
"""
import itertools

import numpy as np
import pytest
import scipy.optimize

import oracle
from paper_1904_00429_gb300.inputs import make_params


def _bracket(A, B):
    n = A.shape[1]
    colA = (A * A).sum(axis=0)
    rowB = (B * B).sum(axis=1)
    AB = A @ B
    return n * float(colA @ rowB) - float((AB * AB).sum())


@pytest.mark.parametrize("n,c,R", [(5, 4, 2), (8, 4, 2), (6, 4, 4), (7, 3, 3), (4, 2, 2)])
def test_bruteforce_sketch_and_coupled_difference(n, c, R):
    rng = np.random.default_rng(n * 100 + c)
    m, p = 3, 2
    A = rng.normal(size=(m, n)) + 0.5
    B = rng.normal(size=(n, p)) - 0.3
    AB = A @ B
    cc = c // R
    sum_Z = np.zeros((m, p))
    sum_err = 0.0
    sum_D = np.zeros((m, p))
    sum_D2 = 0.0
    seqs = list(itertools.product(range(n), repeat=c))
    for seq in seqs:
        idx = np.array(seq)
        Z = oracle.sketch(A, B, idx)
        sum_Z += Z
        sum_err += float(((Z - AB) ** 2).sum())
        coarse = oracle.sketch(A, B, idx, off=R - 1, stride=R, cnt=cc)
        D = Z - coarse
        sum_D += D
        sum_D2 += float((D * D).sum())
    N = len(seqs)
    scale = np.abs(A).max() * np.abs(B).max() * n
    np.testing.assert_allclose(sum_Z / N, AB, rtol=0, atol=1e-12 * scale)
    assert np.isclose(sum_err / N, _bracket(A, B) / c, rtol=1e-10)
    np.testing.assert_allclose(sum_D / N, 0.0, atol=1e-12 * scale)
    assert np.isclose(sum_D2 / N, (1.0 / cc - 1.0 / c) * _bracket(A, B), rtol=1e-10)


def _realised(pr, l, s, magnitudes=False):
    """The full realisation A, B of sample s at level l, entry by entry (tiny n only);
    with magnitudes=True, also |M| + |S||Z| and |M'| + |S'||Z'|."""
    sA, sB, _, pid = pr.seeds
    ZA = np.array([[oracle.normal(sA, pid, l, s, i, k) for k in range(pr.n)] for i in range(pr.m)])
    ZB = np.array([[oracle.normal(sB, pid, l, s, j, k) for j in range(pr.p)] for k in range(pr.n)])
    A, B = pr.M + pr.S * ZA, pr.Mp + pr.Sp * ZB
    if magnitudes:
        return A, B, np.abs(pr.M) + np.abs(pr.S * ZA), np.abs(pr.Mp) + np.abs(pr.Sp * ZB)
    return A, B


@pytest.mark.parametrize("R", [2, 3])
def test_sample_is_the_coupled_pair_of_one_realisation(R):
    pp = make_params(3, 6, 4, seed_A=4, seed_B=5)
    pr = oracle.Problem(*pp.f64(), seed_A=4, seed_B=5, seed_idx=6, problem_id=1)
    lv = oracle.Levels(2, R, 3)
    for l in range(4):
        for s in (0, 3, 2**33 + 1):
            c = lv.cl(l)
            idx = np.array([oracle.index(6, 1, l, s, t, pr.n) for t in range(c)])
            A, B, Aa, Ba = _realised(pr, l, s, magnitudes=True)
            D, Pf, Pc, mag = oracle.sample(pr, lv, l, s)
            np.testing.assert_allclose(Pf, oracle.sketch(A, B, idx), rtol=1e-13, atol=1e-13)
            if l == 0:
                assert np.all(Pc == 0)
            else:
                # coarse uses r_{jR}, j = 1..c/R (1-based), i.e. 0-based slots jR - 1
                sel = np.array([idx[j * R - 1] for j in range(1, c // R + 1)])
                np.testing.assert_allclose(Pc, oracle.sketch(A, B, sel), rtol=1e-13, atol=1e-13)
            np.testing.assert_array_equal(D, Pf - Pc)
            w = pr.n / c
            terms = Aa[:, idx] @ Ba[idx, :] * w
            if l > 0:
                terms += Aa[:, sel] @ Ba[sel, :] * (pr.n / (c // R))
            assert np.all(mag >= np.abs(Pf) + np.abs(Pc) - 1e-12 * mag)
            np.testing.assert_allclose(mag, terms, rtol=1e-12)


def test_nested_chain_telescopes():
    rng = np.random.default_rng(3)
    m, n, p, R, c0, L = 4, 9, 3, 2, 2, 4
    A, B = rng.normal(size=(m, n)), rng.normal(size=(n, p))
    cL = c0 * R**L
    idx = rng.integers(0, n, size=cL)
    P = []
    for l in range(L + 1):
        step = R ** (L - l)
        P.append(oracle.sketch(A, B, idx, off=step - 1, stride=step, cnt=c0 * R**l))
    total = P[0] + sum(P[l] - P[l - 1] for l in range(1, L + 1))
    np.testing.assert_allclose(total, P[L], rtol=1e-12, atol=1e-12)
    # the coarse half of each level is the fine estimate of the level below
    for l in range(1, L + 1):
        step = R ** (L - l)
        sub = idx[step - 1::step]
        np.testing.assert_allclose(oracle.sketch(A, B, sub, off=R - 1, stride=R, cnt=len(sub) // R), P[l - 1],
                                   rtol=1e-13, atol=1e-13)


def closed_form_V(M, S, Mp, Sp, c0, R, L):
    """V_l = E||D_l - E D_l||_F^2 for A = M + S o Z, B = M' + S' o Z' (independent N(0,1) Z):
    per entry Q = sum_k (M^2+S^2)(M'^2+S'^2), Rr = sum_k M^2 M'^2, mu = M M',
    K = n Q - Q + Rr - mu^2;  V_0 = sum (K / c0 + Q - Rr),  V_l = (1/c_{l-1} - 1/c_l) sum K."""
    n = M.shape[1]
    Q = (M**2 + S**2) @ (Mp**2 + Sp**2)
    Rr = (M**2) @ (Mp**2)
    mu = M @ Mp
    K = n * Q - Q + Rr - mu**2
    V = [float((K / c0 + Q - Rr).sum())]
    per_entry = [K / c0 + Q - Rr]
    for l in range(1, L + 1):
        c, cc = c0 * R**l, c0 * R ** (l - 1)
        V.append((1.0 / cc - 1.0 / c) * float(K.sum()))
        per_entry.append((1.0 / cc - 1.0 / c) * K)
    return np.array(V), per_entry


@pytest.mark.parametrize("zero_S", [False, True])
def test_level_variance_matches_closed_form(zero_S):
    pp = make_params(3, 8, 2, seed_A=10, seed_B=11)
    M, S, Mp, Sp = pp.f64()
    if zero_S:
        S, Sp = np.zeros_like(S), np.zeros_like(Sp)
    pr = oracle.Problem(M, S, Mp, Sp, seed_A=10, seed_B=11, seed_idx=12)
    lv = oracle.Levels(4, 2, 2)
    Vc, _ = closed_form_V(M, S, Mp, Sp, 4, 2, 2)
    N = 3000
    for l in range(3):
        mean, M2, _ = oracle.level_stats(pr, lv, l, 0, N)
        V = M2 / (N - 1)
        # sampling spread of V from the per-sample squared deviations
        sq = np.array([float(((oracle.sample(pr, lv, l, s)[0] - mean) ** 2).sum()) for s in range(N)])
        assert np.isclose(sq.sum(), M2, rtol=1e-10)
        z = (V - Vc[l]) / (sq.std() / np.sqrt(N))
        assert abs(z) < 5.0, (l, V, Vc[l], z)


def test_estimator_is_unbiased_and_differences_have_mean_zero():
    zs, zd = [], []
    c0, R, L, Nl = 2, 2, 2, [400, 200, 100]
    for rep in range(12):
        pp = make_params(3, 6, 2, seed_A=20 + rep, seed_B=40 + rep)
        M, S, Mp, Sp = pp.f64()
        pr = oracle.Problem(M, S, Mp, Sp, seed_A=20 + rep, seed_B=40 + rep, seed_idx=60 + rep)
        lv = oracle.Levels(c0, R, L)
        _, Vij = closed_form_V(M, S, Mp, Sp, c0, R, L)
        Y = np.zeros((3, 2))
        var = np.zeros((3, 2))
        for l in range(L + 1):
            mean, _, _ = oracle.level_stats(pr, lv, l, 0, Nl[l])
            Y += mean
            var += Vij[l] / Nl[l]
            if l > 0:
                zd.extend(((mean - 0.0) / np.sqrt(Vij[l] / Nl[l])).ravel())
        zs.extend(((Y - M @ Mp) / np.sqrt(var)).ravel())
    zs, zd = np.array(zs), np.array(zd)
    for z in (zs, zd):
        assert np.max(np.abs(z)) < 5.0
        assert 0.6 < np.mean(z**2) < 1.5


def test_n_equal_one_every_sketch_is_exact():
    pp = make_params(4, 1, 3, seed_A=1, seed_B=2)
    pr = oracle.Problem(*pp.f64())
    lv = oracle.Levels(4, 2, 3)
    for l in range(4):
        for s in range(5):
            D, Pf, Pc, mag = oracle.sample(pr, lv, l, s)
            A, B = _realised(pr, l, s)
            np.testing.assert_allclose(Pf, A @ B, rtol=1e-14, atol=1e-14)
            if l > 0:
                assert np.all(np.abs(D) <= 1e-14 * mag)


def test_allocation_is_the_constrained_optimum():
    V = np.array([50.0, 8.0, 3.0, 0.7, 0.2])
    C = np.array([4.0, 12.0, 24.0, 48.0, 96.0])
    eps = 0.05
    Nl = oracle.allocate(V, C, eps, pilot=0)
    # continuous minimiser of sum N_l C_l subject to sum V_l / N_l = eps^2 / 2 (units of 1e5 samples)
    u = 1e5
    cons = {"type": "eq", "fun": lambda x: (V / (u * x)).sum() / (eps**2 / 2) - 1.0}
    res = scipy.optimize.minimize(lambda x: float((x * C).sum()), np.ones(5), constraints=[cons],
                                  bounds=[(1e-6, 1e3)] * 5, method="SLSQP",
                                  options={"ftol": 1e-15, "maxiter": 1000})
    assert res.success
    opt = u * res.x
    np.testing.assert_allclose(Nl, np.ceil(opt), rtol=2e-3, atol=1)
    assert (V / Nl).sum() <= eps**2 / 2 * (1 + 1e-12)
    # scale and pilot floor
    half = oracle.allocate(V, C, eps, nl_scale=0.05, pilot=0)
    assert np.all(half <= np.ceil(Nl * 0.05) + 1)
    floored = oracle.allocate(V, C, eps, nl_scale=1e-6, pilot=256)
    assert np.all(floored == 256)
    with pytest.raises(ValueError):
        oracle.allocate(V, C, -1.0)


def test_estimate_follows_algorithm_2():
    pp = make_params(3, 16, 2, seed_A=3, seed_B=4)
    pr = oracle.Problem(*pp.f64(), seed_A=3, seed_B=4, seed_idx=5)
    lv = oracle.Levels(2, 2, 3)
    eps = 0.05 * np.linalg.norm(pp.exact_mean())
    Y, Nl, V, means = oracle.estimate(pr, lv, eps, pilot=32)
    assert np.all(Nl >= 32)
    # top-ups keep the pilot samples: level means equal statistics over samples 0..N_l-1
    for l in range(lv.L + 1):
        mean, M2, _ = oracle.level_stats(pr, lv, l, 0, int(Nl[l]))
        np.testing.assert_allclose(means[l], mean, rtol=1e-12, atol=1e-12)
        assert np.isclose(V[l], M2 / (Nl[l] - 1), rtol=1e-12)
    np.testing.assert_allclose(Y, means.sum(axis=0), rtol=1e-14)
    # the allocation met its own variance budget from the pilot variances
    C = np.array([lv.cost(l) for l in range(lv.L + 1)])
    assert np.all(np.diff(C) > 0)


def test_optimal_base_number_is_eleven():
    # Sec. 2.1: g(M) = (M+1)^2 / (M log^2 M) is minimised over integers M >= 2 at M = 11
    g = {M: (M + 1) ** 2 / (M * np.log(M) ** 2) for M in range(2, 40)}
    assert min(g, key=g.get) == 11
