"""Pins of the oracle's variance-optimal sampling law xi** (Thm 3.1, Eq. optproM).  No GPU.

  * the weights: xi**_j proportional to sqrt(E||A_{:,j}||^2 E||B_{j,:}||^2) with E[(M + S Z)^2]
    = M^2 + S^2, summing to one; a column whose parameters are all zero is never drawn;
  * the draw is the inverse of the cumulative law: rebuilt here from the (already pinned) Philox
    words by a linear scan; the histogram of 2e5 draws passes a chi-square test against xi**;
  * the sketch (1/c) sum_t A[:, r_t] B[r_t, :] / xi_{r_t} (Eq. matrixsketch): enumerating every
    index sequence of a frozen realisation (n = 3, c = 2) with its probability gives E[Z] = AB
    and E||Z - AB||^2 = (1/c)(sum_k ||a_k||^2 ||b_k||^2 / xi_k - ||AB||^2) exactly, and the
    oracle's own sample equals Z of the sequence it drew;
  * Thm 3.1: over the entry laws as well, the level-0 variance is mu_bar / c plus the spread of
    AB, mu_bar = (sum_j sqrt(E||A_j||^2 E||B_j||^2))^2 - E||AB||^2, and it is below the uniform
    law's (Thm 3.2: (n nu_bar + mu_bar) / c) on columns of unequal size;
  * the coupling keeps level differences centred: E[D_l] = 0 for l >= 1 (z-test).
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def _problem(m=3, n=12, p=2, seed=3, zero_col=None, skew=True, **kw):
    rng = np.random.default_rng(seed)
    scale = np.linspace(0.2, 2.0, n) if skew else np.ones(n)   # columns of unequal size
    M = rng.uniform(-1, 1, (m, n)) * scale
    S = rng.uniform(0.1, 1, (m, n)) * scale
    Mp = rng.uniform(-1, 1, (n, p))
    Sp = rng.uniform(0.1, 1, (n, p))
    if zero_col is not None:
        M[:, zero_col] = 0.0
        S[:, zero_col] = 0.0
    return oracle.Problem(M, S, Mp, Sp, seed_A=5, seed_B=6, seed_idx=7, problem_id=2, **kw)


def test_weights_follow_the_definition():
    pr = _problem(sampling="optimal", zero_col=4)
    ea = (pr.M**2 + pr.S**2).sum(axis=0)
    eb = (pr.Mp**2 + pr.Sp**2).sum(axis=1)
    q = np.sqrt(ea * eb)
    np.testing.assert_allclose(pr.q, q, rtol=1e-15)
    np.testing.assert_allclose(pr.Q, np.cumsum(q), rtol=1e-14)
    assert abs(pr.xi.sum() - 1.0) < 1e-14 and pr.xi[4] == 0.0


def _draw_by_scan(pr, l, s, t):
    w = oracle.philox4x32([t >> 1, 0xFFFFFFFF, s & 0xFFFFFFFF, ((s >> 32) << 8) | l], [pr.seeds[2], pr.seeds[3]])
    word = (int(w[3]) << 32 | int(w[2])) if t & 1 else (int(w[1]) << 32 | int(w[0]))
    x = float(word >> 11) * 2.0**-53 * pr.Q[-1]
    for j in range(pr.n):
        if x < pr.Q[j]:
            return j
    return max(j for j in range(pr.n) if pr.q[j] > 0)


def test_draw_inverts_the_cumulative_law():
    pr = _problem(sampling="optimal", zero_col=0)
    for (l, s, t) in [(0, 0, 0), (0, 0, 1), (2, 17, 5), (5, 123456789, 30), (1, 2**40 + 3, 7)]:
        assert oracle.index_xi(pr, l, s, t) == _draw_by_scan(pr, l, s, t)


def test_draws_follow_xi_star_star():
    pr = _problem(sampling="optimal", zero_col=6)
    counts = np.zeros(pr.n)
    draws = 0
    for s in range(2000):
        for t in range(100):
            counts[oracle.index_xi(pr, 1, s, t)] += 1
            draws += 1
    assert counts[6] == 0
    expect = pr.xi * draws
    keep = expect > 0
    chi2 = float((((counts - expect) ** 2)[keep] / expect[keep]).sum())
    dof = int(keep.sum()) - 1
    # chi-square with 10 degrees of freedom: P(chi2 > 35) < 1e-4
    assert chi2 < 35.0, (chi2, dof)


def test_sketch_enumeration_of_a_frozen_realisation():
    pr = _problem(m=2, n=3, p=2, sampling="optimal")
    lv = oracle.Levels(2, 2, 1)
    l, s = 0, 11
    xi = pr.xi
    # the realisation: column k of A and row k of B at (l, s) do not depend on where k is drawn
    A = np.array([[pr.M[i, k] + pr.S[i, k] * oracle.normal(pr.seeds[0], pr.seeds[3], l, s, i, k)
                   for k in range(pr.n)] for i in range(pr.m)])
    B = np.array([[pr.Mp[k, j] + pr.Sp[k, j] * oracle.normal(pr.seeds[1], pr.seeds[3], l, s, j, k)
                   for j in range(pr.p)] for k in range(pr.n)])
    AB = A @ B
    c = 2
    mean = np.zeros_like(AB)
    second = 0.0
    for seq in itertools.product(range(pr.n), repeat=c):
        prob = np.prod([xi[r] for r in seq])
        Z = sum(np.outer(A[:, r], B[r, :]) / xi[r] for r in seq) / c
        mean += prob * Z
        second += prob * float(np.sum((Z - AB) ** 2))
    np.testing.assert_allclose(mean, AB, rtol=1e-12, atol=1e-14)
    norms = np.array([np.sum(A[:, k] ** 2) * np.sum(B[k, :] ** 2) for k in range(pr.n)])
    exact = (float(np.sum(norms / xi)) - float(np.sum(AB**2))) / c
    assert abs(second - exact) <= 1e-12 * exact
    # the oracle's sample of this (l, s) is Z of the sequence it drew
    seq = [oracle.index_xi(pr, l, s, t) for t in range(c)]
    Z = sum(np.outer(A[:, r], B[r, :]) / xi[r] for r in seq) / c
    _, Pf, _, _ = oracle.sample(pr, lv, l, s)
    np.testing.assert_allclose(Pf, Z, rtol=1e-12, atol=1e-14)


def _closed_form_V0(pr, c, optimal):
    ea = (pr.M**2 + pr.S**2).sum(axis=0)
    eb = (pr.Mp**2 + pr.Sp**2).sum(axis=1)
    root = np.sqrt(ea * eb)
    # E||AB||^2 and the spread of AB about MM'
    EA2, EB2 = pr.M**2 + pr.S**2, pr.Mp**2 + pr.Sp**2
    spread = float(np.sum(EA2 @ EB2 - (pr.M**2) @ (pr.Mp**2)))
    EAB2 = spread + float(np.sum((pr.M @ pr.Mp) ** 2))
    mu_bar = float(root.sum()) ** 2 - EAB2
    nu_bar = float(np.sum((root - root.mean()) ** 2))
    err = mu_bar / c if optimal else (pr.n * nu_bar + mu_bar) / c
    return err + spread     # Var(Z) = E||Z - AB||^2 + E||AB - MM'||^2


def test_theorem_3_1_level_zero_variance():
    c = 4
    lv = oracle.Levels(c, 2, 0)
    N = 4000
    out = {}
    for law in ("optimal", "uniform"):
        pr = _problem(m=3, n=12, p=2, sampling=law)
        _, M2, _ = oracle.level_stats(pr, lv, 0, 0, N)
        V = M2 / (N - 1)
        want = _closed_form_V0(pr, c, law == "optimal")
        assert abs(V - want) <= 0.15 * want, (law, V, want)
        out[law] = want
    assert out["optimal"] < out["uniform"]


def test_level_differences_are_centred():
    pr = _problem(m=2, n=10, p=2, sampling="optimal")
    lv = oracle.Levels(2, 2, 2)
    N = 3000
    for l in (1, 2):
        mean, M2, _ = oracle.level_stats(pr, lv, l, 0, N)
        se = math.sqrt(M2 / (N - 1) / N / mean.size)   # entrywise standard error (pooled)
        assert np.all(np.abs(mean) <= 5.0 * se * math.sqrt(mean.size)), (l, np.abs(mean).max(), se)
