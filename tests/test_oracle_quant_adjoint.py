"""Pins of the oracle's reduced-precision emulation and of its reparameterised adjoint.

* bfloat16 and OCP FP8 E4M3 rounding against PyTorch's own conversions (round to nearest
  even) and against the format definitions (every representable value is a fixed point,
  midpoints go to the even neighbour, saturation at 448).
* The power-of-two absmax block scale: the smallest 2^e with absmax / 2^e <= 448.
* Stochastic E4M3 rounding: the result is always one of the two grid neighbours, grid values are
  fixed points, the sign is kept, and over all 2^16 dithers the mean is the input within 2^-17
  of the spacing (unbiased rounding, checked by enumeration); round to nearest even on the same
  grid, averaged over a Gaussian input, shrinks it by about 10^-3 of its mean (the reason the
  FP8 form rounds stochastically), while the stochastic rounding's mean stays exact.
* The dither stream: each 16-bit dither is the stated half of the stated word of one
  Philox4x32-10 block, and the dithers of one block are those of 4 rows x 2 slots.
* A quantised sample stays within the operand-rounding bound of the exact one.
* The adjoint of the loss ||Yhat - T||_F^2 against central finite differences with common
  random numbers.  Yhat is affine in each single parameter (every sampled product has one
  factor from A and one from B, and A = M + S o Z is affine in M and in S), so the loss is
  quadratic in it and the central difference is exact up to rounding.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300.inputs import make_params, make_target


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.normal(size=4000) * 10.0 ** rng.integers(-30, 30, size=4000),
        rng.uniform(-1, 1, size=1000) * 1e-39,           # binary32 subnormals
        np.float32(1.0) + np.arange(1, 200) * 2.0**-8,   # exact midpoints and neighbours
    ]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_bf16(float(v)) for v in x])
    np.testing.assert_array_equal(got, ref)


def test_e4m3_rounding_matches_torch_and_format():
    rng = np.random.default_rng(1)
    x = np.concatenate([
        rng.uniform(-463.9, 463.9, size=3000),
        rng.normal(size=3000) * 2.0 ** rng.integers(-12, 6, size=3000),
    ]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([oracle.round_e4m3(float(v)) for v in x])
    np.testing.assert_array_equal(got, ref)
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    finite = np.unique(codes[np.isfinite(codes)])
    assert finite.max() == 448.0 and len(finite) == 253
    for v in finite:
        assert oracle.round_e4m3(float(v)) == v
    # midpoints between neighbours round to the one with an even last fraction bit
    pos = finite[finite >= 0]
    for a, b in zip(pos[:-1], pos[1:]):
        mid = oracle.round_e4m3((a + b) / 2)
        even = a if (np.where(codes == a)[0][0] & 1) == 0 else b
        assert mid == even
    assert oracle.round_e4m3(1e6) == 448.0 and oracle.round_e4m3(-500.0) == -448.0


def test_e4m3_block_scale_is_smallest_power_of_two():
    for absmax in [1e-30, 0.003, 1.0, 447.0, 448.0, 448.0001, 896.0, 900.0, 3.7e5]:
        s = oracle.e4m3_block_scale(absmax)
        e = np.log2(s)
        assert e == np.round(e)
        assert absmax / s <= 448.0
        assert absmax / (s / 2) > 448.0
    assert oracle.e4m3_block_scale(0.0) == 1.0


def _e4m3_grid():
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    return np.unique(codes[np.isfinite(codes) & (codes >= 0)])


def test_e4m3_stochastic_rounding_is_unbiased_by_enumeration():
    grid = _e4m3_grid()
    rng = np.random.default_rng(5)
    ys = np.concatenate([rng.uniform(0, 448, size=40), rng.uniform(0, 2.0**-6, size=10),
                         2.0 ** rng.uniform(-9, 8, size=40), grid[1:-1:17] + 1e-9, [447.99, 255.9, 2.0**-9 * 0.3]])
    d = np.arange(65536, dtype=np.uint32)
    for y in ys:
        k = np.searchsorted(grid, y, side="right") - 1
        lo, hi = grid[k], grid[min(k + 1, len(grid) - 1)]
        outs = np.array([oracle.round_e4m3_sr(float(y), int(v)) for v in d[::1 if y < 1e-3 else 257]])
        assert set(np.unique(outs)) <= {lo, hi}, (y, np.unique(outs), lo, hi)
        if y >= 1e-3:
            continue
        # the full enumeration for a few inputs: mean over all dithers = y within 2^-17 h
        assert abs(outs.mean() - y) <= 2.0**-17 * (hi - lo) + 1e-300
    for y in [0.3, 1.7, 37.0 + 1.0 / 3.0, 300.0, 447.0]:
        outs = np.array([oracle.round_e4m3_sr(y, int(v)) for v in d])
        k = np.searchsorted(grid, y, side="right") - 1
        h = grid[k + 1] - grid[k]
        assert abs(outs.mean() - y) <= 2.0**-17 * h, (y, outs.mean() - y)
        neg = np.array([oracle.round_e4m3_sr(-y, int(v)) for v in d[:4096]])
        np.testing.assert_array_equal(neg, -outs[:4096])
    for v in grid:
        for dd in (0, 1, 32767, 65535):
            assert oracle.round_e4m3_sr(float(v), dd) == v
    assert oracle.round_e4m3_sr(0.0, 123) == 0.0


def test_nearest_even_on_the_e4m3_grid_shrinks_a_gaussian_stochastic_rounding_does_not():
    """E[RNE(Y)] for Y ~ N(mu, sigma^2) by quadrature: the grid spacing grows with |y|, so the
    rounding intervals of a smooth density are lopsided at every power of two and the mean moves
    towards zero by about 10^-3 of mu (3 fraction bits); E[SR(Y)] = E[Y] to the quadrature's
    accuracy, because the stochastic rounding is unbiased for every y."""
    mu, sigma = 200.0, 60.0
    y = np.linspace(mu - 8 * sigma, mu + 8 * sigma, 200001)
    w = np.exp(-0.5 * ((y - mu) / sigma) ** 2)
    w /= w.sum()
    y = np.clip(y, 0.0, 448.0)
    w_mean = float((w * y).sum())
    rne = np.array([oracle.round_e4m3(float(v)) for v in y])
    bias_rne = float((w * rne).sum()) - w_mean
    grid = _e4m3_grid()
    k = np.searchsorted(grid, y, side="right") - 1
    lo, hi = grid[k], grid[np.minimum(k + 1, len(grid) - 1)]
    f = np.where(hi > lo, (y - lo) / np.where(hi > lo, hi - lo, 1.0), 0.0)
    sr_mean = float((w * (lo + f * (hi - lo))).sum())   # E over the dither of SR(y), exact
    print(f"E[RNE(Y)] - E[Y] = {bias_rne:.4e} ({bias_rne / w_mean:.2e} relative); "
          f"E[SR(Y)] - E[Y] = {sr_mean - w_mean:.2e}")
    assert bias_rne / w_mean < -3e-4
    assert abs(sr_mean - w_mean) <= 1e-9 * w_mean


def test_e4m3_dither_is_its_philox_word_half():
    for seed, pid, l, s, row, t in [(4, 1, 0, 0, 0, 0), (4, 1, 3, 12345, 7, 9), (9, 2, 8, (1 << 40) + 5, 130, 511)]:
        ctr = np.array([row >> 2, 0x80000000 | (t >> 1), s & 0xFFFFFFFF, ((s >> 32) << 8) | l], dtype=np.uint32)
        w = oracle.philox4x32(ctr, np.array([seed, pid], dtype=np.uint32))
        word = int(w[row & 3])
        want = (word >> 16) if (t & 1) else (word & 0xFFFF)
        assert oracle.e4m3_dither(seed, pid, l, s, row, t) == want


@pytest.mark.parametrize("quant,u", [(oracle.QUANT_BF16, 2.0**-8), (oracle.QUANT_E4M3, 2.0**-3),
                                     (oracle.QUANT_E4M3_RNE, 2.0**-4)])
def test_quantised_sample_within_operand_rounding_bound(quant, u):
    pp = make_params(8, 40, 6, seed_A=2, seed_B=3)
    pr = oracle.Problem(*pp.f64())
    lv = oracle.Levels(16, 2, 2)
    for l in range(3):
        for s in range(3):
            D, _, _, mag = oracle.sample(pr, lv, l, s)
            Dq, _, _, magq = oracle.sample(pr, lv, l, s, quant=quant)
            bound = (2 * u + u * u) * mag + 1e-12 * mag
            assert np.all(np.abs(Dq - D) <= bound)
            assert np.any(Dq != D)


def _loss(pr, lv, Nl, T):
    Y = np.zeros((pr.m, pr.p))
    for l in range(lv.L + 1):
        mean, _, _ = oracle.level_stats(pr, lv, l, 0, int(Nl[l]))
        Y += mean
    return float(((Y - T) ** 2).sum()), Y


def test_adjoint_matches_central_differences_with_common_random_numbers():
    m, n, p = 32, 512, 32
    pp = make_params(m, n, p, seed_A=0, seed_B=1)
    M, S, Mp, Sp = [x.copy() for x in pp.f64()]
    T = make_target(m, p)
    lv = oracle.Levels(16, 2, 3)
    Nl = np.array([64, 64, 64, 64])
    pr = oracle.Problem(M, S, Mp, Sp)
    L0, Y = _loss(pr, lv, Nl, T)
    G = 2.0 * (Y - T)
    dM, dS, dMp, dSp = oracle.adjoint(pr, lv, Nl, G)
    h = 1e-3
    rng = np.random.default_rng(5)
    # entries that were sampled (nonzero gradient) and one that probably was not
    mats = {"M": (M, dM), "S": (S, dS), "Mp": (Mp, dMp), "Sp": (Sp, dSp)}
    for name, (X, dX) in mats.items():
        nz = np.argwhere(dX != 0)
        picks = [tuple(nz[i]) for i in rng.choice(len(nz), size=2, replace=False)]
        picks.append(tuple(np.unravel_index(np.argmin(np.abs(dX)), dX.shape)))
        for ij in picks:
            old = X[ij]
            X[ij] = old + h
            Lp, _ = _loss(oracle.Problem(M, S, Mp, Sp), lv, Nl, T)
            X[ij] = old - h
            Lm, _ = _loss(oracle.Problem(M, S, Mp, Sp), lv, Nl, T)
            X[ij] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - dX[ij]) <= 1e-7 * (abs(dX[ij]) + 1e-3 * np.abs(dX).max()), (name, ij, fd, dX[ij])
