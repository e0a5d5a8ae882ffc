"""Pins of the oracle's reduced-precision emulation and of its reparameterised adjoint.

* bfloat16 and OCP FP8 E4M3 rounding against PyTorch's own conversions (round to nearest
  even) and against the format definitions (every representable value is a fixed point,
  midpoints go to the even neighbour, saturation at 448).
* The power-of-two absmax block scale: the smallest 2^e with absmax / 2^e <= 448.
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


@pytest.mark.parametrize("quant,u", [(oracle.QUANT_BF16, 2.0**-8), (oracle.QUANT_E4M3, 2.0**-4)])
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
