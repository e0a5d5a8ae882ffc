"""Parity of the BF16 tensor-core level kernel with the FP64 oracle, through the C ABI.

Bars (derived from the arithmetic):
  * against the plain FP64 oracle: |D - D_oracle| <= tau_bf16(c) * mag with
    tau_bf16(c) = 2^-7 + 2^-15 + (c + 8) 2^-23: both operands rounded to bfloat16 (unit roundoff
    2^-8 each, so 2u + u^2 per product), FP32 generation of the entries (2^-16 each), and FP32
    accumulation of c products in the tensor core;
  * against the oracle's own bf16 operand emulation (ORC_QUANT_BF16): only the accumulation
    differs, except for the rare terms whose FP32 and FP64 values round to different bfloat16
    neighbours; at least 90 % of the entries are within (c + 8) 2^-23 * mag + 2^-16 * mag.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu


def tau_bf16(c):
    return 2.0**-7 + 2.0**-15 + (c + 8) * 2.0**-23


def tau_acc(c):
    return (c + 8) * 2.0**-23 + 2.0**-16


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _plan(pp, c0, L, **kw):
    dev = torch.device("cuda:0")
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev, torch.float32) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    spec = binding.ProblemSpec(*ts, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)
    return binding.Plan([spec], c0=c0, L=L, ratio=2, precision="bf16", **kw)


def _orc(pp):
    return oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                          problem_id=pp.problem_id)


CASES = [
    # m, n, p, c0, L, (level, sample) pairs
    (64, 1024, 64, 16, 5, [(0, 0), (1, 3), (3, 9), (5, 61)]),          # precision workload shapes
    (256, 65536, 256, 64, 8, [(0, 0), (0, 777), (2, 5), (8, 1)]),      # large workload shapes
    (37, 1000, 53, 16, 3, [(0, 1), (2, 8), (3, 2)]),                   # ragged, small tiles
    (200, 3000, 300, 32, 2, [(0, 4), (2, 11)]),                        # two column tiles, M = 256
    (130, 500, 20, 1, 4, [(0, 0), (1, 2), (4, 7)]),                    # c0 = 1, odd slot counts
]


@pytest.mark.parametrize("m,n,p,c0,L,picks", CASES)
def test_bf16_samples_match_oracle(m, n, p, c0, L, picks):
    pp = make_params(m, n, p, seed_A=3, seed_B=4, seed_idx=5, problem_id=1, dtype=np.float32)
    orc = _orc(pp)
    lv = oracle.Levels(c0, 2, L)
    with _plan(pp, c0, L) as plan:
        for l, s in picks:
            c = lv.cl(l)
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, _, _, mag = oracle.sample(orc, lv, l, s)
            Demu, _, _, _ = oracle.sample(orc, lv, l, s, quant=oracle.QUANT_BF16)
            plain = np.abs(D - Dref) / mag
            emu = np.abs(D - Demu) / mag
            assert np.all(plain <= tau_bf16(c)), (l, s, plain.max(), tau_bf16(c))
            assert np.mean(emu <= tau_acc(c)) >= 0.9, (l, s, np.mean(emu <= tau_acc(c)))
            # rounding to bf16 is visible: the device agrees with the emulation far better than
            # with the unrounded FP64 result
            assert np.median(emu) < 0.25 * np.median(plain) + 1e-30, (np.median(emu), np.median(plain))


def test_bf16_level_means_against_fp64_oracle_precision_workload():
    """64x1024x64, c_l = 16 * 2^l, N_l = 2000 * 2^-l: error of each level mean vs the FP64 oracle."""
    m, n, p, c0, L = 64, 1024, 64, 16, 5
    Nl = [2000, 1000, 500, 250, 125, 62]
    pp = make_params(m, n, p, seed_A=0, seed_B=1, dtype=np.float32)
    orc = _orc(pp)
    lv = oracle.Levels(c0, 2, L)
    Y = np.zeros((m, p))
    Yref = np.zeros((m, p))
    with _plan(pp, c0, L) as plan:
        for l, N in enumerate(Nl):
            plan.level_stats(0, l, 0, N)
        for l, N in enumerate(Nl):
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 0, N)
            err = np.abs(mean.cpu().numpy() - mref)
            assert n_got == N
            assert np.all(err <= tau_bf16(lv.cl(l)) * magm), (l, (err / magm).max())
            rel = np.linalg.norm(mean.cpu().numpy() - mref) / np.linalg.norm(mref)
            print(f"bf16 level {l}: ||mean - mean_fp64||/||mean_fp64|| = {rel:.3e}; "
                  f"V_l rel. diff = {abs(M2 - M2ref) / M2ref:.3e}")
            assert abs(M2 - M2ref) <= 4 * tau_bf16(lv.cl(l)) * M2ref
            Y += mean.cpu().numpy()
            Yref += mref
    print(f"bf16 estimate: ||Yhat - Yhat_fp64||/||Yhat_fp64|| = "
          f"{np.linalg.norm(Y - Yref) / np.linalg.norm(Yref):.3e}")


def test_bf16_split_calls_are_bit_identical():
    pp = make_params(96, 2048, 80, seed_A=8, seed_B=9, dtype=np.float32)
    with _plan(pp, 32, 3) as one, _plan(pp, 32, 3) as two:
        one.level_stats(0, 2, 0, 192)
        two.level_stats(0, 2, 0, 64)
        two.level_stats(0, 2, 64, 128)
        N1, s1, q1 = one.get_level_state(0, 2)
        N2, s2, q2 = two.get_level_state(0, 2)
        assert N1 == N2 == 192 and q1 == q2 and torch.equal(s1, s2)


def test_bf16_estimate_runs_algorithm_2():
    pp = make_params(64, 1024, 64, seed_A=0, seed_B=1, dtype=np.float32)
    eps = 0.05 * np.linalg.norm(pp.exact_mean())
    with _plan(pp, 16, 4, pilot_n=64) as plan:
        (Y,), (rep,) = plan.estimate([eps])
        err = np.linalg.norm(Y.cpu().numpy() - pp.exact_mean())
        assert err <= 5 * rep["rmse_pred"]
        assert rep["rmse_pred"] <= 1.3 * eps / np.sqrt(2)


def test_bf16_rejects_other_ratios():
    pp = make_params(16, 64, 16, dtype=np.float32)
    with pytest.raises(binding.MLMCError) as e:
        dev = torch.device("cuda:0")
        ts = [torch.from_numpy(x).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
        binding.Plan([binding.ProblemSpec(*ts)], c0=4, L=2, ratio=3, precision="bf16")
    assert e.value.status == 6


PAIR_CASES = [
    (256, 65536, 256, 64, 8, [(0, 0), (0, 777), (2, 5), (8, 1)]),     # the large workload's shape
    (200, 3000, 300, 32, 2, [(0, 4), (2, 11)]),                       # ragged rows, two column tiles
    (300, 2000, 260, 16, 3, [(0, 0), (3, 5)]),                        # three row tiles: one pair half empty
]


@pytest.mark.parametrize("pair_tile", [3256, 4256])
@pytest.mark.parametrize("m,n,p,c0,L,picks", PAIR_CASES)
def test_bf16_cta_pair_tile_matches_oracle_and_single_cta_tile(m, n, p, c0, L, picks, pair_tile):
    """Tiles 3256 and 4256 (two CTAs of a cluster share a 256 x 256 tile, each generating half of B
    for both; 4256 with 16 generator warps on 4-slot items) against the FP64 oracle, and their
    level sums against the 128 x 256 single-CTA tile (the same MMA chain per element, so the sums
    of D agree bit for bit; the M2 are grouped by the drain's column split, so they agree up to
    FP32 rounding)."""
    pp = make_params(m, n, p, seed_A=3, seed_B=4, seed_idx=5, problem_id=1, dtype=np.float32)
    orc = _orc(pp)
    lv = oracle.Levels(c0, 2, L)
    with _plan(pp, c0, L, tile_override=pair_tile) as plan:
        for l, s in picks:
            c = lv.cl(l)
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, _, _, mag = oracle.sample(orc, lv, l, s)
            assert np.all(np.abs(D - Dref) / mag <= tau_bf16(c)), (l, s)
    with _plan(pp, c0, L, tile_override=pair_tile) as a, _plan(pp, c0, L, tile_override=1256) as b:
        for l in range(min(L, 3) + 1):
            a.level_stats(0, l, 0, 96)
            b.level_stats(0, l, 0, 96)
            na, sa, qa = a.get_level_state(0, l)
            nb, sb, qb = b.get_level_state(0, l)
            assert na == nb == 96
            assert torch.equal(sa, sb)
            # M2 is accumulated per thread in FP32 (at most 128 columns x 64 samples of squares, a
            # relative rounding of at most 192 * 2^-24 each) and grouped by the drain's column split
            assert abs(qa - qb) <= 2e-5 * qb


def test_generation_rate_is_measured():
    """mlmc_measure_generation_rate: entries per second of generation alone.  152 SMs at about
    2 GHz issue at most ~1.2e12 warp instructions per second and an entry costs tens of thread
    instructions, so any sane measurement lies between 1e11 and 1e14 entries/s; two calls agree
    to a few per cent (best of three launches each)."""
    r1 = binding.generation_rate()
    r2 = binding.generation_rate()
    print(f"generation rate: {r1:.3e} / {r2:.3e} entries/s")
    assert 1e11 < r1 < 1e14 and 1e11 < r2 < 1e14
    assert abs(r1 - r2) <= 0.1 * max(r1, r2)
