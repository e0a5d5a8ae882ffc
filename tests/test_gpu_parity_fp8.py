"""Parity of the FP8 E4M3 (block-scaled) level kernel with the FP64 oracle, through the C ABI.

The E4M3 form quantises every generated entry x of A (and sigma b of B) as 2^e q, e the smallest
integer with max|x| <= 448 2^e over the entry's row (column of B) and 32-slot block of the
sample, q = x / 2^e rounded to the E4M3 grid stochastically: up to the upper neighbour when the
entry's 16-bit dither (its own Philox stream) lies below the fractional position, else down, so
the rounding is unbiased.  Bars:
  * against the plain FP64 oracle: |D - D_oracle| <= tau_e4m3(c) * mag with
    tau_e4m3(c) = 2^-2 + 2^-6 + 2^-15 + (c + 8) 2^-23: each operand moves by less than one E4M3
    spacing, 2^-3 relative (u = 2^-3, so 2u + u^2 per product), plus FP32 generation and
    accumulation as in the bfloat16 bound;
  * against the oracle's own E4M3 emulation (ORC_QUANT_E4M3, the same dithers): the same
    rounding except where an FP32 and an FP64 entry fall on different sides of a dither's
    threshold; at least 90 % of the entries are within (c + 8) 2^-23 * mag + 2^-16 * mag and the
    typical error is far below the plain one.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def tau_e4m3(c):
    return 2.0**-2 + 2.0**-6 + 2.0**-15 + (c + 8) * 2.0**-23


def tau_acc(c):
    return (c + 8) * 2.0**-23 + 2.0**-16


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _spec(pp):
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(DEV, torch.float32) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    return binding.ProblemSpec(*ts, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)


def _orc(pp):
    return oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                          problem_id=pp.problem_id)


CASES = [
    (64, 1024, 64, 16, 5, [(0, 0), (1, 3), (3, 9), (5, 61)]),      # precision workload shapes
    (37, 1000, 53, 16, 3, [(0, 1), (2, 8), (3, 2)]),               # ragged
    (200, 3000, 300, 32, 2, [(0, 4), (2, 11)]),                    # 256-row tiles, several column tiles
    (130, 500, 20, 1, 4, [(0, 0), (1, 2), (4, 7)]),                # c0 = 1: blocks shorter than 32 slots
]


@pytest.mark.parametrize("m,n,p,c0,L,picks", CASES)
def test_e4m3_samples_match_oracle(m, n, p, c0, L, picks):
    pp = make_params(m, n, p, seed_A=3, seed_B=4, seed_idx=5, problem_id=1, dtype=np.float32)
    orc = _orc(pp)
    lv = oracle.Levels(c0, 2, L)
    with binding.Plan([_spec(pp)], c0=c0, L=L, ratio=2, precision="fp8") as plan:
        for l, s in picks:
            c = lv.cl(l)
            D = plan.debug_sample(0, l, s).cpu().numpy()
            Dref, _, _, mag = oracle.sample(orc, lv, l, s)
            Demu, _, _, _ = oracle.sample(orc, lv, l, s, quant=oracle.QUANT_E4M3)
            plain = np.abs(D - Dref) / mag
            emu = np.abs(D - Demu) / mag
            assert np.all(plain <= tau_e4m3(c)), (l, s, plain.max(), tau_e4m3(c))
            assert np.mean(emu <= tau_acc(c)) >= 0.9, (l, s, np.mean(emu <= tau_acc(c)))
            assert np.median(emu) < 0.1 * np.median(plain), (np.median(emu), np.median(plain))


def test_e4m3_level_means_against_fp64_oracle_precision_workload():
    """64x1024x64, c_l = 16 * 2^l, N_l = 2000 * 2^-l: error of each level mean vs the FP64 oracle."""
    m, n, p, c0, L = 64, 1024, 64, 16, 5
    Nl = [2000, 1000, 500, 250, 125, 62]
    pp = make_params(m, n, p, seed_A=0, seed_B=1, dtype=np.float32)
    orc = _orc(pp)
    lv = oracle.Levels(c0, 2, L)
    Y = np.zeros((m, p))
    Yref = np.zeros((m, p))
    with binding.Plan([_spec(pp)], c0=c0, L=L, ratio=2, precision="fp8") as plan:
        for l, N in enumerate(Nl):
            plan.level_stats(0, l, 0, N)
        for l, N in enumerate(Nl):
            n_got, mean, M2 = plan.get_level_stats(0, l)
            mref, M2ref, magm = oracle.level_stats(orc, lv, l, 0, N)
            err = np.abs(mean.cpu().numpy() - mref)
            assert n_got == N
            assert np.all(err <= tau_e4m3(lv.cl(l)) * magm), (l, (err / magm).max())
            rel = np.linalg.norm(mean.cpu().numpy() - mref) / np.linalg.norm(mref)
            print(f"e4m3 level {l}: ||mean - mean_fp64||/||mean_fp64|| = {rel:.3e}; "
                  f"V_l rel. diff = {abs(M2 - M2ref) / M2ref:.3e}")
            assert abs(M2 - M2ref) <= 4 * tau_e4m3(lv.cl(l)) * M2ref
            Y += mean.cpu().numpy()
            Yref += mref
    print(f"e4m3 estimate: ||Yhat - Yhat_fp64||/||Yhat_fp64|| = "
          f"{np.linalg.norm(Y - Yref) / np.linalg.norm(Yref):.3e}")


@pytest.mark.parametrize("tile", [1064, 3256])
def test_e4m3_batched_matches_one_by_one(tile):
    shapes = [(37, 1000, 53), (64, 1024, 64), (200, 3000, 300)]
    specs = []
    for q, (m, n, p) in enumerate(shapes):
        pp = make_params(m, n, p, seed_A=2 * q, seed_B=2 * q + 1, seed_idx=2, problem_id=q, dtype=np.float32)
        specs.append(_spec(pp))
    ranges = [(q, l, 0, 50) for q in range(3) for l in range(3)]
    with binding.Plan(specs, c0=16, L=2, precision="fp8", tile_override=tile) as a, \
            binding.Plan(specs, c0=16, L=2, precision="fp8", tile_override=tile) as b:
        a.level_stats_batch(ranges)
        for r in ranges:
            b.level_stats(*r)
        for q in range(3):
            for l in range(3):
                na, sa, qa = a.get_level_state(q, l)
                nb, sb, qb = b.get_level_state(q, l)
                assert na == nb == 50 and torch.equal(sa, sb) and qa == qb


def test_e4m3_rejects_wide_tiles_and_backward():
    pp = make_params(16, 64, 16, dtype=np.float32)
    with pytest.raises(binding.MLMCError) as e:
        binding.Plan([_spec(pp)], c0=4, L=2, precision="fp8", tile_override=2256)
    assert e.value.status == 1
    with binding.Plan([_spec(pp)], c0=4, L=2, precision="fp8") as plan:
        plan.level_stats(0, 0, 0, 8)
        with pytest.raises(binding.MLMCError) as e:
            plan.backward([torch.zeros(16, 16, device=DEV, dtype=torch.float64)])
        assert e.value.status == 6


def test_e4m3_pair_tiles_agree():
    """The two cluster-pair forms (3256: 8 generator warps on 8-slot items; 4256, the E4M3
    default: 16 warps on 4-slot items, the block maximum over 8 lanes) quantise every entry
    alike (same block maxima, same dithers), so their level sums of D agree bit for bit and
    their M2 up to the FP32 grouping of the drains."""
    pp = make_params(200, 3000, 300, seed_A=13, seed_B=14, seed_idx=15, problem_id=0, dtype=np.float32)
    with binding.Plan([_spec(pp)], c0=32, L=2, precision="fp8", tile_override=3256) as a, \
            binding.Plan([_spec(pp)], c0=32, L=2, precision="fp8", tile_override=4256) as b:
        for l in range(3):
            a.level_stats(0, l, 0, 40)
            b.level_stats(0, l, 0, 40)
            na, sa, qa = a.get_level_state(0, l)
            nb, sb, qb = b.get_level_state(0, l)
            assert na == nb == 40 and torch.equal(sa, sb)
            assert abs(qa - qb) <= 2e-5 * qb
