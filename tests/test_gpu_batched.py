"""Batched persistent launch (BF16): parity with one-by-one launches and with the FP64 oracle.

The per-level sums of D are sums over samples of FP32 tensor-memory accumulators folded per
chunk in chunk order.  Tiles of at most 256 accumulator columns per CTA (and the CTA pairs) keep
the chunk's running sum in tensor memory (one MMA chain per element, independent of the tile's
shape and of how items are spread over CTAs), so batched and one-by-one runs with such tiles
agree bit for bit.  The 256 x 256 single-CTA tile adds each scaled sample to the chunk partial in
global memory instead, which rounds differently: against it the sums agree up to FP32 rounding.
The sums of ||D||^2 are grouped by output tile: bit-identical for the same tile, equal up to
rounding otherwise.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
SHAPES = [(37, 1000, 53), (200, 3000, 300), (64, 1024, 64), (130, 700, 20), (300, 2500, 260)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _specs(shapes, seed0=0):
    specs, pps = [], []
    for q, (m, n, p) in enumerate(shapes):
        pp = make_params(m, n, p, seed_A=seed0 + 2 * q, seed_B=seed0 + 2 * q + 1, seed_idx=2, problem_id=q,
                         dtype=np.float32)
        ts = [torch.from_numpy(np.ascontiguousarray(x)).to(DEV) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
        specs.append(binding.ProblemSpec(*ts, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                                         problem_id=q))
        pps.append(pp)
    return specs, pps


def _single_tile(m, p):
    # the single-problem launch's tile for an m x p output: the CTA pair 3256 above 128 x 128,
    # else 128 or 256 rows and 32..256 columns
    if m > 128 and p > 128:
        return 3256
    mh = 1 if m <= 128 else 2
    bn = 32 if p <= 32 else 64 if p <= 64 else 128 if p <= 128 else 256
    return 1000 * mh + bn


def _sum_scheme(tile_id):
    # the pair's CTAs hold 128 x 256 each, like tile 1256
    rows, cols = (1, 256) if tile_id // 1000 >= 3 else (tile_id // 1000, tile_id % 1000)
    return "mma" if rows * cols <= 256 else "global"


def _states(plan, nprob, L):
    return [[plan.get_level_state(q, l) for l in range(L + 1)] for q in range(nprob)]


def _ranges(nprob, L, begin, count):
    return [(q, l, begin, count) for q in range(nprob) for l in range(L + 1)]


@pytest.mark.parametrize("tile", [1064, 2128, 1256, 3256])
def test_batched_matches_one_by_one_same_tile(tile):
    """With the same tile (3256: clusters of two CTAs walking per-cluster item lists) a batched
    call and the same ranges run one by one give the same bits."""
    specs, _ = _specs(SHAPES)
    L = 3
    with binding.Plan(specs, c0=16, L=L, precision="bf16", tile_override=tile) as a, \
            binding.Plan(specs, c0=16, L=L, precision="bf16", tile_override=tile) as b:
        a.level_stats_batch(_ranges(len(SHAPES), L, 0, 100))
        for q, l, s0, cnt in _ranges(len(SHAPES), L, 0, 100):
            b.level_stats(q, l, s0, cnt)
        assert a.batch_tile()[0] == tile
        for ra, rb in zip(_states(a, len(SHAPES), L), _states(b, len(SHAPES), L)):
            for (na, sa, qa), (nb, sb, qb) in zip(ra, rb):
                assert na == nb == 100
                assert torch.equal(sa, sb)
                assert qa == qb


def test_batched_autotuned_matches_one_by_one_sums():
    specs, _ = _specs(SHAPES, seed0=10)
    L = 2
    with binding.Plan(specs, c0=32, L=L, precision="bf16") as a, \
            binding.Plan(specs, c0=32, L=L, precision="bf16") as b:
        a.level_stats_batch(_ranges(len(SHAPES), L, 0, 70))
        for q, l, s0, cnt in _ranges(len(SHAPES), L, 0, 70):
            b.level_stats(q, l, s0, cnt)
        tile, timings = a.batch_tile()
        assert tile in timings and timings[tile] == min(timings.values())
        for (m, _, p), ra, rb in zip(SHAPES, _states(a, len(SHAPES), L), _states(b, len(SHAPES), L)):
            same_scheme = _sum_scheme(tile) == _sum_scheme(_single_tile(m, p)) != "global"
            for l, ((na, sa, qa), (nb, sb, qb)) in enumerate(zip(ra, rb)):
                assert na == nb
                if same_scheme:
                    assert torch.equal(sa, sb)
                else:
                    # FP32 sums of at most 64 samples of c_l products each, kept in two ways (one
                    # MMA chain over all products, or each scaled D added in global memory)
                    c = 32 * 2**l
                    assert float((sa - sb).abs().max()) <= (64 + 2 * c) * 2.0**-23 * float(sb.abs().max()), l
                # M2: FP32 sums of squares per thread (at most 256 columns x 64 samples) grouped by
                # each tile's drain, and Welford (2256) against the raw form (zero-mean levels)
                assert abs(qa - qb) <= 2e-5 * qb


def test_batched_many_waves_and_graph_replay():
    """Repeated (problem, level) ranges force one wave each: 6 waves = two graph launches; a
    second call with the same structure replays the cached graph."""
    specs, _ = _specs(SHAPES[:2], seed0=20)
    with binding.Plan(specs, c0=16, L=2, precision="bf16", tile_override=2128) as a, \
            binding.Plan(specs, c0=16, L=2, precision="bf16", tile_override=2128) as b:
        ranges = [(0, 1, 64 * i, 64) for i in range(6)] + [(1, 2, 0, 40)]
        a.level_stats_batch(ranges)
        starts = [40 + 4 * i * (i + 1) for i in range(5)]   # 40, 48, 64, 88, 120
        a.level_stats_batch([(0, 1, 384, 64)] + [(1, 2, starts[i], 8 * (i + 1)) for i in range(5)] + [(0, 0, 0, 9)])
        for q, l, s0, cnt in ranges:
            b.level_stats(q, l, s0, cnt)
        b.level_stats(0, 1, 384, 64)
        s = 40
        for i in range(5):
            b.level_stats(1, 2, s, 8 * (i + 1))
            s += 8 * (i + 1)
        b.level_stats(0, 0, 0, 9)
        for q, l in [(0, 1), (1, 2), (0, 0)]:
            na, sa, qa = a.get_level_state(q, l)
            nb, sb, qb = b.get_level_state(q, l)
            assert na == nb and torch.equal(sa, sb) and qa == qb


@pytest.mark.parametrize("tile", [0, 3256])
def test_batched_levels_match_fp64_oracle(tile):
    """Level means of batched problems against the FP64 oracle (BF16 bound of the level kernel),
    with the autotuned tile and with the CTA pair (whose second CTA holds no rows when m <= 128)."""
    shapes = [(37, 1000, 53), (64, 1024, 64)] + ([(200, 3000, 300)] if tile else [])
    specs, pps = _specs(shapes, seed0=30)
    L, N = 3, 40
    lv = oracle.Levels(16, 2, L)
    with binding.Plan(specs, c0=16, L=L, precision="bf16", tile_override=tile) as plan:
        plan.level_stats_batch(_ranges(len(shapes), L, 0, N))
        for q, pp in enumerate(pps):
            orc = oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                                 problem_id=q)
            for l in range(L + 1):
                n_got, mean, _ = plan.get_level_stats(q, l)
                mref, _, magm = oracle.level_stats(orc, lv, l, 0, N)
                c = lv.cl(l)
                tau = 2.0**-7 + 2.0**-15 + (c + 8) * 2.0**-23
                assert n_got == N
                assert np.all(np.abs(mean.cpu().numpy() - mref) <= tau * magm)


def test_batched_estimate():
    shapes = [(48, 800, 40), (96, 2000, 72), (33, 4096, 130)]
    specs, pps = _specs(shapes, seed0=40)
    eps = [0.05 * np.linalg.norm(pp.exact_mean()) for pp in pps]
    with binding.Plan(specs, c0=16, L=3, precision="bf16", pilot_n=64) as plan:
        ys, reps = plan.estimate(eps)
        for y, rep, pp, e in zip(ys, reps, pps, eps):
            assert np.linalg.norm(y.cpu().numpy() - pp.exact_mean()) <= 5 * rep["rmse_pred"]
            assert rep["rmse_pred"] <= 1.3 * e / np.sqrt(2)
        assert plan.batch_tile()[0] > 0


def test_batched_rejects_bad_ranges():
    specs, _ = _specs(SHAPES[:1])
    with binding.Plan(specs, c0=16, L=2, precision="bf16") as plan:
        with pytest.raises(binding.MLMCError) as e:
            plan.level_stats_batch([(0, 3, 0, 8)])
        assert e.value.status == 1
        with pytest.raises(binding.MLMCError) as e:
            plan.level_stats_batch([(1, 0, 0, 8)])
        assert e.value.status == 1
        plan.level_stats_batch([])
        plan.level_stats_batch([(0, 0, 0, 0)])
    with binding.Plan(specs, c0=16, L=2, precision="bf16", tile_override=4256) as plan:
        with pytest.raises(binding.MLMCError) as e:   # the 16-warp pair serves single-problem launches
            plan.level_stats_batch([(0, 0, 0, 8)])
        assert e.value.status == 6


def test_batched_fp32_runs_one_by_one():
    specs, _ = _specs(SHAPES[:2])
    with binding.Plan(specs, c0=16, L=2, precision="fp32") as a, binding.Plan(specs, c0=16, L=2, precision="fp32") as b:
        a.level_stats_batch(_ranges(2, 2, 0, 30))
        for q, l, s0, cnt in _ranges(2, 2, 0, 30):
            b.level_stats(q, l, s0, cnt)
        for ra, rb in zip(_states(a, 2, 2), _states(b, 2, 2)):
            for (na, sa, qa), (nb, sb, qb) in zip(ra, rb):
                assert na == nb and torch.equal(sa, sb) and qa == qb


def test_batched_graph_replay_with_new_ranges():
    """Three calls with the same wave structure (the graph is captured once and replayed) agree
    with the one-by-one evaluation of the same sample ranges."""
    specs, _ = _specs(SHAPES[:3], seed0=50)
    L = 2
    with binding.Plan(specs, c0=16, L=L, precision="bf16", tile_override=1128) as a, \
            binding.Plan(specs, c0=16, L=L, precision="bf16", tile_override=1128) as b:
        for step in range(3):
            a.level_stats_batch(_ranges(3, L, 64 * step, 64))
            for q, l, s0, cnt in _ranges(3, L, 64 * step, 64):
                b.level_stats(q, l, s0, cnt)
        for ra, rb in zip(_states(a, 3, L), _states(b, 3, L)):
            for (na, sa, qa), (nb, sb, qb) in zip(ra, rb):
                assert na == nb == 192 and torch.equal(sa, sb) and qa == qb
