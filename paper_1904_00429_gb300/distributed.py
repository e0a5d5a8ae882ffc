"""Sample-parallel Alg. 2 over several processes (one GPU each).

Samples of a level are independent and every draw is a pure function of (seed, problem, level,
sample, entry), so the sample ids of each round (the pilot, then the top-up of the allocation)
are split into contiguous, chunk-aligned shards, one per rank.  Each rank folds its shard into
an empty copy of the level statistics, the per-level raw sums (N, sum of D, sum of ||D||_F^2)
are added over the ranks with one all-reduce per round, and the merged statistics replace every
rank's own, so every rank computes the same variances and the same allocation N_l (Remark 3.6)
and the same estimate Yhat (Eq. hatY).  The merged sums equal the single-process ones up to the
order of the FP64 additions.

The driver works on any object with the plan methods used below (``binding.Plan`` on a GPU);
``torch.distributed`` provides the reduction (NCCL between GPUs, gloo on CPUs).
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import torch
import torch.distributed as dist

# Shards start on multiples of this many sample ids, so that every shard is made of whole
# chunks of the level kernels (whose chunk lengths divide 64).
ALIGN = 64


def shard(begin: int, count: int, rank: int, world: int, align: int = ALIGN) -> Tuple[int, int]:
    """Rank ``rank``'s part (begin, count) of the sample ids [begin, begin + count): contiguous
    pieces in rank order whose inner boundaries are multiples of ``align``."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    end = begin + count
    cuts = [begin]
    for r in range(1, world):
        c = begin + (count * r) // world
        c = min(end, max(cuts[-1], -(-c // align) * align))
        cuts.append(c)
    cuts.append(end)
    return cuts[rank], cuts[rank + 1] - cuts[rank]


def _levels(plan) -> List[Tuple[int, int]]:
    return [(q, l) for q in range(len(plan.problems)) for l in range(plan.levels[q] + 1)]


class _Merged:
    """The merged (N, sum, sumsq) of every (problem, level), kept beside the plan."""

    def __init__(self, plan):
        self.state = {}
        for q, l in _levels(plan):
            N, s, sq = plan.get_level_state(q, l)
            self.state[(q, l)] = [N, s.clone(), sq]


def _allreduce_round(plan, merged: _Merged, group, device) -> None:
    keys = sorted(merged.state)
    parts = []
    for q, l in keys:
        N, s, sq = plan.get_level_state(q, l)
        parts.append(torch.tensor([float(N), sq], dtype=torch.float64, device=device))
        parts.append(s.reshape(-1).to(device=device, dtype=torch.float64))
    flat = torch.cat(parts)
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for q, l in keys:
        N, sq = int(round(float(flat[off]))), float(flat[off + 1])
        off += 2
        entry = merged.state[(q, l)]
        n_el = entry[1].numel()
        s = flat[off:off + n_el].reshape(entry[1].shape).to(entry[1].device)
        off += n_el
        entry[0] += N
        entry[1] = entry[1] + s
        entry[2] += sq
        plan.set_level_state(q, l, entry[0], entry[1], entry[2])


def _run_round(plan, ranges: Sequence[Tuple[int, int, int, int]], merged: _Merged, group, device) -> None:
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    for q, l in _levels(plan):
        plan.reset(q, l)
    mine = []
    for q, l, b, c in ranges:
        sb, sc = shard(b, c, rank, world)
        if sc > 0:
            mine.append((q, l, sb, sc))
    if mine:
        plan.level_stats_batch(mine)
    _allreduce_round(plan, merged, group, device)


def _allocate(plan, merged: _Merged, q: int, L: int, eps: float) -> List[int]:
    """N_l of levels 0..L (Remark 3.6 with C_0 = c_0, C_l = c_l + c_{l-1}) from the merged sums."""
    c = [plan.c0 * plan.ratio ** l for l in range(L + 1)]
    V, C = [], []
    for l in range(L + 1):
        N, s, sq = merged.state[(q, l)]
        M2 = sq - float((s * s).sum()) / N
        V.append(max(0.0, M2 / (N - 1)))
        C.append(float(c[0] if l == 0 else c[l] + c[l - 1]))
    root = sum(math.sqrt(v * cc) for v, cc in zip(V, C))
    return [max(plan.pilot_n, int(math.ceil(plan.nl_scale * 2.0 / eps**2 * math.sqrt(v / cc) * root)))
            for v, cc in zip(V, C)]


def _mean_norm(merged: _Merged, q: int, l: int) -> float:
    N, s, _ = merged.state[(q, l)]
    return float(torch.linalg.norm(s.double())) / N if N > 0 else 0.0


def _estimate_adaptive(plan, eps_abs, group, device):
    """Alg. 2 choosing L per problem: rounds on levels 0..L_q for L_q = 0, 1, ... (pilot on the new
    level, allocation over levels 0..L_q from the merged sums, top-ups), stopping after the first
    round with L_q >= 2 whose finest mean satisfies ||Y_L||_F < (sqrt(R) + 1) eps / sqrt(2)
    (Remark 3.5), or at the plan's L for the problem.  The decisions use merged statistics, so
    every rank takes the same ones."""
    merged = _Merged(plan)
    nprob = len(plan.problems)
    Lc = [0] * nprob
    running = [True] * nprob
    pilot = plan.pilot_n
    while True:
        ranges = []
        for q in range(nprob):
            if running[q]:
                for l in range(Lc[q] + 1):
                    have = merged.state[(q, l)][0]
                    if have < pilot:
                        ranges.append((q, l, have, pilot - have))
        _run_round(plan, ranges, merged, group, device)
        ranges = []
        for q in range(nprob):
            if running[q]:
                Nl = _allocate(plan, merged, q, Lc[q], eps_abs[q])
                for l in range(Lc[q] + 1):
                    have = merged.state[(q, l)][0]
                    if Nl[l] > have:
                        ranges.append((q, l, have, Nl[l] - have))
        _run_round(plan, ranges, merged, group, device)
        more = False
        for q in range(nprob):
            if not running[q]:
                continue
            bound = (math.sqrt(plan.ratio) + 1.0) * eps_abs[q] / math.sqrt(2.0)
            if Lc[q] >= 2 and _mean_norm(merged, q, Lc[q]) < bound:
                running[q] = False
            elif Lc[q] == plan.levels[q]:
                running[q] = False
            else:
                Lc[q] += 1
                more = True
        if not more:
            break
    return plan.telescoping_sum(), [[merged.state[(q, l)][0] for l in range(Lc[q] + 1)] for q in range(nprob)]


def estimate(plan, eps_abs: Sequence[float], group=None, device: Optional[torch.device] = None,
             adaptive: bool = False):
    """Alg. 2 with its samples sharded over the ranks of ``group``: the finest level fixed at the
    plan's L, or (``adaptive``) chosen by Alg. 2's while loop (Remark 3.5).

    Returns (list of m x p FP64 estimates, list of per-problem N_l, one entry per level used).
    Every rank returns the same values.  ``device`` is where the reduction buffer lives (the
    plan's device for NCCL, CPU for gloo)."""
    if device is None:
        device = torch.device("cpu") if dist.get_backend(group) == "gloo" else plan.device
    if adaptive:
        return _estimate_adaptive(plan, eps_abs, group, device)
    merged = _Merged(plan)
    pilot = plan.pilot_n
    ranges = []
    for q, l in _levels(plan):
        have = merged.state[(q, l)][0]
        if have < pilot:
            ranges.append((q, l, have, pilot - have))
    _run_round(plan, ranges, merged, group, device)
    Nl = plan.allocate(eps_abs)
    ranges = []
    for q, l in _levels(plan):
        have = merged.state[(q, l)][0]
        if Nl[q][l] > have:
            ranges.append((q, l, have, Nl[q][l] - have))
    _run_round(plan, ranges, merged, group, device)
    return plan.telescoping_sum(), [[merged.state[(q, l)][0] for l in range(plan.levels[q] + 1)]
                                    for q in range(len(plan.problems))]
