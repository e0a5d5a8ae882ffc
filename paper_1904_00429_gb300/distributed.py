"""Sample-parallel Alg. 2 over several processes (one GPU each).

Samples of a level are independent and every draw is a pure function of (seed, problem, level,
sample, entry), so the sample ids of each round (the pilot, then the top-up of the allocation)
are split into contiguous, chunk-aligned shards, one per rank.  Each rank folds its shard into
an empty copy of the level statistics; the per-level states (N, sum of D, M2) of all ranks are
gathered with one all-gather per round, and every rank folds them, in rank order, into the
statistics merged so far with the library's Chan update (mlmc_merge_level_state).  Every rank
thus holds the same statistics, computes the same variances, allocation N_l (Remark 3.6,
mlmc_allocate / mlmc_allocate_levels), stopping decisions (Remark 3.5, mlmc_bias_test) and
estimate Yhat (Eq. hatY); they equal the single-process ones up to the order of the FP64
operations.  No arithmetic of the method runs in this module: it moves states between
processes and calls the library.

The driver works on any object with the plan methods used below (``binding.Plan`` on a GPU);
``torch.distributed`` provides the exchange (NCCL between GPUs, gloo on CPUs).
"""
from __future__ import annotations

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
    """The merged (N, sum, M2) of every (problem, level), kept beside the plan."""

    def __init__(self, plan):
        self.state = {}
        for q, l in _levels(plan):
            N, s, M2 = plan.get_level_state(q, l)
            self.state[(q, l)] = [N, s.clone(), M2]


def _gather_round(plan, merged: _Merged, group, device) -> None:
    """All-gather every rank's round state and fold the states, in rank order, into the merged
    statistics of the earlier rounds (on every rank, with the same calls)."""
    keys = sorted(merged.state)
    parts = []
    for q, l in keys:
        N, s, M2 = plan.get_level_state(q, l)
        parts.append(torch.tensor([float(N), M2], dtype=torch.float64, device=device))
        parts.append(s.reshape(-1).to(device=device, dtype=torch.float64))
    flat = torch.cat(parts)
    gathered = [torch.empty_like(flat) for _ in range(dist.get_world_size(group))]
    dist.all_gather(gathered, flat, group=group)
    off = 0
    for q, l in keys:
        entry = merged.state[(q, l)]
        n_el = entry[1].numel()
        plan.set_level_state(q, l, entry[0], entry[1], entry[2])
        for g in gathered:
            N, M2 = int(round(float(g[off]))), float(g[off + 1])
            plan.merge_level_state(q, l, N, g[off + 2:off + 2 + n_el].reshape(entry[1].shape), M2)
        off += 2 + n_el
        N, s, M2 = plan.get_level_state(q, l)
        merged.state[(q, l)] = [N, s.clone(), M2]


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
    _gather_round(plan, merged, group, device)


def _estimate_adaptive(plan, eps_abs, group, device):
    """Alg. 2 choosing L per problem: rounds on levels 0..L_q for L_q = 0, 1, ... (pilot on the new
    level, allocation over levels 0..L_q from the merged sums, top-ups), stopping after the first
    round with L_q >= 2 whose finest mean satisfies ||Y_L||_F < (sqrt(R) + 1) eps / sqrt(2)
    (Remark 3.5), or at the plan's L for the problem.  The allocation and the stopping test are
    the library's (mlmc_allocate_levels, mlmc_bias_test) on the merged statistics, so every rank
    takes the same decisions."""
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
                Nl = plan.allocate_levels(q, Lc[q], eps_abs[q])
                for l in range(Lc[q] + 1):
                    have = merged.state[(q, l)][0]
                    if Nl[l] > have:
                        ranges.append((q, l, have, Nl[l] - have))
        _run_round(plan, ranges, merged, group, device)
        more = False
        for q in range(nprob):
            if not running[q]:
                continue
            if Lc[q] >= 2 and plan.bias_test(q, Lc[q], eps_abs[q])[0]:
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
