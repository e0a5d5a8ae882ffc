"""Sample-parallel Alg. 2 over two gloo ranks on CPU (the oracle stands in for the GPU plan).

Checks: the shards partition every round's sample ids into chunk-aligned contiguous pieces;
both ranks obtain the same N_l and the same estimate; the N_l equal those of one process
running the same rounds; the estimate equals the one-process estimate up to the order of the
FP64 additions; the union of the ranks' evaluated ids is exactly 0 .. N_l - 1 of every level.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1904_00429_gb300 import distributed
from paper_1904_00429_gb300.inputs import make_params

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("begin,count,world", [(0, 256, 2), (256, 1000, 2), (64, 5, 2), (0, 0, 3),
                                               (128, 777, 4), (7, 130, 2)])
def test_shards_partition_the_range(begin, count, world):
    pieces = [distributed.shard(begin, count, r, world) for r in range(world)]
    ids = []
    for b, c in pieces:
        assert c >= 0
        ids.extend(range(b, b + c))
    assert ids == list(range(begin, begin + count))
    for b, c in pieces[1:]:
        if c > 0 and b != begin:
            assert b % distributed.ALIGN == 0


def _problems():
    return [make_params(6, 40, 5, seed_A=3, seed_B=4, seed_idx=5, problem_id=0),
            make_params(4, 25, 7, seed_A=6, seed_B=7, seed_idx=8, problem_id=1)]


EPS_REL = 0.15


def _eps(pps):
    return [EPS_REL * float(np.linalg.norm(pp.exact_mean())) for pp in pps]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, HERE)
    from fake_plan import FakePlan
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pps = _problems()
    plan = FakePlan(pps, c0=2, L=2, pilot_n=8)
    ys, Nl = distributed.estimate(plan, _eps(pps))
    torch.save({"y": [y.clone() for y in ys], "Nl": Nl, "evaluated": plan.evaluated},
               os.path.join(out_dir, f"rank{rank}.pt"))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_estimate_matches_one_process(tmp_path):
    sys.path.insert(0, HERE)
    from fake_plan import FakePlan
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [torch.load(tmp_path / f"rank{r}.pt") for r in range(world)]
    # one process, same rounds
    pps = _problems()
    ref = FakePlan(pps, c0=2, L=2, pilot_n=8)
    ref.level_stats_batch([(q, l, 0, 8) for q in range(2) for l in range(3)])
    Nl_ref = ref.allocate(_eps(pps))
    ref.level_stats_batch([(q, l, 8, Nl_ref[q][l] - 8) for q in range(2) for l in range(3) if Nl_ref[q][l] > 8])
    y_ref = ref.telescoping_sum()
    assert res[0]["Nl"] == res[1]["Nl"] == Nl_ref
    assert max(Nl_ref[0]) > 8 and max(Nl_ref[1]) > 8      # the allocation asked for a top-up
    for q in range(2):
        assert torch.equal(res[0]["y"][q], res[1]["y"][q])
        assert torch.allclose(res[0]["y"][q], y_ref[q], rtol=1e-12, atol=1e-12 * float(y_ref[q].abs().max()))
        for l in range(3):
            ids = sorted(res[0]["evaluated"][(q, l)] + res[1]["evaluated"][(q, l)])
            assert ids == list(range(Nl_ref[q][l]))
            # both ranks carried about half of the top-up
            share = len(res[1]["evaluated"][(q, l)]) / Nl_ref[q][l]
            assert 0.4 < share < 0.6, share


def _bias_params():
    # m = p = 2, n = 16, entries of AB spread around the jump of f(x) = |x| H(2 - x)
    from paper_1904_00429_gb300.inputs import ProblemParams
    rng = np.random.default_rng(9)
    M = rng.uniform(0.2, 0.6, (2, 16))
    S = np.full((2, 16), 0.3)
    Mp = rng.uniform(0.05, 0.35, (16, 2))
    Sp = np.full((16, 2), 0.1)
    return ProblemParams(M, S, Mp, Sp, 21, 22, 23, 0, {"law": "custom"})


ADAPT_EPS = 0.08


def _adaptive_worker(rank, world, port, out_dir):
    sys.path.insert(0, HERE)
    from fake_plan import FakePlan
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = FakePlan([_bias_params()], c0=1, L=10, pilot_n=32, fkind=oracle.F_ABS_STEP)
    ys, Nl = distributed.estimate(plan, [ADAPT_EPS], adaptive=True)
    torch.save({"y": [y.clone() for y in ys], "Nl": Nl, "evaluated": plan.evaluated},
               os.path.join(out_dir, f"rank{rank}.pt"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_adaptive_L_matches_the_oracle(tmp_path):
    """Alg. 2 with the adaptive L (E[f(AB)], f(x) = |x| H(2 - x)) sharded over two gloo ranks:
    the same finest level and N_l as the oracle's single-process Alg. 2, the same estimate up to
    the order of the FP64 additions, and every sample id evaluated exactly once."""
    world = 2
    mp.start_processes(_adaptive_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [torch.load(tmp_path / f"rank{r}.pt") for r in range(world)]
    pp = _bias_params()
    orc = oracle.Problem(*pp.f64(), seed_A=21, seed_B=22, seed_idx=23, problem_id=0)
    Yref, Lref, Nref, _, _ = oracle.estimate_f(orc, oracle.Levels(1, 2, 10), ADAPT_EPS, fkind=oracle.F_ABS_STEP,
                                               adaptive=True, pilot=32)
    assert Lref >= 3
    assert res[0]["Nl"] == res[1]["Nl"] == [list(Nref)]
    assert torch.equal(res[0]["y"][0], res[1]["y"][0])
    np.testing.assert_allclose(res[0]["y"][0].numpy(), Yref, rtol=1e-11, atol=1e-13)
    for l in range(Lref + 1):
        ids = sorted(res[0]["evaluated"][(0, l)] + res[1]["evaluated"][(0, l)])
        assert ids == list(range(int(Nref[l])))


def _second_bias_params():
    from paper_1904_00429_gb300.inputs import ProblemParams
    rng = np.random.default_rng(11)
    M = rng.uniform(0.1, 0.5, (3, 12))
    S = np.full((3, 12), 0.25)
    Mp = rng.uniform(0.1, 0.4, (12, 2))
    Sp = np.full((12, 2), 0.15)
    return ProblemParams(M, S, Mp, Sp, 31, 32, 33, 1, {"law": "custom"})


def _multi_worker(rank, world, port, out_dir):
    sys.path.insert(0, HERE)
    from fake_plan import FakePlan
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = FakePlan([_bias_params(), _second_bias_params()], c0=1, L=10, pilot_n=32, fkind=oracle.F_ABS_STEP)
    ys, Nl = distributed.estimate(plan, [ADAPT_EPS, 0.1], adaptive=True)
    torch.save({"y": [y.clone() for y in ys], "Nl": Nl}, os.path.join(out_dir, f"rank{rank}.pt"))
    dist.barrier()
    dist.destroy_process_group()


def test_adaptive_L_is_decided_per_problem(tmp_path):
    """Two problems in one plan, one rank: each stops at its own finest level, with the N_l and
    estimate of its own single-problem Alg. 2 (rounds interleave, decisions do not)."""
    mp.start_processes(_multi_worker, args=(1, _free_port(), str(tmp_path)), nprocs=1, join=True,
                       start_method="spawn")
    res = torch.load(tmp_path / "rank0.pt")
    Ls = []
    for q, (pp, eps) in enumerate([(_bias_params(), ADAPT_EPS), (_second_bias_params(), 0.1)]):
        orc = oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                             problem_id=pp.problem_id)
        Yref, Lref, Nref, _, _ = oracle.estimate_f(orc, oracle.Levels(1, 2, 10), eps, fkind=oracle.F_ABS_STEP,
                                                   adaptive=True, pilot=32)
        assert res["Nl"][q] == list(Nref)
        np.testing.assert_allclose(res["y"][q].numpy(), Yref, rtol=1e-11, atol=1e-13)
        Ls.append(Lref)
    assert Ls[0] != Ls[1], Ls   # the case exercises problems that stop at different levels
