"""Failure detection without a GPU fault: a device wait that nothing can satisfy gives up after its
bound, the kernel records MLMC_ERR_TIMEOUT in the plan's error word, the host reports it and the
error sticks to the plan, while the CUDA context stays usable for other plans."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _spec(pp, dtype=torch.float32):
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    return binding.ProblemSpec(*ts, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)


def test_bounded_wait_gives_up_and_the_error_sticks():
    pp = make_params(32, 256, 24, dtype=np.float32)
    with binding.Plan([_spec(pp)], c0=8, L=1, precision="bf16") as plan:
        t0 = time.perf_counter()
        plan.debug_bounded_wait(200_000_000)          # 0.2 s
        with pytest.raises(binding.MLMCError) as e:
            plan.synchronize()
        elapsed = time.perf_counter() - t0
        assert e.value.status == 4                     # MLMC_ERR_TIMEOUT
        assert 0.15 < elapsed < 10.0
        # every later call on this plan returns the same error
        with pytest.raises(binding.MLMCError) as e2:
            plan.level_stats(0, 0, 0, 8)
        assert e2.value.status == 4


def test_context_is_usable_after_a_timeout():
    pp = make_params(48, 512, 40, seed_A=5, seed_B=6, dtype=np.float32)
    with binding.Plan([_spec(pp)], c0=8, L=1, precision="bf16") as plan:
        plan.debug_bounded_wait(10_000_000)
        with pytest.raises(binding.MLMCError):
            plan.synchronize()
    # a new plan on the same device computes correct statistics
    lv = oracle.Levels(8, 2, 1)
    orc = oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                         problem_id=pp.problem_id)
    with binding.Plan([_spec(pp)], c0=8, L=1, precision="bf16") as plan:
        plan.level_stats(0, 1, 0, 40)
        n, mean, _ = plan.get_level_stats(0, 1)
        mref, _, magm = oracle.level_stats(orc, lv, 1, 0, 40)
        tau = 2.0**-7 + 2.0**-15 + (lv.cl(1) + 8) * 2.0**-23
        assert n == 40
        assert np.all(np.abs(mean.cpu().numpy() - mref) <= tau * magm)


def test_bounded_wait_rejects_bad_bounds():
    pp = make_params(16, 64, 16, dtype=np.float32)
    with binding.Plan([_spec(pp)], c0=4, L=1, precision="bf16") as plan:
        for bad in (0, -5, 20_000_000_000):
            with pytest.raises(binding.MLMCError) as e:
                plan.debug_bounded_wait(bad)
            assert e.value.status == 1


def test_injected_launch_failure_is_reported_and_sticks(monkeypatch):
    pp = make_params(32, 256, 24, dtype=np.float32)
    with binding.Plan([_spec(pp)], c0=8, L=1, precision="bf16") as plan:
        monkeypatch.setenv("MLMC_FAULT", "launch")
        with pytest.raises(binding.MLMCError) as e:
            plan.level_stats(0, 0, 0, 8)
        assert e.value.status == 2 and "injected" in str(e.value)
        with pytest.raises(binding.MLMCError) as e:
            plan.level_stats_batch([(0, 1, 0, 8)])
        assert e.value.status == 2
        monkeypatch.delenv("MLMC_FAULT")
        with pytest.raises(binding.MLMCError) as e:      # sticky
            plan.level_stats(0, 0, 0, 8)
        assert e.value.status == 2


def test_injected_cancel(monkeypatch):
    pp = make_params(32, 256, 24, dtype=np.float32)
    with binding.Plan([_spec(pp)], c0=8, L=1, precision="fp32") as plan:
        monkeypatch.setenv("MLMC_FAULT", "cancel")
        with pytest.raises(binding.MLMCError) as e:
            plan.level_stats(0, 0, 0, 8)
        assert e.value.status == 2
        monkeypatch.delenv("MLMC_FAULT")
        with pytest.raises(binding.MLMCError):
            plan.synchronize()
