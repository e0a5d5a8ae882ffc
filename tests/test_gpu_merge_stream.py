"""Chunk merges overlapped with the next batch's level kernel.

A level call cuts its chunks into batches (as many chunks as one set of the plan's partial
buffers holds, rounded for the tensor-core kernels to whole rounds of their persistent CTAs).
The merges of a batch run on a stream the plan owns, beside the level kernel of the next batch,
with two sets of partials in turn: batch i + 2 reuses the set of batch i only after its merges.
Checks, in BF16 (tensor cores) and FP64 (CUDA cores), for calls of about three to six batches,
against the same samples in calls of at most `batch` samples each (at most one batch each, so no
overlap):
  * N and the per-entry FP64 sums equal bit for bit: each entry's sum is one chain of additions
    in chunk order, whatever the launch boundaries;
  * M2 within rounding of the between-chunk terms, which are summed per launch (1e-12 relative in
    FP64, 1e-5 with FP32 partials); a partial set reused before its merge, or a read before the
    join, would move it by whole samples;
  * the states are read right after the calls (get_level_state synchronises the plan's stream),
    so the call's join of the merge stream is what makes its last batches visible.
"""
import numpy as np
import pytest
import torch

from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _plan(pp, precision, stream=None):
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev, dt) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    spec = binding.ProblemSpec(*ts, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)
    return binding.Plan([spec], c0=16, L=1, precision=precision, stream=stream)


# (precision, m = p, about the samples per batch at level 0: chunks of 64 samples, as many chunks
# per batch as 256 MB (tensor cores) or 64 MB (CUDA cores) of FP32 / FP64 m x p partials hold,
# M2 tolerance)
CASES = [("bf16", 512, 256 * 64, 1e-5), ("fp64", 128, 512 * 64, 1e-12)]


@pytest.mark.parametrize("precision,mp_side,batch,tol", CASES)
@pytest.mark.parametrize("nbatches", [3, 6])
def test_overlapped_merges_match_single_batch_calls(precision, mp_side, batch, tol, nbatches):
    if precision == "fp64" and nbatches == 6:
        pytest.skip("FP64 runs at a small fraction of the FP32 rate here; three batches cover it")
    pp = make_params(mp_side, 1024, mp_side, seed_A=21, seed_B=22, dtype=np.float64)
    total = nbatches * batch - batch // 2 + 37   # a ragged last batch
    side = torch.cuda.Stream()
    with _plan(pp, precision, stream=side) as one, _plan(pp, precision) as split:
        one.level_stats(0, 0, 0, total)
        s = 0
        while s < total:
            n = min(batch, total - s)
            split.level_stats(0, 0, s, n)
            s += n
        N1, s1, q1 = one.get_level_state(0, 0)
        N2, s2, q2 = split.get_level_state(0, 0)
    assert N1 == N2 == total
    assert torch.equal(s1, s2)
    assert np.isfinite(q1) and q1 > 0
    assert abs(q1 - q2) <= tol * q2
