"""Level variances where the mean dwarfs the spread of the samples.

A level's M2 = sum_s ||D_s - mean||_F^2 grows by Welford's update inside each chunk of samples
(kernels) and by Chan's pairwise update across chunks and calls (merge).  A one-pass form,
sum ||D||^2 - ||sum D||^2 / N, loses about log10(||mean||^2 / V) digits to cancellation; on the
workload below (every column of M equal, every row of M' equal, S = 1e-4 |M|) that ratio is about
8 * 10^8, so in FP32 a one-pass V would have no correct digit and in FP64 only six or seven.

Checks, on level 0 of that workload (c_0 = 16 slots, 2000 samples, chunks of 64 samples, calls
split at a ragged sample id so that a call starts inside a chunk and the merge starts from a
non-empty level):
  * every precision (the ratio is about 10^9 in FP64 and FP32, 1.5 * 10^7 in BF16, whose rounding
    noise adds to V): the plan's M2 against the two-pass M2 (FP64, mean first) of the plan's own
    samples, each read back through mlmc_debug_sample (the same kernel, one sample at a time):
    this isolates the accumulation of the statistics from the arithmetic of the samples.  FP64
    within 1e-12 relative.  FP32 partials (FP32 and BF16 paths): the chunk's running sum is FP32,
    so a deviation k D - sum_k carries the rounding of that sum, about u k^1.5 |mean| / 3 against
    k sigma (u = 2^-24): 3e-3 of it per deviation at this ratio, which averages down over the 128
    entries and 2000 samples to well below the 1e-3 bar;
  * FP64: V_0 against the oracle's Welford V_0 in sample order, within 1e-12 relative (the
    samples differ by rounding, 3e-16 of the magnitude of their terms, i.e. 1e-11 of sigma per
    entry, and that difference averages over entries and samples).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_concentrated_params

pytestmark = pytest.mark.gpu

M_, N_, P_ = 8, 64, 16
C0, L = 16, 2
NS = 2000
SPLIT = 1037   # a call boundary inside a chunk


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _plan(pp, precision):
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev, dt) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    spec = binding.ProblemSpec(*ts, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)
    return binding.Plan([spec], c0=C0, L=L, precision=precision)


def _params(precision):
    dt = np.float64 if precision == "fp64" else np.float32
    return make_concentrated_params(M_, N_, P_, seed_A=11, seed_B=12, seed_idx=13, dtype=dt)


# (precision, bar on M2, least ||mean||^2 / V, bar on the mean relative to max |mean|): BF16's own
# rounding noise (2^-8 of entries whose spread is 1e-4 of their size) raises its V, so its ratio
# is lower, still far beyond what a one-pass FP32 form survives; FP32 chunk sums of 64 samples
# carry 64 roundings of 2^-24
CASES = [("fp64", 1e-12, 1e8, 1e-12), ("fp32", 1e-3, 1e8, 64 * 2.0**-24), ("bf16", 1e-3, 1e7, 64 * 2.0**-24)]


@pytest.mark.parametrize("level", [0, 2])
@pytest.mark.parametrize("precision,tol,least_ratio,tol_mean", CASES)
def test_m2_matches_two_pass_of_own_samples(precision, tol, least_ratio, tol_mean, level):
    """Level 0 carries the large mean; level 2 (mean zero by the coupling) checks the tensor-core
    kernel's raw second moment of zero-mean levels against the same two-pass reference."""
    pp = _params(precision)
    with _plan(pp, precision) as plan:
        plan.level_stats(0, level, 0, SPLIT)
        plan.level_stats(0, level, SPLIT, NS - SPLIT)
        N, mean, M2 = plan.get_level_stats(0, level)
        assert N == NS
        D = np.stack([plan.debug_sample(0, level, s).cpu().numpy() for s in range(NS)])
    mu = D.mean(axis=0)
    M2_ref = float(((D - mu) ** 2).sum())
    ratio = float((mu ** 2).sum()) / (M2_ref / (NS - 1))
    rel = abs(M2 - M2_ref) / M2_ref
    print(f"{precision} level {level}: ||mean||^2 / V = {ratio:.3e}; M2 vs two-pass of its samples: {rel:.3e}")
    assert rel <= tol
    if level == 0:
        assert ratio > least_ratio
        assert np.abs(mean.cpu().numpy() - mu).max() <= tol_mean * np.abs(mu).max()
    else:
        assert ratio < 1e-2   # E[D_l] = 0: the level mean is sampling noise
        assert np.abs(mean.cpu().numpy() - mu).max() <= tol_mean * np.abs(D).max()


def test_fp64_v0_matches_oracle_welford():
    pp = _params("fp64")
    orc = oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                         problem_id=pp.problem_id)
    lv = oracle.Levels(C0, 2, L)
    mref, M2ref, magm = oracle.level_stats(orc, lv, 0, 0, NS)
    with _plan(pp, "fp64") as plan:
        plan.level_stats(0, 0, 0, SPLIT)
        plan.level_stats(0, 0, SPLIT, NS - SPLIT)
        N, mean, M2 = plan.get_level_stats(0, 0)
    rel = abs(M2 - M2ref) / M2ref
    print(f"fp64: V_0 {M2 / (N - 1):.6e} vs oracle {M2ref / (NS - 1):.6e}, rel. {rel:.3e}; "
          f"||mean||^2 / V = {float((mref ** 2).sum()) / (M2ref / (NS - 1)):.3e}")
    assert rel <= 1e-12
    assert np.all(np.abs(mean.cpu().numpy() - mref) <= 1e-12 * magm)


def test_merge_level_state_equals_one_plan():
    """mlmc_merge_level_state: the states of two plans holding disjoint sample ranges, merged with
    Chan's update, give the statistics of one plan holding both ranges (FP64, same regime)."""
    pp = _params("fp64")
    with _plan(pp, "fp64") as a, _plan(pp, "fp64") as b, _plan(pp, "fp64") as one:
        a.level_stats(0, 0, 0, SPLIT)
        b.level_stats(0, 0, SPLIT, NS - SPLIT)
        one.level_stats(0, 0, 0, NS)
        Nb, sb, M2b = b.get_level_state(0, 0)
        a.merge_level_state(0, 0, Nb, sb, M2b)
        Na, sa, M2a = a.get_level_state(0, 0)
        N1, s1, M21 = one.get_level_state(0, 0)
        assert Na == N1 == NS
        torch.testing.assert_close(sa, s1, rtol=1e-14, atol=0.0)
        assert abs(M2a - M21) <= 1e-12 * M21
        # the allocation and the stopping test read the merged state like any other
        assert a.allocate_levels(0, 0, 1.0) == one.allocate_levels(0, 0, 1.0)
