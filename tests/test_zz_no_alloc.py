"""mlmc_level_stats_noalloc: level statistics for callers that cannot allocate device memory.

Callers inside CUDA-graph stream capture, inference-runtime plugins that must not allocate in
their enqueue step, and applications that hand all device memory to their own pool cannot go
through mlmc_plan (it allocates).  The no-alloc entry point keeps its scratch in a fixed array
of the library image instead.  This test calls it through the C ABI twice in a row (the second
call reuses the scratch the first one left behind) and compares each result (the sum of D and
the level's M2) with what the plan-based entry points (mlmc_level_stats + mlmc_get_level_state)
give for the same samples, within the FP64 parity tolerance of the other tests (1e-12 of the
summed term magnitudes); a problem near the size limit makes one call run several launches,
each folding its chunks into the outputs left by the one before; and a call captured into a
CUDA graph is replayed.

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    lib = binding.lib()
    f = lib.mlmc_level_stats_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert torch.cuda.is_available()


def _args(tensors, pp, c0, level, precision, dtype_code):
    M, S, Mp, Sp = tensors
    m, n = M.shape
    p = Mp.shape[1]
    prob = binding.Problem(m, n, p, M.data_ptr(), S.data_ptr(), M.stride(0), Mp.data_ptr(), Sp.data_ptr(),
                           Mp.stride(0), dtype_code, -1, pp.seed_A, pp.seed_B, pp.seed_idx, pp.problem_id)
    opts = binding.Options(c0, 2, level, binding.PRECISION[precision], 2, 1.0, 0, 0, 0)
    out_sum = torch.full((m, p), float("nan"), dtype=torch.float64, device=M.device)
    out_q = torch.full((1,), float("nan"), dtype=torch.float64, device=M.device)
    return prob, opts, out_sum, out_q


def _call(prob, opts, level, begin, count, out_sum, out_q, stream):
    return binding.lib().mlmc_level_stats_noalloc(ctypes.byref(prob), ctypes.byref(opts), level, begin, count,
                                                  out_sum.data_ptr(), out_q.data_ptr(), stream.cuda_stream)


def _noalloc(tensors, pp, c0, level, begin, count, precision, dtype_code, stream):
    prob, opts, out_sum, out_q = _args(tensors, pp, c0, level, precision, dtype_code)
    rc = _call(prob, opts, level, begin, count, out_sum, out_q, stream)
    return rc, out_sum, out_q


def _plan_state(tensors, pp, c0, L, level, begin, count, precision):
    spec = binding.ProblemSpec(*tensors, seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)
    with binding.Plan([spec], c0=c0, L=L, precision=precision) as plan:
        plan.level_stats(0, level, begin, count)
        N, s, M2 = plan.get_level_state(0, level)
        assert N == count
        return s.clone(), M2


@pytest.mark.parametrize("precision,np_dtype,t_dtype,code", [("fp64", np.float64, torch.float64, 0),
                                                              ("fp32", np.float32, torch.float32, 1)])
def test_noalloc_matches_plan_path_on_two_calls_in_a_row(precision, np_dtype, t_dtype, code):
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    m, n, p, c0, L = 70, 900, 45, 8, 3
    pp = make_params(m, n, p, seed_A=21, seed_B=22, seed_idx=23, problem_id=5, dtype=np_dtype)
    tensors = [torch.from_numpy(np.ascontiguousarray(x)).to(dev, t_dtype) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    orc = oracle.Problem(*pp.f64(), seed_A=21, seed_B=22, seed_idx=23, problem_id=5)
    lv = oracle.Levels(c0, 2, L)
    tol = 1e-12 if precision == "fp64" else (c0 * 2**L + 8) * 2.0**-24 + 2.0**-16
    for level, begin, count in [(2, 0, 40), (3, 13, 27)]:   # two calls in a row, second one ragged
        rc, s_na, q_na = _noalloc(tensors, pp, c0, level, begin, count, precision, code, stream)
        assert rc == 0, binding.lib().mlmc_last_error()
        s_plan, q_plan = _plan_state(tensors, pp, c0, L, level, begin, count, precision)
        torch.cuda.synchronize()
        _, _, magm = oracle.level_stats(orc, lv, level, begin, count)
        bound = tol * count * magm
        diff = np.abs(s_na.cpu().numpy() - s_plan.cpu().numpy())
        assert np.all(diff <= bound), diff.max()
        assert abs(float(q_na.item()) - q_plan) <= tol * count * float((magm**2).sum()) + 1e-12 * q_plan


def test_noalloc_near_its_size_limit_runs_several_launches():
    """m = p = 700 in FP64: one chunk of partials fills most of the 4 MiB scratch, so a call over
    50 samples starting at a ragged id runs seven launches (chunks of 8 ids), each merging into
    the outputs of the previous one; twice in a row, against the plan path."""
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    m, n, p, c0, L = 700, 300, 700, 8, 2
    pp = make_params(m, n, p, seed_A=31, seed_B=32, seed_idx=33, problem_id=2)
    tensors = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    orc = oracle.Problem(*pp.f64(), seed_A=31, seed_B=32, seed_idx=33, problem_id=2)
    lv = oracle.Levels(c0, 2, L)
    for level, begin, count in [(2, 3, 50), (1, 101, 50)]:
        rc, s_na, q_na = _noalloc(tensors, pp, c0, level, begin, count, "fp64", 0, stream)
        assert rc == 0, binding.lib().mlmc_last_error()
        s_plan, q_plan = _plan_state(tensors, pp, c0, L, level, begin, count, "fp64")
        torch.cuda.synchronize()
        # magnitude scale of one sample's terms (the oracle on one sample is enough for the bound)
        _, _, _, mag = oracle.sample(orc, lv, level, begin)
        diff = np.abs(s_na.cpu().numpy() - s_plan.cpu().numpy())
        assert np.all(diff <= 1e-12 * count * 4.0 * mag), diff.max()
        assert abs(float(q_na.item()) - q_plan) <= 1e-11 * q_plan


def test_noalloc_inside_cuda_graph_capture():
    """A warm-up call (it looks the scratch up), then a call captured into a CUDA graph on a side
    stream and replayed twice: each replay writes the plan path's result into the outputs."""
    dev = torch.device("cuda:0")
    m, n, p, c0, L = 70, 900, 45, 8, 3
    pp = make_params(m, n, p, seed_A=41, seed_B=42, seed_idx=43, problem_id=6)
    tensors = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    level, begin, count = 3, 5, 40
    prob, opts, out_sum, out_q = _args(tensors, pp, c0, level, "fp64", 0)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        assert _call(prob, opts, level, 0, 16, out_sum, out_q, side) == 0   # warm-up
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        rc = _call(prob, opts, level, begin, count, out_sum, out_q, side)
    assert rc == 0, binding.lib().mlmc_last_error()
    s_plan, q_plan = _plan_state(tensors, pp, c0, L, level, begin, count, "fp64")
    orc = oracle.Problem(*pp.f64(), seed_A=41, seed_B=42, seed_idx=43, problem_id=6)
    _, _, magm = oracle.level_stats(orc, oracle.Levels(c0, 2, L), level, begin, count)
    for _ in range(2):
        out_sum.fill_(float("nan"))
        out_q.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        diff = np.abs(out_sum.cpu().numpy() - s_plan.cpu().numpy())
        assert np.all(diff <= 1e-12 * count * magm), diff.max()
        assert abs(float(out_q.item()) - q_plan) <= 1e-11 * q_plan


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    m, n, p = 1024, 16, 1024   # 1024 * 1024 * 8 bytes of FP64 partials > 4 MiB
    pp = make_params(m, n, p)
    tensors = [torch.from_numpy(x).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    rc, s, q = _noalloc(tensors, pp, 4, 1, 0, 8, "fp64", 0, stream)
    assert rc == 1
    assert b"scratch" in binding.lib().mlmc_last_error()
    rc, _, _ = _noalloc(tensors, pp, 4, 1, 0, 8, "bf16", 0, stream)
    assert rc == 6
