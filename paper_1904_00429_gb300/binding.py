"""ctypes binding of ``libmlmc.so`` (the C ABI of include/mlmc.h).

Argument marshalling only: every step of the estimator runs in the CUDA library.
PyTorch provides device memory and streams.  There is no fallback of any kind:
if the library is missing or was built for another machine, loading raises.

Names follow the C entry points: ``Plan`` wraps ``mlmc_plan`` / ``mlmc_plan_destroy``
and its methods ``level_stats``, ``get_level_stats``, ``estimate``, ``backward`` ... call
the functions of the same name.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmlmc.so")
MAX_LEVELS = 32

STATUS = {0: "MLMC_OK", 1: "MLMC_ERR_INVALID_ARG", 2: "MLMC_ERR_CUDA", 3: "MLMC_ERR_OOM",
          4: "MLMC_ERR_TIMEOUT", 5: "MLMC_ERR_NUMERIC", 6: "MLMC_ERR_UNSUPPORTED", 7: "MLMC_ERR_STATE"}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2, "fp8": 3, "fp8_e4m3": 3}
FUNCTION = {"identity": 0, "abs_step": 1}   # mlmc_function
SAMPLING = {"uniform": 0, "optimal": 1}     # mlmc_sampling
DTYPE = {torch.float64: 0, torch.float32: 1}


class MLMCError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("p", ctypes.c_int64),
                ("M_dev", ctypes.c_void_p), ("S_dev", ctypes.c_void_p), ("ldA", ctypes.c_int64),
                ("Mp_dev", ctypes.c_void_p), ("Sp_dev", ctypes.c_void_p), ("ldB", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("L", ctypes.c_int32),
                ("seed_A", ctypes.c_uint32), ("seed_B", ctypes.c_uint32),
                ("seed_idx", ctypes.c_uint32), ("problem_id", ctypes.c_uint32)]


class Options(ctypes.Structure):
    _fields_ = [("c0", ctypes.c_int32), ("ratio", ctypes.c_int32), ("L", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("pilot_n", ctypes.c_int64), ("nl_scale", ctypes.c_double),
                ("timeout_ns", ctypes.c_int64), ("tile_override", ctypes.c_int32), ("adjoint_batch_log2", ctypes.c_int32),
                ("f", ctypes.c_int32), ("adaptive_L", ctypes.c_int32), ("sampling", ctypes.c_int32)]


class Range(ctypes.Structure):
    _fields_ = [("prob", ctypes.c_int32), ("level", ctypes.c_int32), ("sample_begin", ctypes.c_uint64),
                ("count", ctypes.c_uint64)]


class Report(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("bias_unmet", ctypes.c_int32),
                ("N", ctypes.c_int64 * MAX_LEVELS), ("V", ctypes.c_double * MAX_LEVELS),
                ("cost", ctypes.c_double * MAX_LEVELS), ("mean_norm", ctypes.c_double * MAX_LEVELS),
                ("rmse_pred", ctypes.c_double), ("eps_abs", ctypes.c_double), ("outer_products", ctypes.c_double)]

    def as_dict(self) -> dict:
        L = self.L
        return {"L": L, "bias_unmet": bool(self.bias_unmet), "N": list(self.N[:L + 1]), "V": list(self.V[:L + 1]), "cost": list(self.cost[:L + 1]),
                "mean_norm": list(self.mean_norm[:L + 1]), "rmse_pred": self.rmse_pred, "eps_abs": self.eps_abs,
                "outer_products": self.outer_products}


_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Open libmlmc.so (raises if it has not been built: run ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, U64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "mlmc_plan": [P, I32, P, P, P],
            "mlmc_plan_host": [P, I32, P, P, P],
            "mlmc_telescoping_sum_host": [P, P],
            "mlmc_plan_destroy": [P],
            "mlmc_level_stats": [P, I32, I32, U64, U64],
            "mlmc_level_stats_batch": [P, P, I32],
            "mlmc_get_batch_tile": [P, P, P],
            "mlmc_get_level_stats": [P, I32, I32, P, P, P],
            "mlmc_get_level_state": [P, I32, I32, P, P, P],
            "mlmc_set_level_state": [P, I32, I32, U64, P, D],
            "mlmc_merge_level_state": [P, I32, I32, U64, P, D],
            "mlmc_allocate_levels": [P, I32, I32, D, P],
            "mlmc_bias_test": [P, I32, I32, D, P, P],
            "mlmc_reset_level_stats": [P, I32, I32],
            "mlmc_estimate": [P, P, P, P],
            "mlmc_telescoping_sum": [P, P],
            "mlmc_allocate": [P, P, P],
            "mlmc_launch_count": [P, P],
            "mlmc_backward": [P, P, P, P, P, P],
            "mlmc_synchronize": [P],
            "mlmc_debug_philox": [P, P, I64, P, P],
            "mlmc_debug_indices": [P, I32, I32, U64, I64, I64, P],
            "mlmc_debug_normals": [P, I32, I32, I32, U64, I64, I64, I64, P],
            "mlmc_debug_sample": [P, I32, I32, U64, P],
            "mlmc_debug_bounded_wait": [P, I64],
            "mlmc_measure_generation_rate": [P, ctypes.POINTER(ctypes.c_double)],
            "mlmc_measure_peaks": [P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.mlmc_last_error.argtypes = []
        L.mlmc_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(status: int, where: str):
    if status != 0:
        msg = lib().mlmc_last_error().decode(errors="replace")
        raise MLMCError(status, where, msg)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


@dataclass
class ProblemSpec:
    """One problem: M, S (m x n) and Mp, Sp (n x p) as 2-D CUDA tensors (float32 or float64)."""
    M: torch.Tensor
    S: torch.Tensor
    Mp: torch.Tensor
    Sp: torch.Tensor
    seed_A: int = 0
    seed_B: int = 1
    seed_idx: int = 2
    problem_id: int = 0
    L: int = -1

    def shape(self):
        return self.M.shape[0], self.M.shape[1], self.Mp.shape[1]


class Plan:
    """A plan over one or more problems sharing the level schedule c_l = c0 * ratio**l.

    precision: "fp64", "fp32" (CUDA cores), "bf16" or "fp8" (tensor cores).  f: "identity"
    (E[AB]) or "abs_step" (E[f(AB)] with f(x) = |x| H(2 - x); FP64/FP32/BF16).  adaptive_L: let
    estimate() choose the finest level by Alg. 2's while loop, up to L.  sampling: "uniform"
    (xi^u) or "optimal" (xi** of Thm 3.1; FP64/FP32/BF16).  The fields mirror mlmc_options."""

    def __init__(self, problems: Sequence[ProblemSpec], *, c0: int, L: int, ratio: int = 2,
                 precision: str = "fp32", pilot_n: int = 256, nl_scale: float = 1.0,
                 timeout_ns: int = 0, tile_override: int = 0, adjoint_batch_log2: int = 0,
                 f: str = "identity", adaptive_L: bool = False, sampling: str = "uniform", stream=None,
                 host: bool = False):
        """host=True: the parameters are CPU tensors (pinned for asynchronous copies); the plan is
        made by mlmc_plan_host, which copies them to the current CUDA device itself."""
        self.problems = list(problems)
        self.host = host
        self.device = torch.device("cuda", torch.cuda.current_device()) if host else self.problems[0].M.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        arr = (Problem * len(self.problems))()
        self.shapes = []
        self.levels = []
        for q, pr in enumerate(self.problems):
            for t in (pr.M, pr.S, pr.Mp, pr.Sp):
                if t.is_cuda == host or t.dim() != 2 or t.dtype not in DTYPE or t.stride(1) != 1:
                    raise ValueError("parameters must be 2-D row-major float32/float64 " +
                                     ("CPU tensors (host=True)" if host else "CUDA tensors"))
            if pr.S.shape != pr.M.shape or pr.Sp.shape != pr.Mp.shape or pr.M.shape[1] != pr.Mp.shape[0]:
                raise ValueError("inconsistent parameter shapes")
            dtypes = {pr.M.dtype, pr.S.dtype, pr.Mp.dtype, pr.Sp.dtype}
            if len(dtypes) != 1:
                raise ValueError("the four parameter matrices must share one dtype")
            m, n, p = pr.shape()
            if pr.M.stride(0) != pr.S.stride(0) or pr.Mp.stride(0) != pr.Sp.stride(0):
                raise ValueError("M and S (and Mp and Sp) must share a leading dimension")
            arr[q] = Problem(m, n, p, pr.M.data_ptr(), pr.S.data_ptr(), pr.M.stride(0),
                             pr.Mp.data_ptr(), pr.Sp.data_ptr(), pr.Mp.stride(0), DTYPE[pr.M.dtype],
                             pr.L, pr.seed_A, pr.seed_B, pr.seed_idx, pr.problem_id)
            self.shapes.append((m, n, p))
            self.levels.append(pr.L if pr.L >= 0 else L)
        self.options = Options(c0, ratio, L, PRECISION[precision], pilot_n, nl_scale, timeout_ns, tile_override,
                               adjoint_batch_log2, FUNCTION[f], int(bool(adaptive_L)), SAMPLING[sampling])
        self.precision = precision
        self.c0, self.ratio, self.L = c0, ratio, L
        self.pilot_n = pilot_n
        self.nl_scale = nl_scale
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            make = lib().mlmc_plan_host if host else lib().mlmc_plan
            _check(make(arr, len(self.problems), ctypes.byref(self.options), _stream_handle(self.stream),
                        ctypes.byref(h)), "mlmc_plan_host" if host else "mlmc_plan")
        self._h = h

    # -- lifetime ---------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mlmc_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def cl(self, l: int) -> int:
        return self.c0 * self.ratio ** l

    def _out(self, *shape, dtype=torch.float64):
        return torch.empty(*shape, dtype=dtype, device=self.device)

    # -- Alg. 1, incremental ------------------------------------------------------------------
    def level_stats(self, prob: int, level: int, begin: int, count: int):
        _check(lib().mlmc_level_stats(self._h, prob, level, begin, count), "mlmc_level_stats")

    def level_stats_batch(self, ranges):
        """``ranges``: iterable of (prob, level, begin, count); one batched launch sequence."""
        ranges = list(ranges)
        arr = (Range * max(1, len(ranges)))(*[Range(int(q), int(l), int(b), int(c)) for q, l, b, c in ranges])
        _check(lib().mlmc_level_stats_batch(self._h, arr, len(ranges)), "mlmc_level_stats_batch")

    def batch_tile(self):
        """(tile id of the batched launches, autotuner ms per candidate tile id)."""
        tid = ctypes.c_int32()
        ms = (ctypes.c_double * 9)()
        _check(lib().mlmc_get_batch_tile(self._h, ctypes.byref(tid), ms), "mlmc_get_batch_tile")
        ids = (1032, 1064, 1128, 1256, 2032, 2064, 2128, 2256, 3256)
        return tid.value, {i: ms[k] for k, i in enumerate(ids) if ms[k] >= 0}

    def get_level_stats(self, prob: int, level: int):
        """(N, mean (m x p FP64 CUDA tensor), M2 = sum_s ||D_s - mean||_F^2)."""
        m, _, p = self.shapes[prob]
        mean = self._out(m, p)
        N = ctypes.c_uint64()
        M2 = ctypes.c_double()
        _check(lib().mlmc_get_level_stats(self._h, prob, level, ctypes.byref(N), _ptr(mean), ctypes.byref(M2)),
               "mlmc_get_level_stats")
        return N.value, mean, M2.value

    def get_level_state(self, prob: int, level: int):
        """(N, sum of D (m x p FP64 CUDA tensor), M2 = sum_s ||D_s - mean||_F^2)."""
        m, _, p = self.shapes[prob]
        s = self._out(m, p)
        N = ctypes.c_uint64()
        q = ctypes.c_double()
        _check(lib().mlmc_get_level_state(self._h, prob, level, ctypes.byref(N), _ptr(s), ctypes.byref(q)),
               "mlmc_get_level_state")
        return N.value, s, q.value

    def set_level_state(self, prob: int, level: int, N: int, sum_dev: torch.Tensor, M2: float):
        _check(lib().mlmc_set_level_state(self._h, prob, level, N, _ptr(self._dev_f64(sum_dev)), float(M2)),
               "mlmc_set_level_state")

    def merge_level_state(self, prob: int, level: int, N: int, sum_dev: torch.Tensor, M2: float):
        """Fold another (N, sum, M2) of the same level into the held one (Chan's update, in the library)."""
        _check(lib().mlmc_merge_level_state(self._h, prob, level, N, _ptr(self._dev_f64(sum_dev)), float(M2)),
               "mlmc_merge_level_state")

    def _dev_f64(self, t: torch.Tensor) -> torch.Tensor:
        t = t.to(device=self.device, dtype=torch.float64).contiguous()
        self._keep = t   # alive until the (synchronous) call has used it
        return t

    def reset(self, prob: int, level: int = -1):
        _check(lib().mlmc_reset_level_stats(self._h, prob, level), "mlmc_reset_level_stats")

    # -- Alg. 2 ---------------------------------------------------------------------------------
    def estimate(self, eps_abs):
        """Returns (list of m x p FP64 estimates, list of report dicts)."""
        nprob = len(self.problems)
        if not hasattr(eps_abs, "__len__"):
            eps_abs = [float(eps_abs)] * nprob
        eps = (ctypes.c_double * nprob)(*[float(e) for e in eps_abs])
        total = sum(m * p for m, _, p in self.shapes)
        y = self._out(total)
        reps = (Report * nprob)()
        _check(lib().mlmc_estimate(self._h, eps, _ptr(y), reps), "mlmc_estimate")
        return self._split(y), [r.as_dict() for r in reps]

    def allocate(self, eps_abs):
        """N_l of the allocation (Remark 3.6) from the statistics held now, per problem."""
        nprob = len(self.problems)
        if not hasattr(eps_abs, "__len__"):
            eps_abs = [float(eps_abs)] * nprob
        eps = (ctypes.c_double * nprob)(*[float(e) for e in eps_abs])
        out = (ctypes.c_int64 * (nprob * MAX_LEVELS))()
        _check(lib().mlmc_allocate(self._h, eps, out), "mlmc_allocate")
        return [list(out[q * MAX_LEVELS:q * MAX_LEVELS + self.levels[q] + 1]) for q in range(nprob)]

    def allocate_levels(self, prob: int, L: int, eps_abs: float):
        """N_l of levels 0..L of one problem (Remark 3.6, one round of Alg. 2)."""
        out = (ctypes.c_int64 * (L + 1))()
        _check(lib().mlmc_allocate_levels(self._h, prob, L, float(eps_abs), out), "mlmc_allocate_levels")
        return list(out)

    def bias_test(self, prob: int, L: int, eps_abs: float):
        """(met, ||Y_L||_F): Alg. 2's stopping test on level L (Remark 3.5)."""
        met = ctypes.c_int32()
        nrm = ctypes.c_double()
        _check(lib().mlmc_bias_test(self._h, prob, L, float(eps_abs), ctypes.byref(met), ctypes.byref(nrm)),
               "mlmc_bias_test")
        return bool(met.value), nrm.value

    def launch_count(self) -> int:
        c = ctypes.c_uint64()
        _check(lib().mlmc_launch_count(self._h, ctypes.byref(c)), "mlmc_launch_count")
        return c.value

    def telescoping_sum(self):
        total = sum(m * p for m, _, p in self.shapes)
        y = self._out(total)
        _check(lib().mlmc_telescoping_sum(self._h, _ptr(y)), "mlmc_telescoping_sum")
        return self._split(y)

    def telescoping_sum_host(self, out: Optional[torch.Tensor] = None):
        """Yhat written to host memory by mlmc_telescoping_sum_host (plans made with host=True);
        ``out``: an optional (pinned) FP64 CPU tensor of sum m p elements."""
        total = sum(m * p for m, _, p in self.shapes)
        if out is None:
            out = torch.empty(total, dtype=torch.float64)
        if out.is_cuda or out.dtype != torch.float64 or out.numel() != total or not out.is_contiguous():
            raise ValueError("out must be a contiguous FP64 CPU tensor of sum m p elements")
        _check(lib().mlmc_telescoping_sum_host(self._h, _ptr(out)), "mlmc_telescoping_sum_host")
        return self._split(out)

    def _split(self, flat: torch.Tensor):
        out, off = [], 0
        for m, _, p in self.shapes:
            out.append(flat[off:off + m * p].view(m, p))
            off += m * p
        return out

    # -- adjoint ---------------------------------------------------------------------------------
    def backward(self, G: Sequence[torch.Tensor], grads: Optional[Sequence[Sequence[torch.Tensor]]] = None):
        """Gradient of sum_q <G_q, Yhat_q> w.r.t. (M, S, Mp, Sp) of every problem.

        Returns one (dM, dS, dMp, dSp) tuple per problem, shaped and strided like the
        problem's parameters (or written into ``grads`` when given)."""
        if len(G) != len(self.problems):
            raise ValueError("one upstream gradient per problem")
        for g, (m, _, p) in zip(G, self.shapes):
            if tuple(g.shape) != (m, p) or g.device != self.device:
                raise ValueError("each G must be an m x p tensor on the plan's device")
        G_flat = torch.cat([g.reshape(-1).to(torch.float64) for g in G]).contiguous()
        if grads is None:
            grads = [tuple(torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=t.device)
                           for t in (pr.M, pr.S, pr.Mp, pr.Sp)) for pr in self.problems]
        else:
            for gr, pr in zip(grads, self.problems):
                for d, t in zip(gr, (pr.M, pr.S, pr.Mp, pr.Sp)):
                    if d.shape != t.shape or d.stride() != t.stride() or d.dtype != t.dtype:
                        raise ValueError("gradient buffers must match the parameters' shape, strides and dtype")
        n = len(self.problems)
        ptrs = [(ctypes.c_void_p * n)(*[g[i].data_ptr() for g in grads]) for i in range(4)]
        _check(lib().mlmc_backward(self._h, _ptr(G_flat), *ptrs), "mlmc_backward")
        return grads

    def synchronize(self):
        _check(lib().mlmc_synchronize(self._h), "mlmc_synchronize")

    # -- verification hooks ------------------------------------------------------------------
    def debug_indices(self, prob: int, level: int, sample: int, t0: int, count: int) -> torch.Tensor:
        out = self._out(count, dtype=torch.int64)
        _check(lib().mlmc_debug_indices(self._h, prob, level, sample, t0, count, _ptr(out)), "mlmc_debug_indices")
        return out

    def debug_normals(self, prob: int, which: int, level: int, sample: int, k: int, row0: int,
                      count: int) -> torch.Tensor:
        out = self._out(count)
        _check(lib().mlmc_debug_normals(self._h, prob, which, level, sample, k, row0, count, _ptr(out)),
               "mlmc_debug_normals")
        return out

    def debug_bounded_wait(self, timeout_ns: int):
        """Launch a kernel whose bounded wait must give up (failure-detection check)."""
        _check(lib().mlmc_debug_bounded_wait(self._h, int(timeout_ns)), "mlmc_debug_bounded_wait")

    def debug_sample(self, prob: int, level: int, sample: int) -> torch.Tensor:
        m, _, p = self.shapes[prob]
        out = self._out(m, p)
        _check(lib().mlmc_debug_sample(self._h, prob, level, sample, _ptr(out)), "mlmc_debug_sample")
        return out


def debug_philox(ctr: torch.Tensor, key: torch.Tensor, stream=None) -> torch.Tensor:
    """Philox4x32-10 blocks on the device: ctr (count x 4) and key (count x 2) int32 CUDA tensors
    holding the 32-bit words; returns count x 4 int32 words."""
    count = ctr.shape[0]
    out = torch.empty(count, 4, dtype=torch.int32, device=ctr.device)
    _check(lib().mlmc_debug_philox(_ptr(ctr.contiguous()), _ptr(key.contiguous()), count, _ptr(out),
                                   _stream_handle(stream)), "mlmc_debug_philox")
    return out


def generation_rate(stream=None) -> float:
    """Entries per second the GPU generates on their own (Philox4x32-10, special-function
    Box-Muller, M + S z, bfloat16) at full occupancy: the generation bound of the
    reduced-precision level kernels.  Synchronises the stream."""
    out = ctypes.c_double(0.0)
    _check(lib().mlmc_measure_generation_rate(_stream_handle(stream), ctypes.byref(out)),
           "mlmc_measure_generation_rate")
    return out.value


def measure_peaks(stream=None) -> dict:
    """Measured operations per second of this GPU (mlmc_measure_peaks): FP32 and FP64 FLOP/s
    (2 per fused multiply-add), INT32 multiply-adds/s and special-function sines/s."""
    out = (ctypes.c_double * 4)()
    _check(lib().mlmc_measure_peaks(_stream_handle(stream), out), "mlmc_measure_peaks")
    return {"fp32_flops": 2.0 * out[0], "fp64_flops": 2.0 * out[1], "int32_imad_per_s": out[2],
            "mufu_sin_per_s": out[3]}
