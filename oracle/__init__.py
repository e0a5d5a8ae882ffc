"""FP64 CPU oracle of the MLMC estimator for E[AB] (Wu & Polydorides, arXiv:1904.00429).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; the product package never imports it.  The
arithmetic lives in ``mlmc_oracle.c`` (plain C, FP64, single-threaded); this module
compiles it with gcc on first use and marshals numpy arrays through ctypes.

Every function mirrors one C entry point; see ``mlmc_oracle.h`` for the paper
passage each one restates (Eq. matrixsketch, Alg. 1, Eq. hatYl, Remark 3.6,
Alg. 2, Eq. hatY) and for the Philox counter layout of the random draws.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlmc_oracle.c")
_HDR = os.path.join(_HERE, "mlmc_oracle.h")
_LIB = os.path.join(_HERE, "libmlmc_oracle.so")

QUANT_NONE, QUANT_BF16, QUANT_E4M3, QUANT_E4M3_RNE = 0, 1, 2, 3
F_IDENTITY, F_ABS_STEP = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libmlmc_oracle.so`` (gcc, -O2, no FP contraction
    so that x86-64 and aarch64 hosts round identically)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("p", ctypes.c_int64),
                ("M", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("Mp", ctypes.c_void_p), ("Sp", ctypes.c_void_p),
                ("seed_A", ctypes.c_uint32), ("seed_B", ctypes.c_uint32),
                ("seed_idx", ctypes.c_uint32), ("problem_id", ctypes.c_uint32),
                ("q", ctypes.c_void_p), ("Q", ctypes.c_void_p)]


class _Levels(ctypes.Structure):
    _fields_ = [("c0", ctypes.c_int64), ("R", ctypes.c_int64), ("L", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P, D, I64, U32, U64, I = (ctypes.c_void_p, ctypes.c_double, ctypes.c_int64,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int)
            sig = {
                "orc_philox4x32_10": (None, [P, P, P]),
                "orc_philox4x64_10": (None, [P, P, P]),
                "orc_uniform": (D, [U32]),
                "orc_normal": (D, [U32, U32, I, U64, I64, I64]),
                "orc_index": (I64, [U32, U32, I, U64, I64, I64]),
                "orc_cl": (I64, [P, I]),
                "orc_cost": (D, [P, I]),
                "orc_round_bf16": (D, [D]),
                "orc_round_e4m3": (D, [D]),
                "orc_round_e4m3_sr": (D, [D, U32]),
                "orc_e4m3_dither": (U32, [U32, U32, I, U64, I64, I64]),
                "orc_e4m3_block_scale": (D, [D]),
                "orc_sketch": (None, [I64, I64, I64, P, P, P, I64, I64, I64, P]),
                "orc_sample": (None, [P, P, I, U64, I, P, P, P, P]),
                "orc_level_stats": (None, [P, P, I, U64, U64, I, P, P, P]),
                "orc_allocate": (I, [I, P, P, D, D, I64, P]),
                "orc_estimate": (I, [P, P, D, I64, D, I, P, P, P, P]),
                "orc_adjoint": (None, [P, P, P, P, I, P, P, P, P]),
                "orc_f": (D, [I, D]),
                "orc_xi_optimal": (None, [P, P, P]),
                "orc_index_xi": (I64, [U32, U32, I, U64, I64, I64, P, P]),
                "orc_sample_f": (None, [P, P, I, U64, I, I, P, P, P, P]),
                "orc_level_stats_f": (None, [P, P, I, U64, U64, I, I, P, P, P]),
                "orc_estimate_f": (I, [P, P, D, I64, D, I, I, I, P, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """One E[AB] problem: A = M + S o Z (m x n), B = M' + S' o Z' (n x p), FP64 row-major."""

    def __init__(self, M, S, Mp, Sp, seed_A=0, seed_B=1, seed_idx=2, problem_id=0, sampling: str = "uniform"):
        """sampling: "uniform" (xi^u, Eq. unique) or "optimal" (xi** of Thm 3.1)."""
        self.M, self.S, self.Mp, self.Sp = _f64(M), _f64(S), _f64(Mp), _f64(Sp)
        m, n = self.M.shape
        n2, p = self.Mp.shape
        assert self.S.shape == (m, n) and self.Sp.shape == (n2, p) and n2 == n
        self.m, self.n, self.p = m, n, p
        self.seeds = (seed_A, seed_B, seed_idx, problem_id)
        self._c = _Problem(m, n, p, _ptr(self.M), _ptr(self.S), _ptr(self.Mp), _ptr(self.Sp),
                           seed_A, seed_B, seed_idx, problem_id, None, None)
        self.q = self.Q = None
        if sampling == "optimal":
            self.q, self.Q = np.zeros(n), np.zeros(n)
            lib().orc_xi_optimal(ctypes.byref(self._c), _ptr(self.q), _ptr(self.Q))
            self._c.q, self._c.Q = _ptr(self.q), _ptr(self.Q)
        elif sampling != "uniform":
            raise ValueError(sampling)

    @property
    def xi(self):
        """The sampling probabilities (uniform: 1/n each)."""
        return np.full(self.n, 1.0 / self.n) if self.Q is None else self.q / self.Q[-1]

    @property
    def ref(self):
        return ctypes.byref(self._c)


class Levels:
    """c_l = c0 * R**l for l = 0..L."""

    def __init__(self, c0: int, R: int, L: int):
        self.c0, self.R, self.L = c0, R, L
        self._c = _Levels(c0, R, L)

    @property
    def ref(self):
        return ctypes.byref(self._c)

    def cl(self, l: int) -> int:
        return int(lib().orc_cl(self.ref, l))

    def cost(self, l: int) -> float:
        return float(lib().orc_cost(self.ref, l))


def philox4x32(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(w: int) -> float:
    return lib().orc_uniform(w)


def normal(seed, problem_id, l, s, row, k) -> float:
    return lib().orc_normal(seed, problem_id, l, s, row, k)


def index_xi(pr: "Problem", l, s, t) -> int:
    """Index of slot t under the problem's xi** (inverse of its cumulative law)."""
    return int(lib().orc_index_xi(pr.seeds[2], pr.seeds[3], l, s, t, pr.n, _ptr(pr.q), _ptr(pr.Q)))


def index(seed_idx, problem_id, l, s, t, n) -> int:
    return int(lib().orc_index(seed_idx, problem_id, l, s, t, n))


def round_bf16(x: float) -> float:
    return lib().orc_round_bf16(x)


def round_e4m3(x: float) -> float:
    return lib().orc_round_e4m3(x)


def round_e4m3_sr(y: float, d: int) -> float:
    return lib().orc_round_e4m3_sr(y, d)


def e4m3_dither(seed, problem_id, l, s, row, t) -> int:
    return int(lib().orc_e4m3_dither(seed, problem_id, l, s, row, t))


def e4m3_block_scale(absmax: float) -> float:
    return lib().orc_e4m3_block_scale(absmax)


def sketch(A, B, idx, off=0, stride=1, cnt=None) -> np.ndarray:
    """(n / cnt) sum_j A[:, idx[off + j*stride]] B[idx[off + j*stride], :]  (Eq. matrixsketch)."""
    A, B = _f64(A), _f64(B)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m, n = A.shape
    p = B.shape[1]
    if cnt is None:
        cnt = (len(idx) - off + stride - 1) // stride
    out = np.zeros((m, p))
    lib().orc_sketch(m, n, p, _ptr(A), _ptr(B), _ptr(idx), off, stride, cnt, _ptr(out))
    return out


def f(fkind: int, x: float) -> float:
    """The targeted function (F_IDENTITY, or F_ABS_STEP: |x| H(2 - x) with H(0) = 1)."""
    return lib().orc_f(fkind, float(x))


def sample(pr: Problem, lv: Levels, l: int, s: int, quant: int = QUANT_NONE, fkind: int = F_IDENTITY):
    """One coupled sample: returns (D, P_fine, P_coarse, mag), each m x p; D = f(P_fine) -
    f(P_coarse) (f(P_fine) at level 0)."""
    shp = (pr.m, pr.p)
    D, Pf, Pc, mag = np.zeros(shp), np.zeros(shp), np.zeros(shp), np.zeros(shp)
    lib().orc_sample_f(pr.ref, lv.ref, l, s, quant, fkind, _ptr(D), _ptr(Pf), _ptr(Pc), _ptr(mag))
    return D, Pf, Pc, mag


def level_stats(pr: Problem, lv: Levels, l: int, s0: int, N: int, quant: int = QUANT_NONE,
                fkind: int = F_IDENTITY):
    """Returns (mean m x p, M2 total, mag_mean m x p) over samples s0 .. s0+N-1."""
    mean = np.zeros((pr.m, pr.p))
    mag = np.zeros((pr.m, pr.p))
    M2 = ctypes.c_double(0.0)
    lib().orc_level_stats_f(pr.ref, lv.ref, l, s0, N, quant, fkind, _ptr(mean), ctypes.addressof(M2), _ptr(mag))
    return mean, M2.value, mag


def allocate(V, C, eps: float, nl_scale: float = 1.0, pilot: int = 0) -> np.ndarray:
    V, C = _f64(V), _f64(C)
    L = len(V) - 1
    Nl = np.zeros(L + 1, dtype=np.int64)
    rc = lib().orc_allocate(L, _ptr(V), _ptr(C), eps, nl_scale, pilot, _ptr(Nl))
    if rc != 0:
        raise ValueError("orc_allocate rejected its arguments")
    return Nl


def estimate(pr: Problem, lv: Levels, eps: float, pilot: int = 256, nl_scale: float = 1.0,
             quant: int = QUANT_NONE):
    """Alg. 2 with L fixed.  Returns (Yhat, Nl, V, means)."""
    Y = np.zeros((pr.m, pr.p))
    Nl = np.zeros(lv.L + 1, dtype=np.int64)
    V = np.zeros(lv.L + 1)
    means = np.zeros((lv.L + 1, pr.m, pr.p))
    rc = lib().orc_estimate(pr.ref, lv.ref, eps, pilot, nl_scale, quant, _ptr(Y), _ptr(Nl), _ptr(V),
                            _ptr(means))
    if rc != 0:
        raise ValueError("orc_estimate rejected its arguments")
    return Y, Nl, V, means


def estimate_f(pr: Problem, lv: Levels, eps: float, fkind: int = F_IDENTITY, adaptive: bool = False,
               pilot: int = 256, nl_scale: float = 1.0, quant: int = QUANT_NONE):
    """Alg. 2 with the targeted function, L fixed at lv.L or chosen adaptively up to lv.L.
    Returns (Yhat, L, Nl[:L+1], V[:L+1], means[:L+1])."""
    Y = np.zeros((pr.m, pr.p))
    Nl = np.zeros(lv.L + 1, dtype=np.int64)
    V = np.zeros(lv.L + 1)
    means = np.zeros((lv.L + 1, pr.m, pr.p))
    L = ctypes.c_int(-1)
    rc = lib().orc_estimate_f(pr.ref, lv.ref, eps, pilot, nl_scale, quant, fkind, int(bool(adaptive)), _ptr(Y),
                              ctypes.addressof(L), _ptr(Nl), _ptr(V), _ptr(means))
    if rc != 0:
        raise ValueError("orc_estimate_f rejected its arguments")
    k = L.value
    return Y, k, Nl[:k + 1], V[:k + 1], means[:k + 1]


def adjoint(pr: Problem, lv: Levels, Nl, G, quant: int = QUANT_NONE):
    """Gradient of <G, Yhat> with respect to (M, S, M', S') with the draws held fixed."""
    Nl = np.ascontiguousarray(Nl, dtype=np.int64)
    G = _f64(G)
    dM, dS = np.zeros((pr.m, pr.n)), np.zeros((pr.m, pr.n))
    dMp, dSp = np.zeros((pr.n, pr.p)), np.zeros((pr.n, pr.p))
    lib().orc_adjoint(pr.ref, lv.ref, _ptr(Nl), _ptr(G), quant, _ptr(dM), _ptr(dS), _ptr(dMp),
                      _ptr(dSp))
    return dM, dS, dMp, dSp
