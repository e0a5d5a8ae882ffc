"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle's tests.

This module holds no arithmetic of the estimator: it only draws the parameter
matrices of the random-matrix laws and the problem shapes.  The random numbers
the method itself consumes (sampled indices, the Gaussian Z of every entry) are
not drawn here; each side computes them from the Philox4x32-10 definition.

Laws (the Gaussian reparameterisation A = M + S o Z, B = M' + S' o Z', Z ~ N(0,1)):
  * "uniform":  M ~ U[-1, 1],  S ~ U[0.1, 1]     (plain, precision and adjoint workloads)
  * "gauss":    M ~ N(0, 1),   S ~ U[0.05, 2]    (batched workload)
Parameters of A come from seed_A, those of B from seed_B; each seed drives its own
NumPy Philox stream with key 1000 + seed.  Values are produced in FP64 and, when a
FP32 workload asks for it, rounded once to FP32, so that the device and the oracle
see bit-identical parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LAWS = ("uniform", "gauss")


def _rng(seed: int, tag: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[1000 + int(seed), int(tag)]))


def _draw_pair(rng: np.random.Generator, shape, law: str):
    if law == "uniform":
        M = rng.uniform(-1.0, 1.0, size=shape)
        S = rng.uniform(0.1, 1.0, size=shape)
    elif law == "gauss":
        M = rng.standard_normal(size=shape)
        S = rng.uniform(0.05, 2.0, size=shape)
    else:
        raise ValueError(f"unknown law {law!r}")
    return M, S


@dataclass
class ProblemParams:
    """Parameters of one problem.  M, S are m x n; Mp, Sp are n x p (row-major)."""
    M: np.ndarray
    S: np.ndarray
    Mp: np.ndarray
    Sp: np.ndarray
    seed_A: int = 0
    seed_B: int = 1
    seed_idx: int = 2
    problem_id: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.M.shape[0], self.M.shape[1], self.Mp.shape[1]

    def as_dtype(self, dtype) -> "ProblemParams":
        return ProblemParams(*(np.ascontiguousarray(x, dtype=dtype) for x in (self.M, self.S, self.Mp, self.Sp)),
                             self.seed_A, self.seed_B, self.seed_idx, self.problem_id, dict(self.meta))

    def f64(self):
        """The four matrices as FP64 (exact widening of whatever precision they hold)."""
        return tuple(np.asarray(x, dtype=np.float64) for x in (self.M, self.S, self.Mp, self.Sp))

    def exact_mean(self) -> np.ndarray:
        """E[AB] = M M' in FP64 (entries are independent and E[Z] = 0)."""
        M, _, Mp, _ = self.f64()
        return M @ Mp


def make_params(m: int, n: int, p: int, *, law: str = "uniform", seed_A: int = 0, seed_B: int = 1,
                seed_idx: int = 2, problem_id: int = 0, dtype=np.float64) -> ProblemParams:
    """Parameter matrices of one problem, drawn from the named law and rounded to ``dtype``."""
    M, S = _draw_pair(_rng(seed_A, problem_id), (m, n), law)
    Mp, Sp = _draw_pair(_rng(seed_B, problem_id), (n, p), law)
    pp = ProblemParams(M, S, Mp, Sp, seed_A, seed_B, seed_idx, problem_id, {"law": law})
    return pp.as_dtype(dtype)


def make_concentrated_params(m: int, n: int, p: int, *, spread: float = 1e-4, seed_A: int = 0, seed_B: int = 1,
                             seed_idx: int = 2, problem_id: int = 0, dtype=np.float64) -> ProblemParams:
    """A problem whose sketches barely vary: every column of M is the same vector u and every
    row of M' the same vector v (u, v ~ U[0.5, 1.5]), and S = spread u o U[0.5, 1],
    S' = spread U[0.5, 1] o v.  A sampled outer product is then u v^T up to O(spread), so the
    level-0 mean (about n u v^T) exceeds the spread of the samples by far more than 10^4: the
    regime in which a variance must not be formed as a difference of large sums."""
    ra, rb = _rng(seed_A, problem_id), _rng(seed_B, problem_id)
    u = ra.uniform(0.5, 1.5, size=(m, 1))
    v = rb.uniform(0.5, 1.5, size=(1, p))
    M = np.repeat(u, n, axis=1)
    S = spread * u * ra.uniform(0.5, 1.0, size=(m, n))
    Mp = np.repeat(v, n, axis=0)
    Sp = spread * v * rb.uniform(0.5, 1.0, size=(n, p))
    pp = ProblemParams(M, S, Mp, Sp, seed_A, seed_B, seed_idx, problem_id, {"law": "concentrated"})
    return pp.as_dtype(dtype)


def make_target(m: int, p: int, seed: int = 3) -> np.ndarray:
    """A fixed N(0,1) target matrix T (m x p) for the loss ||Yhat - T||_F^2."""
    return _rng(seed, 0xA5).standard_normal(size=(m, p))


def batched_shapes(count: int = 64, seed: int = 7):
    """Shapes of the batched workload: m, p log-uniform on [32, 512], n log-uniform on
    [4096, 262144], number of levels L+1 uniform on {3..9}.  Returns a list of
    (m, n, p, L) tuples."""
    rng = _rng(seed, 0xB7)
    out = []
    for _ in range(count):
        m = int(math.floor(math.exp(rng.uniform(math.log(32), math.log(512)))))
        p = int(math.floor(math.exp(rng.uniform(math.log(32), math.log(512)))))
        n = int(math.floor(math.exp(rng.uniform(math.log(4096), math.log(262144)))))
        levels = int(rng.integers(3, 10))  # L + 1 in 3..9
        out.append((m, n, p, levels - 1))
    return out
