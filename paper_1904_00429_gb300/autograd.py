"""``torch.autograd`` entry to the MLMC estimator with its reparameterised adjoint.

``mlmc_matmul(M, S, Mp, Sp, ...)`` returns the estimate Yhat of E[AB] for A = M + S o Z,
B = Mp + Sp o Z' (Eq. hatY) and, on ``backward``, the gradient of the loss with respect to
the four parameter matrices with the draws held fixed, computed by ``mlmc_backward`` of the
C library (the samples are replayed on the device; nothing of the forward is stored).
"""
from typing import Optional, Sequence

import torch

from . import binding


class _MLMCMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M, S, Mp, Sp, cfg):
        spec = binding.ProblemSpec(M.detach(), S.detach(), Mp.detach(), Sp.detach(), seed_A=cfg["seed_A"],
                                   seed_B=cfg["seed_B"], seed_idx=cfg["seed_idx"], problem_id=cfg["problem_id"])
        plan = binding.Plan([spec], c0=cfg["c0"], L=cfg["L"], ratio=cfg["ratio"], precision=cfg["precision"],
                            pilot_n=cfg["pilot_n"])
        if cfg["Nl"] is not None:
            for l, N in enumerate(cfg["Nl"]):
                plan.level_stats(0, l, 0, int(N))
            (Y,) = plan.telescoping_sum()
            report = None
        else:
            (Y,), (report,) = plan.estimate([cfg["eps_abs"]])
        ctx.plan = plan
        ctx.report = report
        return Y.clone()

    @staticmethod
    def backward(ctx, G):
        plan = ctx.plan
        ((dM, dS, dMp, dSp),) = plan.backward([G.contiguous()])
        plan.close()
        ctx.plan = None
        return dM, dS, dMp, dSp, None


def mlmc_matmul(M: torch.Tensor, S: torch.Tensor, Mp: torch.Tensor, Sp: torch.Tensor, *, c0: int, L: int,
                ratio: int = 2, precision: str = "fp32", eps_abs: Optional[float] = None,
                Nl: Optional[Sequence[int]] = None, pilot_n: int = 256, seed_A: int = 0, seed_B: int = 1,
                seed_idx: int = 2, problem_id: int = 0) -> torch.Tensor:
    """MLMC estimate of E[(M + S o Z)(Mp + Sp o Z')] (m x p, float64), differentiable in the parameters.

    Exactly one of ``eps_abs`` (Alg. 2: pilot, allocation, top-up) and ``Nl`` (a fixed number of
    samples per level) is given.  The parameters are 2-D row-major float32/float64 CUDA tensors;
    their gradients come back in the same dtype."""
    if (eps_abs is None) == (Nl is None):
        raise ValueError("give exactly one of eps_abs and Nl")
    if Nl is not None and len(Nl) != L + 1:
        raise ValueError("Nl needs one entry per level 0..L")
    cfg = dict(c0=c0, L=L, ratio=ratio, precision=precision, eps_abs=eps_abs, Nl=None if Nl is None else list(Nl),
               pilot_n=pilot_n, seed_A=seed_A, seed_B=seed_B, seed_idx=seed_idx, problem_id=problem_id)
    return _MLMCMatmul.apply(M, S, Mp, Sp, cfg)
