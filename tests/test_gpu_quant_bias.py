"""Bias of the reduced-precision estimators, by common random numbers.

Rounding the generated entries (bf16, or E4M3 with block scales) makes each sample D_q differ
from the FP32 sample D_32 of the same sample id (same indices, same Z up to the last bits of the
normals).  Levels l >= 1 stay unbiased in every precision: the fine and coarse estimates of a
sample are sketches of one and the same rounded realisation, and the slots of a sample (and of an
E4M3 scale block) are exchangeable, so E[D_l,q] = 0 exactly.  What rounding can bias is level 0:
E[D_0,q] - E[D_0,32] = E[Yhat_q] - E[Yhat_32].  Evaluating level 0 of a BF16 (E4M3) plan and of
an FP32 plan on the same sample ids, the difference of their level means has the quantisation
noise alone as its spread (sum over entries of Var(D_0,q - D_0,32) ~ 7.5e2 for BF16, 1.9e5 for
E4M3 per sample on this workload), so with N samples it measures the bias to about
sqrt(that / N).  The bar: the bias is at most 0.1 eps at relative RMSE 1e-3
(eps = 1e-3 ||M M'||_F ~ 0.69), with N chosen so that the noise alone is about 0.02 eps (BF16,
4e6 samples) and 0.03 eps (E4M3, 4e8 samples).
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


@pytest.mark.parametrize("precision,N", [("bf16", 4_000_000), ("fp8", 400_000_000)])
def test_quantisation_bias_below_a_tenth_of_eps(precision, N):
    pp = make_params(64, 1024, 64, seed_A=0, seed_B=1, dtype=np.float32)
    eps = 1e-3 * float(np.linalg.norm(pp.exact_mean()))
    dev = torch.device("cuda:0")
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    means = {}
    for prec in (precision, "fp32"):
        spec = binding.ProblemSpec(*ts, seed_A=40, seed_B=41, seed_idx=42, problem_id=0)
        with binding.Plan([spec], c0=16, L=0, precision=prec) as plan:
            plan.level_stats(0, 0, 0, N)
            n_got, mean, _ = plan.get_level_stats(0, 0)
            assert n_got == N
            means[prec] = mean.cpu().numpy()
    diff = float(np.linalg.norm(means[precision] - means["fp32"]))
    print(f"{precision}: ||mean_q - mean_fp32||_F over {N} level-0 samples = {diff:.4e} = {diff / eps:.4f} eps")
    assert diff <= 0.1 * eps
