"""Accuracy of the whole estimator (Alg. 2 through mlmc_estimate) over independent replicas.

For f = identity the MLMC estimate is unbiased, E[Yhat] = E[A] E[B] = M M' exactly (the entries
are independent and the sketch of each level is unbiased), so its mean squared error is its
variance, sum_l V_l / N_l, which the allocation of Remark 3.6 keeps at or below eps^2 / 2.  Each
replica draws fresh Philox keys (indices, A and B entries) for the same parameters and runs the
pilot, the allocation and the top-up; the test compares the replicas' mean ||Yhat - M M'||_F^2
with the mean of their own predicted variances (rmse_pred^2, from the run's variance estimates).

Bars: the squared error of one replica is a sum over m p correlated entries (effective degrees
of freedom in the hundreds at 64 x 64), so over 16 replicas the ratio of the two means stays
within a few per cent of 1 for an exact estimator; [0.6, 1.6] leaves room for the correlation
and catches a bias or a mis-sized allocation (a dropped level, a wrong weight or a
variance off by a factor of two all move it well outside).  The achieved RMSE must also meet the
target eps (the allocation aims at eps / sqrt(2)).  The reduced precisions take part too: their
rounding noise is part of every level's variance, so the allocation sizes for it, and their
rounding bias is far below these targets (tests/test_gpu_quant_bias.py bounds it by common
random numbers at a tenth of the 1e-3 target).
"""
import numpy as np
import pytest
import torch

from paper_1904_00429_gb300 import binding
from paper_1904_00429_gb300.inputs import make_params

pytestmark = pytest.mark.gpu

REPLICAS = 16


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("precision,rel", [("bf16", 3e-2), ("fp8", 3e-2), ("fp32", 3e-2)])
def test_rmse_over_replicas(precision, rel):
    """Precision workload shape (64 x 1024 x 64, M ~ U[-1,1], S ~ U[0.1,1], c_l = 16 2^l, L = 5)."""
    pp = make_params(64, 1024, 64, seed_A=0, seed_B=1, dtype=np.float32)
    exact = pp.exact_mean()
    eps = rel * float(np.linalg.norm(exact))
    dev = torch.device("cuda:0")
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    err2, pred2, nls = [], [], []
    for r in range(REPLICAS):
        spec = binding.ProblemSpec(*ts, seed_A=100 + r, seed_B=200 + r, seed_idx=300 + r, problem_id=0)
        with binding.Plan([spec], c0=16, L=5, ratio=2, precision=precision, pilot_n=256) as plan:
            (Y,), (rep,) = plan.estimate([eps])
            err2.append(float(np.sum((Y.cpu().numpy() - exact) ** 2)))
            pred2.append(rep["rmse_pred"] ** 2)
            nls.append(rep["N"])
    ratio = np.mean(err2) / np.mean(pred2)
    rmse = float(np.sqrt(np.mean(err2)))
    print(f"{precision}: eps {eps:.4e}, empirical RMSE {rmse:.4e} ({rmse / eps:.3f} eps), "
          f"mean predicted {np.sqrt(np.mean(pred2)):.4e}, ratio {ratio:.3f}, N_l of replica 0 {nls[0]}")
    assert 0.6 <= ratio <= 1.6, ratio
    assert rmse <= eps, (rmse, eps)
    # every replica sized its levels for the same target: the predicted RMSE is eps / sqrt(2) up
    # to the sampling error of the pilot variances
    assert max(np.sqrt(pred2)) <= 1.3 * eps / np.sqrt(2)
