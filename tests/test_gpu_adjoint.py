"""Parity of mlmc_backward (the reparameterised adjoint) with the FP64 oracle, through the C ABI.

Bars:
  * FP64 parameters and arithmetic: every entry within 1e-11 of the largest oracle entry of
    its matrix (the two sides sum the same FP64 products in different orders);
  * FP32: each contraction u = G b (or G^T a) runs over k_in <= 300 FP32 products, so its
    error is at most (k_in + 2) 2^-24 sum |G| |b| plus 2^-21 from the FP32 entries; checked as
    2e-5 of the largest entry per element and 2e-6 in Frobenius norm;
  * BF16 (straight-through): against the oracle's bfloat16 emulation the operands agree
    except where an FP32 and an FP64 value round to different bfloat16 neighbours, so a
    Frobenius bar of 1e-3 holds; against the unrounded oracle the operand rounding (2^-8)
    shows, 2^-6 in Frobenius norm.  Contracted dimensions up to 256 run on the tensor cores with
    G split into bfloat16 hi and lo parts (2^-16 relative per product, FP32 accumulation), the
    same bars; BF16_CASES mix both kernels (k_in = 300 keeps the CUDA-core one).
The gradient is also checked against central differences of the GPU estimator itself: the
estimate is a polynomial of degree two in the parameters (bilinear in A and B), so the
central difference is exact up to rounding.
"""
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


def _tensors(pp, dtype):
    return [torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]


def _plan(pp, c0, L, precision, dtype, **kw):
    spec = binding.ProblemSpec(*_tensors(pp, dtype), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                               problem_id=pp.problem_id)
    return binding.Plan([spec], c0=c0, L=L, ratio=2, precision=precision, **kw)


def _orc(pp):
    return oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                          problem_id=pp.problem_id)


def _run(pp, c0, L, Nl, G, precision, dtype, **kw):
    with _plan(pp, c0, L, precision, dtype, **kw) as plan:
        for l, N in enumerate(Nl):
            plan.level_stats(0, l, 0, N)
        ((dM, dS, dMp, dSp),) = plan.backward([torch.from_numpy(G).to(DEV)])
        torch.cuda.synchronize()
        return [t.double().cpu().numpy() for t in (dM, dS, dMp, dSp)]


def _gauss(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


ADJ_CASES = [
    # m, n, p, c0, L, N_l
    (32, 512, 32, 16, 3, [64, 64, 64, 64]),        # finite-difference shape
    (37, 1000, 53, 16, 3, [40, 17, 9, 3]),          # ragged: partial output blocks, odd counts
    (200, 3000, 300, 8, 2, [20, 10, 5]),            # several output blocks on both sides
    (5, 64, 3, 1, 4, [7, 0, 5, 2, 1]),              # c0 = 1, an empty level, tiny n (dense segments)
]


@pytest.mark.parametrize("m,n,p,c0,L,Nl", ADJ_CASES)
def test_backward_fp64_matches_oracle(m, n, p, c0, L, Nl):
    pp = make_params(m, n, p, seed_A=3, seed_B=4, seed_idx=5, problem_id=2)
    G = _gauss((m, p), 11)
    got = _run(pp, c0, L, Nl, G, "fp64", torch.float64)
    ref = oracle.adjoint(_orc(pp), oracle.Levels(c0, 2, L), Nl, G)
    for name, a, b in zip(("dM", "dS", "dMp", "dSp"), got, ref):
        scale = np.abs(b).max()
        assert scale > 0
        assert np.all(np.abs(a - b) <= 1e-11 * scale), (name, np.abs(a - b).max() / scale)


@pytest.mark.parametrize("m,n,p,c0,L,Nl", ADJ_CASES[:3])
def test_backward_fp32_matches_oracle(m, n, p, c0, L, Nl):
    pp = make_params(m, n, p, seed_A=6, seed_B=7, seed_idx=8, problem_id=0, dtype=np.float32)
    G = _gauss((m, p), 12)
    got = _run(pp, c0, L, Nl, G, "fp32", torch.float32)
    ref = oracle.adjoint(_orc(pp), oracle.Levels(c0, 2, L), Nl, G)
    for name, a, b in zip(("dM", "dS", "dMp", "dSp"), got, ref):
        scale = np.abs(b).max()
        assert np.all(np.abs(a - b) <= 2e-5 * scale), (name, np.abs(a - b).max() / scale)
        assert np.linalg.norm(a - b) <= 2e-6 * np.linalg.norm(b), (name, np.linalg.norm(a - b) / np.linalg.norm(b))


BF16_CASES = ADJ_CASES + [
    (256, 4000, 129, 16, 3, [64, 33, 16, 9]),      # two 128-output blocks on one side, ragged other
    (129, 2000, 256, 32, 2, [70, 65, 1]),           # k_in = 256 and 129, records not a multiple of 64
]


@pytest.mark.parametrize("m,n,p,c0,L,Nl", BF16_CASES)
def test_backward_bf16_straight_through(m, n, p, c0, L, Nl):
    pp = make_params(m, n, p, seed_A=1, seed_B=2, seed_idx=3, problem_id=4, dtype=np.float32)
    G = _gauss((m, p), 13)
    got = _run(pp, c0, L, Nl, G, "bf16", torch.float32)
    orc, lv = _orc(pp), oracle.Levels(c0, 2, L)
    emu = oracle.adjoint(orc, lv, Nl, G, quant=oracle.QUANT_BF16)
    plain = oracle.adjoint(orc, lv, Nl, G)
    for name, a, b, c in zip(("dM", "dS", "dMp", "dSp"), got, emu, plain):
        e_emu = np.linalg.norm(a - b) / np.linalg.norm(b)
        e_plain = np.linalg.norm(a - c) / np.linalg.norm(c)
        assert e_emu <= 1e-3, (name, e_emu)
        assert e_plain <= 2.0**-6, (name, e_plain)
        assert e_emu < 0.5 * e_plain, (name, e_emu, e_plain)   # the rounding is what is modelled


def test_backward_matches_central_differences_on_gpu():
    """<G, Yhat> along a random direction of all four parameters, FP64, 32x512x32, c_l = 16 2^l."""
    m, n, p, c0, L, Nl = 32, 512, 32, 16, 3, [64, 64, 64, 64]
    pp = make_params(m, n, p, seed_A=0, seed_B=1)
    G = torch.from_numpy(_gauss((m, p), 14)).to(DEV)
    rng = np.random.default_rng(15)
    base = _tensors(pp, torch.float64)
    dirs = [torch.from_numpy(rng.standard_normal(t.shape)).to(DEV) for t in base]

    def f(params):
        spec = binding.ProblemSpec(*params)
        with binding.Plan([spec], c0=c0, L=L, precision="fp64") as plan:
            for l, N in enumerate(Nl):
                plan.level_stats(0, l, 0, N)
            (Y,) = plan.telescoping_sum()
            return float((G * Y).sum())

    with binding.Plan([binding.ProblemSpec(*base)], c0=c0, L=L, precision="fp64") as plan:
        for l, N in enumerate(Nl):
            plan.level_stats(0, l, 0, N)
        (grads,) = plan.backward([G])
        directional = sum(float((g * d).sum()) for g, d in zip(grads, dirs))
    h = 1e-3
    fd = (f([t + h * d for t, d in zip(base, dirs)]) - f([t - h * d for t, d in zip(base, dirs)])) / (2 * h)
    assert abs(fd - directional) <= 1e-8 * max(abs(fd), 1.0), (fd, directional)


def test_backward_batches_agree():
    """Small replay batches (2^8 records) give the one-batch gradient up to FP64 rounding."""
    m, n, p, c0, L, Nl = 48, 700, 40, 16, 3, [50, 30, 20, 10]
    pp = make_params(m, n, p, seed_A=9, seed_B=10, seed_idx=11, problem_id=1)
    G = _gauss((m, p), 16)
    one = _run(pp, c0, L, Nl, G, "fp64", torch.float64)
    many = _run(pp, c0, L, Nl, G, "fp64", torch.float64, adjoint_batch_log2=8)
    for a, b in zip(one, many):
        assert np.all(np.abs(a - b) <= 1e-12 * np.abs(a).max())


def test_backward_after_estimate_and_state_rules():
    pp = make_params(32, 256, 24, seed_A=2, seed_B=3)
    G = torch.from_numpy(_gauss((32, 24), 17)).to(DEV)
    with _plan(pp, 8, 2, "fp64", torch.float64, pilot_n=16) as plan:
        eps = 0.2 * np.linalg.norm(pp.exact_mean())
        _, (rep,) = plan.estimate([eps])
        ((dM, dS, dMp, dSp),) = plan.backward([G])
        ref = oracle.adjoint(_orc(pp), oracle.Levels(8, 2, 2), rep["N"][:3], G.cpu().numpy())
        assert np.all(np.abs(dM.cpu().numpy() - ref[0]) <= 1e-11 * np.abs(ref[0]).max())
        assert np.all(np.abs(dSp.cpu().numpy() - ref[3]) <= 1e-11 * np.abs(ref[3]).max())
    with _plan(pp, 8, 2, "fp64", torch.float64) as plan:
        plan.level_stats(0, 1, 5, 10)        # ids 5..14: not a prefix, the replay is undefined
        with pytest.raises(binding.MLMCError) as e:
            plan.backward([G])
        assert e.value.status == 7


def test_autograd_function():
    from paper_1904_00429_gb300.autograd import mlmc_matmul
    m, n, p, c0, L, Nl = 32, 512, 32, 16, 3, [64, 64, 64, 64]
    pp = make_params(m, n, p, seed_A=0, seed_B=1, dtype=np.float32)
    params = [t.requires_grad_() for t in _tensors(pp, torch.float32)]
    T = torch.from_numpy(_gauss((m, p), 18)).to(DEV)
    Y = mlmc_matmul(*params, c0=c0, L=L, Nl=Nl, precision="fp32")
    loss = ((Y - T) ** 2).sum()
    loss.backward()
    G = (2 * (Y - T)).detach().cpu().numpy()
    ref = oracle.adjoint(_orc(pp), oracle.Levels(c0, 2, L), Nl, G)
    for t, b in zip(params, ref):
        a = t.grad.double().cpu().numpy()
        assert t.grad.dtype == torch.float32
        assert np.linalg.norm(a - b) <= 2e-6 * np.linalg.norm(b)
