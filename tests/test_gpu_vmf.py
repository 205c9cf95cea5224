"""Smooth-kernel (vMF) form: the CUDA forward and hand-written adjoint against
the FP64 autograd reference (oracle/vmf_ref.py), plus the autograd.Function.

Tolerances: x_T within 1e-5 (FP32 weights and sums); gradients within 1e-4
relative L2 (FP32 recomputation of every weight in the reverse sweep). The
BF16 form (forward steps and adjoint passes on the tensor cores) has its own
bar for x_T, derived below, and the same 1e-4 bar for gradients."""
import numpy as np
import pytest
import torch

import synth
from oracle import vmf_ref

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = a.detach().double().cpu(); b = b.detach().double().cpu()
    return ((a - b).norm() / b.norm()).item()


def _problem(N, M, seed=0, K=16):
    prob = synth.vmf_problem_c5(seed=seed, N=N, M=M, K=K)
    return (torch.from_numpy(prob["P"]), torch.from_numpy(prob["X0"]), torch.from_numpy(prob["target"]))


@pytest.mark.parametrize("N,M,T", [(4096, 64, 10), (3000, 37, 3), (1000, 300, 1)])
def test_vmf_forward_matches_fp64(ms_lib, N, M, T):
    P, X0, _ = _problem(N, M)
    XT = ms_lib.ms_vmf_forward(P.cuda(), X0.cuda(), 20.0, T)
    ref = vmf_ref.vmf_forward(P.double(), X0.double(), 20.0, T)
    assert (XT.cpu().double() - ref).abs().max().item() <= 1e-5
    assert torch.allclose(XT.norm(dim=1).cpu().double(), torch.ones(M, dtype=torch.float64), rtol=0, atol=1e-6)


@pytest.mark.parametrize("N,M,T", [(4096, 64, 10), (3000, 37, 3)])
def test_vmf_adjoint_matches_fp64_vjp(ms_lib, N, M, T):
    P, X0, _ = _problem(N, M, seed=1)
    G = torch.randn(M, 16, generator=torch.Generator().manual_seed(3))
    dP, dX0 = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, T, G.cuda())
    _, rP, rX = vmf_ref.vmf_vjp(P.double(), X0.double(), 20.0, T, G.double())
    assert rel(dP, rP) <= 1e-4, rel(dP, rP)
    assert rel(dX0, rX) <= 1e-4, rel(dX0, rX)


def test_vmf_zero_steps_is_identity(ms_lib):
    P, X0, _ = _problem(512, 32, seed=2)
    XT = ms_lib.ms_vmf_forward(P.cuda(), X0.cuda(), 20.0, 0)
    assert torch.equal(XT.cpu(), X0)
    G = torch.ones(32, 16)
    dP, dX0 = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 0, G.cuda())
    assert torch.equal(dX0.cpu(), G) and dP.abs().max().item() == 0.0


def test_autograd_function_loss_gradients(ms_lib):
    from paper_2007_14283_gb300.autograd import VMFMeanShift
    P, X0, target = _problem(8192, 96, seed=4)
    Pg = P.cuda().requires_grad_(True)
    Xg = X0.cuda().requires_grad_(True)
    XT = VMFMeanShift.apply(Pg, Xg, 20.0, 10)
    loss = ((XT - target.cuda()) ** 2).sum()
    loss.backward()
    rloss, rP, rX = vmf_ref.vmf_loss_and_grads(P.double(), X0.double(), target.double(), 20.0, 10)
    assert abs(loss.item() - rloss.item()) <= 1e-4 * abs(rloss.item())
    assert rel(Pg.grad, rP) <= 1e-4 and rel(Xg.grad, rX) <= 1e-4


def test_vmf_c5_full_config_matches_fp64(ms_lib):
    """The differentiable configuration at its full size: N = 65536 pixels,
    M = 1024 seeds, d = 16, kappa = 20, T = 10. Seeds move independently, so the
    FP64 reference gradient is taken 128 seeds at a time (its autograd graph
    for all 1024 at once would hold about 10 GB) and summed over pixels."""
    P, X0, target = _problem(65536, 1024, seed=0, K=32)
    Pd, Xd = P.cuda(), X0.cuda()
    XT = ms_lib.ms_vmf_forward(Pd, Xd, 20.0, 10)
    G = 2 * (XT - target.cuda())
    dP, dX0 = ms_lib.ms_vmf_backward(Pd, Xd, 20.0, 10, G)
    rP = torch.zeros(P.shape, dtype=torch.float64)
    rX = torch.zeros(X0.shape, dtype=torch.float64)
    rloss = 0.0
    for a in range(0, 1024, 128):
        l, gP, gX = vmf_ref.vmf_loss_and_grads(P.double(), X0[a:a + 128].double(), target[a:a + 128].double(),
                                                20.0, 10)
        rloss += l.item()
        rP += gP
        rX[a:a + 128] = gX
    loss = ((XT - target.cuda()) ** 2).sum().item()
    assert abs(loss - rloss) <= 1e-4 * abs(rloss)
    assert rel(dP, rP) <= 1e-4, rel(dP, rP)
    assert rel(dX0, rX) <= 1e-4, rel(dX0, rX)


def test_vmf_deterministic(ms_lib):
    P, X0, _ = _problem(4096, 64, seed=5)
    G = torch.randn(64, 16, generator=torch.Generator().manual_seed(1)).cuda()
    a = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 5, G)
    b = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 5, G)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


# ---------------------------------------------------------------- BF16 form
# Forward steps on the tensor cores (ms_vmf_forward with MS_BF16). The
# exponent kappa log2(e) x.p comes from six BF16 products of three-term
# splits (terms below 2^-24 |x||p| left out) accumulated in FP32, so its error
# is a few FP32 ulps of |kappa log2(e) x.p| <= 29 (about 2^-19 each); the
# weight is split into two BF16 terms (relative error <= 2^-16), the low term
# against two pixel terms. Per-weight relative errors of a few 1e-6 average
# over the window; the bar below is 5e-6 on every component of x_T (measured:
# at most 1.8e-6, against 1.2e-7 for the FP32 form). The adjoint passes run on
# the tensor cores too: both scores of a pair (kappa log2(e) x.p and gy.p) from
# six products of three-term splits, the weight and kappa w (gy.p) as two BF16
# terms each against three (high term) or two (low term) data terms. Their
# per-term relative errors (<= 2^-16) average over each sum like the
# forward's; gradients keep the 1e-4 relative bar.
BF16_TOL = 5e-6


@pytest.mark.parametrize("N,M,T", [(4096, 64, 10), (3000, 37, 3), (1000, 300, 1), (129, 129, 2)])
def test_vmf_bf16_forward_matches_fp64(ms_lib, N, M, T):
    P, X0, _ = _problem(N, M)
    XT = ms_lib.ms_vmf_forward(P.cuda(), X0.cuda(), 20.0, T, precision=ms_lib.MS_BF16)
    ref = vmf_ref.vmf_forward(P.double(), X0.double(), 20.0, T)
    assert (XT.cpu().double() - ref).abs().max().item() <= BF16_TOL
    assert torch.allclose(XT.norm(dim=1).cpu().double(), torch.ones(M, dtype=torch.float64), rtol=0, atol=1e-6)


def test_vmf_bf16_c5_full_config(ms_lib):
    """N = 65536, M = 1024, T = 10: every seed's x_T against the FP64 reference,
    and the loss gradient through the autograd.Function against the FP64
    reference gradient for 128 of the seeds."""
    from paper_2007_14283_gb300.autograd import vmf_mean_shift
    P, X0, target = _problem(65536, 1024, seed=0, K=32)
    XT = ms_lib.ms_vmf_forward(P.cuda(), X0.cuda(), 20.0, 10, precision=ms_lib.MS_BF16)
    ref = vmf_ref.vmf_forward(P.double(), X0.double(), 20.0, 10)
    assert (XT.cpu().double() - ref).abs().max().item() <= BF16_TOL
    Pg = P.cuda().requires_grad_(True)
    Xg = X0[:128].cuda().requires_grad_(True)
    loss = ((vmf_mean_shift(Pg, Xg, 20.0, 10, precision=ms_lib.MS_BF16) - target[:128].cuda()) ** 2).sum()
    loss.backward()
    rloss, rP, rX = vmf_ref.vmf_loss_and_grads(P.double(), X0[:128].double(), target[:128].double(), 20.0, 10)
    assert abs(loss.item() - rloss.item()) <= 1e-4 * abs(rloss.item())
    assert rel(Pg.grad, rP) <= 1e-4 and rel(Xg.grad, rX) <= 1e-4


def test_vmf_bf16_adjoint_matches_fp64_vjp(ms_lib):
    P, X0, _ = _problem(4096, 64, seed=1)
    G = torch.randn(64, 16, generator=torch.Generator().manual_seed(3))
    dP, dX0 = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 10, G.cuda(), precision=ms_lib.MS_BF16)
    _, rP, rX = vmf_ref.vmf_vjp(P.double(), X0.double(), 20.0, 10, G.double())
    assert rel(dP, rP) <= 1e-4, rel(dP, rP)
    assert rel(dX0, rX) <= 1e-4, rel(dX0, rX)


@pytest.mark.parametrize("N,M,T,kappa", [(3000, 37, 3, 20.0), (1000, 300, 1, 20.0), (129, 129, 2, 20.0),
                                          (65, 1, 2, 20.0), (300, 257, 2, 50.0), (2000, 100, 2, 0.0)])
def test_vmf_bf16_adjoint_ragged_shapes(ms_lib, N, M, T, kappa):
    """Tensor-core adjoint on sizes that leave partial 64-column sub-tiles and
    128-row tiles on both passes (pixels as rows, seeds as rows), one seed,
    a single 64-pixel sub-tile, and kappa = 0 (uniform weights: the scaled seed
    operand is zero and pass B's ds term must still vanish)."""
    P, X0, _ = _problem(N, M, seed=7)
    G = torch.randn(M, 16, generator=torch.Generator().manual_seed(11))
    dP, dX0 = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), kappa, T, G.cuda(), precision=ms_lib.MS_BF16)
    _, rP, rX = vmf_ref.vmf_vjp(P.double(), X0.double(), kappa, T, G.double())
    assert rel(dP, rP) <= 1e-4, rel(dP, rP)
    if kappa == 0.0:  # uniform weights: x_T does not depend on x_0 at all
        assert rX.abs().max().item() == 0.0 and dX0.abs().max().item() == 0.0
    else:
        assert rel(dX0, rX) <= 1e-4, rel(dX0, rX)


def test_vmf_bf16_adjoint_close_to_fp32_adjoint(ms_lib):
    """The tensor-core adjoint against the FP32 one on the same problem, row by
    row: every pixel's and seed's gradient within 1e-4 of the FP32 form's,
    relative to the largest row norm."""
    P, X0, _ = _problem(8192, 256, seed=9)
    G = torch.randn(256, 16, generator=torch.Generator().manual_seed(12))
    a = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 4, G.cuda(), precision=ms_lib.MS_BF16)
    b = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 4, G.cuda())
    for x, y in zip(a, b):
        scale = y.norm(dim=1).max().item()
        assert (x - y).norm(dim=1).max().item() <= 1e-4 * scale


def test_vmf_bf16_deterministic_and_zero_steps(ms_lib):
    P, X0, _ = _problem(4096, 200, seed=5)
    a = ms_lib.ms_vmf_forward(P.cuda(), X0.cuda(), 20.0, 4, precision=ms_lib.MS_BF16)
    b = ms_lib.ms_vmf_forward(P.cuda(), X0.cuda(), 20.0, 4, precision=ms_lib.MS_BF16)
    assert torch.equal(a, b)
    x0 = ms_lib.ms_vmf_forward(P.cuda(), X0.cuda(), 20.0, 0, precision=ms_lib.MS_BF16)
    assert torch.equal(x0.cpu(), X0)
    G = torch.randn(200, 16, generator=torch.Generator().manual_seed(4)).cuda()
    ga = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 3, G, precision=ms_lib.MS_BF16)
    gb = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 3, G, precision=ms_lib.MS_BF16)
    assert torch.equal(ga[0], gb[0]) and torch.equal(ga[1], gb[1])
    g0 = ms_lib.ms_vmf_backward(P.cuda(), X0.cuda(), 20.0, 0, G, precision=ms_lib.MS_BF16)
    assert torch.equal(g0[1], G) and not g0[0].abs().max().item()


def test_vmf_bf16_unknown_precision_rejected(ms_lib):
    P, X0, _ = _problem(256, 8, seed=6)
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_vmf_forward(P.cuda(), X0.cuda(), 20.0, 1, precision=7)
    assert e.value.status == ms_lib.MS_ERR_INVALID_ARG
