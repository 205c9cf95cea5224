"""Pins for the FP64 smooth-kernel (vMF) reference: closed forms, the ascent
property of the fixed-point step, and central finite differences."""
import numpy as np
import pytest
import torch

from oracle import vmf_ref
import synth


def _small(seed=0, N=256, M=16, d=4, K=4):
    rng = np.random.default_rng(seed)
    means = synth.uniform_sphere(rng, K, d)
    lab = rng.integers(0, K, N)
    P = np.concatenate([synth.sample_vmf(rng, means[k], 30.0, int((lab == k).sum())) for k in range(K)])
    X0 = P[rng.choice(N, M, replace=False)]
    target = means[rng.integers(0, K, M)]
    return [torch.tensor(a, dtype=torch.float64) for a in (P, X0, target)]


def test_kappa_zero_is_one_step_to_the_global_mean():
    P, X0, _ = _small()
    s = P.sum(0)
    want = (s / s.norm()).expand_as(X0)
    for T in (1, 3):
        assert torch.allclose(vmf_ref.vmf_forward(P, X0, 0.0, T), want, rtol=0, atol=1e-15)


def test_single_pixel_maps_every_seed_onto_it():
    p = torch.tensor([[0.3, -1.2, 2.0, 0.5]], dtype=torch.float64)
    X0 = torch.nn.functional.normalize(torch.randn(5, 4, dtype=torch.float64), dim=1)
    out = vmf_ref.vmf_forward(p, X0, 20.0, 2)
    assert torch.allclose(out, (p / p.norm()).expand_as(out), rtol=0, atol=1e-15)


def test_objective_ascends_each_step():
    # f(x) = sum exp(kappa x.p) is convex, so x' = grad f / |grad f| satisfies
    # f(x') >= f(x) + grad f . (x' - x) >= f(x) on the sphere.
    P, X0, _ = _small(1)
    X = X0 / X0.norm(dim=1, keepdim=True)
    for _ in range(6):
        f0 = vmf_ref.vmf_objective(P, X, 20.0)
        X = vmf_ref.vmf_forward(P, X, 20.0, 1)
        assert (vmf_ref.vmf_objective(P, X, 20.0) >= f0 * (1 - 1e-14)).all()


def test_gradients_match_central_finite_differences():
    P, X0, target = _small(2)
    kappa, T = 20.0, 3
    loss, gP, gX = vmf_ref.vmf_loss_and_grads(P, X0, target, kappa, T)
    rng = np.random.default_rng(3)
    h = 1e-6
    for which, base, g in (("P", P, gP), ("X", X0, gX)):
        for _ in range(12):
            i = int(rng.integers(base.shape[0])); k = int(rng.integers(base.shape[1]))
            plus, minus = base.clone(), base.clone()
            plus[i, k] += h; minus[i, k] -= h
            if which == "P":
                fp = vmf_ref.vmf_loss(plus, X0, target, kappa, T); fm = vmf_ref.vmf_loss(minus, X0, target, kappa, T)
            else:
                fp = vmf_ref.vmf_loss(P, plus, target, kappa, T); fm = vmf_ref.vmf_loss(P, minus, target, kappa, T)
            fd = (fp - fm).item() / (2 * h)
            scale = max(abs(fd), g.abs().max().item() * 1e-3)
            assert abs(fd - g[i, k].item()) <= 1e-6 * scale + 1e-9, (which, i, k, fd, g[i, k].item())


def test_vjp_is_linear_in_upstream():
    P, X0, _ = _small(4)
    G1 = torch.randn_like(X0); G2 = torch.randn_like(X0)
    _, a1, b1 = vmf_ref.vmf_vjp(P, X0, 20.0, 2, G1)
    _, a2, b2 = vmf_ref.vmf_vjp(P, X0, 20.0, 2, G2)
    _, a3, b3 = vmf_ref.vmf_vjp(P, X0, 20.0, 2, 2 * G1 - G2)
    assert torch.allclose(a3, 2 * a1 - a2, rtol=0, atol=1e-10) and torch.allclose(b3, 2 * b1 - b2, rtol=0, atol=1e-10)


def test_two_pixels_hand_worked_steps():
    # p1 = e1, p2 = e2, x0 = e1, kappa = ln 3: the weights are 3^(x.p), so
    # step 1 has w = (3, 1) and x1 = (3, 1) / sqrt(10); step 2 has
    # w = (3^(3/sqrt10), 3^(1/sqrt10)), i.e. x2 = (1, r) / sqrt(1 + r^2) with
    # r = 3^(-2/sqrt10)
    P = torch.tensor([[1.0, 0.0], [0.0, 1.0]], dtype=torch.float64)
    X0 = torch.tensor([[1.0, 0.0]], dtype=torch.float64)
    k = float(np.log(3.0))
    x1 = vmf_ref.vmf_forward(P, X0, k, 1)
    assert torch.allclose(x1, torch.tensor([[3.0, 1.0]], dtype=torch.float64) / np.sqrt(10.0), rtol=0, atol=1e-15)
    r = 3.0 ** (-2.0 / np.sqrt(10.0))
    x2 = vmf_ref.vmf_forward(P, X0, k, 2)
    assert torch.allclose(x2, torch.tensor([[1.0, r]], dtype=torch.float64) / np.sqrt(1.0 + r * r), rtol=0, atol=1e-15)


def test_kappa_zero_weights_pixels_by_their_length():
    # pixels are not renormalised: with kappa = 0 every weight is 1 and the
    # step lands on normalise(sum p), longer pixels pulling harder
    P = torch.tensor([[4.0, 0.0], [0.0, 1.0], [0.0, 2.0]], dtype=torch.float64)
    X0 = torch.tensor([[0.0, 1.0], [0.6, 0.8]], dtype=torch.float64)
    want = torch.tensor([[0.8, 0.6]], dtype=torch.float64).expand_as(X0)
    assert torch.allclose(vmf_ref.vmf_forward(P, X0, 0.0, 1), want, rtol=0, atol=1e-15)


def test_loss_hand_value():
    # T = 0: x_T = x_0, and the loss of e1 against e2 is |e1 - e2|^2 = 2
    P = torch.tensor([[1.0, 0.0]], dtype=torch.float64)
    X0 = torch.tensor([[1.0, 0.0], [0.0, 1.0]], dtype=torch.float64)
    target = torch.tensor([[0.0, 1.0], [0.0, 1.0]], dtype=torch.float64)
    assert vmf_ref.vmf_loss(P, X0, target, 5.0, 0).item() == 2.0


def test_vjp_matches_central_finite_differences():
    # <G, dx_T/dP> and <G, dx_T/dX0> against central differences of <G, x_T>
    P, X0, _ = _small(5)
    kappa, T = 20.0, 2
    G = torch.tensor(np.random.default_rng(6).standard_normal(tuple(X0.shape)), dtype=torch.float64)
    XT, gP, gX = vmf_ref.vmf_vjp(P, X0, kappa, T, G)
    assert torch.allclose(XT, vmf_ref.vmf_forward(P, X0, kappa, T), rtol=0, atol=0.0)
    rng = np.random.default_rng(7)
    h = 1e-6
    for which, base, g in (("P", P, gP), ("X", X0, gX)):
        assert g.shape == base.shape
        for _ in range(12):
            i = int(rng.integers(base.shape[0])); k = int(rng.integers(base.shape[1]))
            plus, minus = base.clone(), base.clone()
            plus[i, k] += h; minus[i, k] -= h
            if which == "P":
                fp = (G * vmf_ref.vmf_forward(plus, X0, kappa, T)).sum()
                fm = (G * vmf_ref.vmf_forward(minus, X0, kappa, T)).sum()
            else:
                fp = (G * vmf_ref.vmf_forward(P, plus, kappa, T)).sum()
                fm = (G * vmf_ref.vmf_forward(P, minus, kappa, T)).sum()
            fd = (fp - fm).item() / (2 * h)
            scale = max(abs(fd), g.abs().max().item() * 1e-3)
            assert abs(fd - g[i, k].item()) <= 1e-6 * scale + 1e-9, (which, i, k, fd, g[i, k].item())
