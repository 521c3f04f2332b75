"""Differentiation of L = Re<eta, D^{-1} b>: gradients with respect to b (adjoint
solve) and the links (fermion force) through torch.autograd, checked against
central finite differences on 4^4 and against the FP64 oracle gradient on the
16^3x32 workload (kappa = 0.12, eta and b complex Gaussian, seeds 3 and 2)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, KAPPA, dev, lib, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu


def _loss(U, b, eta, L, tol=1e-13, inner=0):
    from paper_2111_04457_b300.autograd import solve_fn
    x = solve_fn(U, b, L, KAPPA, tol=tol, inner_prec=inner)
    return torch.vdot(eta.reshape(-1), x.reshape(-1)).real


def test_autograd_fd_4x4():
    L = (4, 4, 4, 4)
    U0 = synth.random_links(L)
    b0 = synth.gaussian_spinor(L, seed=2)
    eta = to_dev(synth.gaussian_spinor(L, seed=3))
    U = to_dev(U0).requires_grad_(True)
    b = to_dev(b0).requires_grad_(True)
    loss = _loss(U, b, eta, L)
    loss.backward()
    gU, gb = U.grad.clone(), b.grad.clone()
    rng = np.random.default_rng(7)
    h = 1e-4
    with torch.no_grad():
        # b: one random full-lattice direction (L is linear in b)
        d = to_dev(rng.normal(size=b0.shape) + 1j * rng.normal(size=b0.shape))
        fd = (_loss(U, b + h * d, eta, L) - _loss(U, b - h * d, eta, L)) / (2 * h)
        an = torch.vdot(gb.reshape(-1), d.reshape(-1)).real
        assert abs(float(fd - an)) <= 1e-6 * abs(float(an))
        # U: unconstrained random complex direction
        E = to_dev(rng.normal(size=U0.shape) + 1j * rng.normal(size=U0.shape))
        fd = (_loss(U + h * E, b, eta, L) - _loss(U - h * E, b, eta, L)) / (2 * h)
        an = torch.vdot(gU.reshape(-1), E.reshape(-1)).real
        assert abs(float(fd - an)) <= 1e-6 * abs(float(an))
        # su(3) directions on 64 random links: dL/deps = tr(T P)
        bpp = lib()
        g = bpp.Gauge(U.detach(), L)
        x, _ = bpp.solve(g, b.detach(), KAPPA, 0.0, 1e-12, bpp.solve_opts(inner_prec=0))
        lam, _ = bpp.solve(g, eta, KAPPA, 0.0, 1e-12, bpp.solve_opts(inner_prec=0, dagger=True))
        P = to_np(bpp.force(g, x, lam, KAPPA, project=True))
        V = oracle.volume(L)
        from scipy.linalg import expm
        for _ in range(64):
            mu, s = rng.integers(0, 4), rng.integers(0, V)
            A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
            T = 0.5 * (A + A.conj().T)
            T -= np.trace(T) / 3 * np.eye(3)
            Up, Um = U0.copy(), U0.copy()
            Up[mu, s] = expm(1j * h * T) @ U0[mu, s]
            Um[mu, s] = expm(-1j * h * T) @ U0[mu, s]
            fd = (_loss(to_dev(Up), b, eta, L) - _loss(to_dev(Um), b, eta, L)) / (2 * h)
            an = np.trace(T @ P[mu, s]).real
            assert abs(float(fd) - an) <= 1e-6 * max(abs(an), 1e-2)


def test_gradient_16x32_vs_oracle():
    """The 16^3x32 FP64 differentiation workload against the oracle gradient."""
    bpp = lib()
    L = (16, 16, 16, 32)
    U0 = synth.random_links(L)
    b0 = synth.gaussian_spinor(L, seed=2)
    eta0 = synth.gaussian_spinor(L, seed=3)
    U = to_dev(U0).requires_grad_(True)
    b = to_dev(b0).requires_grad_(True)
    loss = _loss(U, b, to_dev(eta0), L, tol=1e-12, inner=0)
    loss.backward()
    x_ref = oracle.solve(U0, b0, KAPPA, L, BC, tol=1e-13)
    lam_ref = oracle.solve(U0, eta0, KAPPA, L, BC, tol=1e-13, dagger=True)
    G_ref = oracle.link_gradient(x_ref, lam_ref, KAPPA, L, BC)
    assert rel_err(to_np(b.grad), lam_ref) <= 1e-9
    assert rel_err(to_np(U.grad), G_ref) <= 1e-8
    assert abs(float(loss) - np.vdot(eta0, x_ref).real) <= 1e-10 * abs(float(loss))


def test_clover_grad_b():
    """Clover (c_SW = 1): gradient with respect to b only, mixed precision."""
    from paper_2111_04457_b300.autograd import solve_fn
    L = (4, 4, 4, 6)
    U0 = synth.random_links(L)
    b = to_dev(synth.gaussian_spinor(L, seed=2, nrhs=2)).requires_grad_(True)
    eta = synth.gaussian_spinor(L, seed=3, nrhs=2)
    x = solve_fn(to_dev(U0), b, L, KAPPA, csw=1.0, tol=1e-10, inner_prec=2)
    torch.vdot(to_dev(eta).reshape(-1), x.reshape(-1)).real.backward()
    F = oracle.clover_field(U0, KAPPA, 1.0, L)
    for r in range(2):
        lam_ref = oracle.solve(U0, eta[r], KAPPA, L, BC, F=F, tol=1e-12, dagger=True)
        assert rel_err(to_np(b.grad[r]), lam_ref) <= 1e-8


def test_autograd_clover_fd_4x4():
    """Wilson-clover (c_SW = 1): grad_U through torch.autograd (hopping and
    clover parts of the force) against central finite differences of the loss
    in one random complex direction of all links, and in su(3) directions of
    16 random links; grad_b in one random direction."""
    bpp = lib()
    L = (4, 4, 4, 4)
    csw = 1.0
    U0 = synth.random_links(L)
    b0 = synth.gaussian_spinor(L, seed=2)
    eta = to_dev(synth.gaussian_spinor(L, seed=3))

    def loss_c(U, b):
        from paper_2111_04457_b300.autograd import solve_fn
        x = solve_fn(U, b, L, KAPPA, csw=csw, tol=1e-13, inner_prec=0)
        return torch.vdot(eta.reshape(-1), x.reshape(-1)).real

    U = to_dev(U0).requires_grad_(True)
    b = to_dev(b0).requires_grad_(True)
    loss_c(U, b).backward()
    gU, gb = U.grad.clone(), b.grad.clone()
    rng = np.random.default_rng(11)
    h = 1e-4
    with torch.no_grad():
        d = to_dev(rng.normal(size=b0.shape) + 1j * rng.normal(size=b0.shape))
        fd = (loss_c(U, b + h * d) - loss_c(U, b - h * d)) / (2 * h)
        an = torch.vdot(gb.reshape(-1), d.reshape(-1)).real
        assert abs(float(fd - an)) <= 1e-6 * abs(float(an))
        E = to_dev(rng.normal(size=U0.shape) + 1j * rng.normal(size=U0.shape))
        fd = (loss_c(U + h * E, b) - loss_c(U - h * E, b)) / (2 * h)
        an = torch.vdot(gU.reshape(-1), E.reshape(-1)).real
        assert abs(float(fd - an)) <= 1e-6 * abs(float(an))
        g = bpp.Gauge(U.detach(), L)
        g.clover_build(KAPPA, csw)
        x, _ = bpp.solve(g, b.detach(), KAPPA, csw, 1e-12, bpp.solve_opts(inner_prec=0))
        lam, _ = bpp.solve(g, eta, KAPPA, csw, 1e-12, bpp.solve_opts(inner_prec=0, dagger=True))
        P = to_np(bpp.force(g, x, lam, KAPPA, project=True, csw=csw))
        V = oracle.volume(L)
        from scipy.linalg import expm
        for _ in range(16):
            mu, s = rng.integers(0, 4), rng.integers(0, V)
            A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
            T = 0.5 * (A + A.conj().T)
            T -= np.trace(T) / 3 * np.eye(3)
            Up, Um = U0.copy(), U0.copy()
            Up[mu, s] = expm(1j * h * T) @ U0[mu, s]
            Um[mu, s] = expm(-1j * h * T) @ U0[mu, s]
            fd = (loss_c(to_dev(Up), b) - loss_c(to_dev(Um), b)) / (2 * h)
            an = np.trace(T @ P[mu, s]).real
            assert abs(float(fd) - an) <= 1e-6 * max(abs(an), 1e-2)


def test_solve_fn_refuses_a_gauge_of_another_field():
    """A prebuilt gauge handle must come from the U it is passed with (the
    gradient would otherwise be the gradient of another field's solve)."""
    bpp = lib()
    from paper_2111_04457_b300.autograd import solve_fn
    L = (4, 4, 4, 4)
    U = synth.random_links(L, seed=1)
    U2 = synth.random_links(L, seed=11)
    g = bpp.Gauge(to_dev(U), L)
    b = to_dev(synth.gaussian_spinor(L, seed=2))
    x = solve_fn(to_dev(U), b, L, KAPPA, gauge=g)          # same field: accepted
    assert x.shape == b.shape
    with pytest.raises(ValueError):
        solve_fn(to_dev(U2), b, L, KAPPA, gauge=g)
    with pytest.raises(ValueError):
        solve_fn(to_dev(U), b, L, KAPPA, csw=1.0, gauge=g)   # no clover term built
