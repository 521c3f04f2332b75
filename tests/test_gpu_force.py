"""GPU link gradient and projected force of L = Re<eta, D^-1 b> against the
FP64 oracle (same x and lambda fed to both), and the GPU gradient chain
(solve, adjoint solve, force) against the oracle's chain."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import BC, KAPPA, gauge, lib, max_err, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 4, 10)])
def test_force_kernel(L):
    bpp = lib()
    g, U = gauge(L)
    x = synth.gaussian_spinor(L, seed=2)
    lam = synth.gaussian_spinor(L, seed=3)
    G_ref = oracle.link_gradient(x, lam, KAPPA, L, BC)
    G = to_np(bpp.force(g, to_dev(x), to_dev(lam), KAPPA, project=False))
    assert rel_err(G, G_ref) <= 1e-13 and max_err(G, G_ref) <= 1e-13
    P_ref = oracle.projected_force(U, G_ref)
    P = to_np(bpp.force(g, to_dev(x), to_dev(lam), KAPPA, project=True))
    assert rel_err(P, P_ref) <= 1e-13


def test_gradient_chain_vs_oracle():
    bpp = lib()
    L = (4, 4, 4, 8)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2)
    eta = synth.gaussian_spinor(L, seed=3)
    x, _ = bpp.solve(g, to_dev(b), KAPPA, 0.0, 1e-12, bpp.solve_opts(inner_prec=0))
    lam, _ = bpp.solve(g, to_dev(eta), KAPPA, 0.0, 1e-12, bpp.solve_opts(inner_prec=0, dagger=True))
    G = to_np(bpp.force(g, x, lam, KAPPA))
    xr = oracle.solve(U, b, KAPPA, L, BC, tol=1e-13)
    lr = oracle.solve(U, eta, KAPPA, L, BC, tol=1e-13, dagger=True)
    G_ref = oracle.link_gradient(xr, lr, KAPPA, L, BC)
    assert rel_err(to_np(lam), lr) <= 1e-9
    assert rel_err(G, G_ref) <= 1e-8


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 4, 10), (2, 4, 2, 6)])
def test_clover_force_kernel(L):
    """Hopping plus clover-term link gradient (c_SW = 1) and its su(3)
    projection against the oracle's (pinned by finite differences), on the
    same x and lambda; L_mu = 2 puts both plaquettes of a plane through the
    same sites."""
    bpp = lib()
    g, U = gauge(L)
    x = synth.gaussian_spinor(L, seed=2)
    lam = synth.gaussian_spinor(L, seed=3)
    G_ref = oracle.link_gradient(x, lam, KAPPA, L, BC, U=U, csw=1.0)
    G = to_np(bpp.force(g, to_dev(x), to_dev(lam), KAPPA, csw=1.0))
    assert rel_err(G, G_ref) <= 1e-13 and max_err(G, G_ref) <= 1e-13
    P_ref = oracle.projected_force(U, G_ref)
    P = to_np(bpp.force(g, to_dev(x), to_dev(lam), KAPPA, project=True, csw=1.0))
    assert rel_err(P, P_ref) <= 1e-13 and max_err(P, P_ref) <= 1e-13


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_force_sums_right_hand_sides(csw):
    """nrhs = 3 in one call equals the sum of the three single-RHS oracle
    gradients."""
    bpp = lib()
    L = (4, 4, 4, 6)
    g, U = gauge(L)
    x = synth.gaussian_spinor(L, seed=4, nrhs=3)
    lam = synth.gaussian_spinor(L, seed=5, nrhs=3)
    G_ref = sum(oracle.link_gradient(x[r], lam[r], KAPPA, L, BC, U=U, csw=csw) for r in range(3))
    G = to_np(bpp.force(g, to_dev(x), to_dev(lam), KAPPA, csw=csw))
    assert rel_err(G, G_ref) <= 1e-13 and max_err(G, G_ref) <= 1e-13


def test_clover_gradient_chain_vs_oracle():
    """The GPU chain (FP64 solve, adjoint solve, force with the clover term)
    against the oracle's chain with the explicit 12x12 clover field."""
    bpp = lib()
    L = (4, 4, 4, 8)
    csw = 1.0
    g, U = gauge(L)
    g.clover_build(KAPPA, csw)
    F = oracle.clover_field(U, KAPPA, csw, L)
    b = synth.gaussian_spinor(L, seed=2)
    eta = synth.gaussian_spinor(L, seed=3)
    x, _ = bpp.solve(g, to_dev(b), KAPPA, csw, 1e-12, bpp.solve_opts(inner_prec=0))
    lam, _ = bpp.solve(g, to_dev(eta), KAPPA, csw, 1e-12, bpp.solve_opts(inner_prec=0, dagger=True))
    G = to_np(bpp.force(g, x, lam, KAPPA, csw=csw))
    xr = oracle.solve(U, b, KAPPA, L, BC, F=F, tol=1e-13)
    lr = oracle.solve(U, eta, KAPPA, L, BC, F=F, tol=1e-13, dagger=True)
    G_ref = oracle.link_gradient(xr, lr, KAPPA, L, BC, U=U, csw=csw)
    assert rel_err(G, G_ref) <= 1e-8
