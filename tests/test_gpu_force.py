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
