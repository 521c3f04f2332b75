"""Pins of the FP64 oracle to mathematics that does not come from the oracle itself.

The paper (Sec. 3, Eq. 1) prints no numerical values for the operator, so the
oracle is pinned by closed forms, invariants and brute force:
  * Clifford algebra of the gamma table (chiral basis);
  * free-field (U = 1) spectrum and plane waves, p4 antiperiodic;
  * constant commuting diagonal links: a colour-dependent momentum shift;
  * gamma5-hermiticity and the adjoint identity <phi, D psi> = <D^dag phi, psi>;
  * gauge covariance of D and of the clover term;
  * dense LU on 2^4 (forward and backward neighbours coincide and add);
  * DFT inverse of the free field against the even-odd Krylov solve;
  * uniform abelian flux: eigenvalues 1 -/+ kappa c_SW sin(theta) of 1 + F.
"""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle
import synth

KAPPA = 0.12


def _matched_max_err(a, b):
    C = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(C)
    return C[r, c].max()


def _rand_spinor(L, seed):
    return synth.gaussian_spinor(L, seed=seed)


def _gauge_transform_links(U, g, L):
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    x = oracle.coords(L)
    V = oracle.volume(L)
    Ug = np.empty_like(U)
    for mu in range(4):
        y = x.copy()
        y[:, mu] = (y[:, mu] + 1) % L[mu]
        ys = y[:, 0] + L[0] * (y[:, 1] + L[1] * (y[:, 2] + L[2] * y[:, 3]))
        Ug[mu] = g @ U[mu] @ np.conj(np.swapaxes(g[ys], -1, -2))
    assert Ug.shape == (4, V, 3, 3)
    return Ug


# --------------------------------------------------------------------------- gamma
def test_clifford_algebra():
    G = oracle.GAMMA
    for m in range(4):
        assert np.allclose(G[m], G[m].conj().T)
        for n in range(4):
            assert np.allclose(G[m] @ G[n] + G[n] @ G[m], 2.0 * (m == n) * np.eye(4), atol=0)
    assert np.allclose(oracle.GAMMA5, np.diag([-1, -1, 1, 1]))
    for m in range(4):
        for n in range(m + 1, 4):
            sig = 0.5j * (G[m] @ G[n] - G[n] @ G[m])
            assert np.allclose(sig[:2, 2:], 0) and np.allclose(sig[2:, :2], 0)


# --------------------------------------------------------------------------- free field
@pytest.mark.parametrize("L,bc", [((2, 2, 2, 2), (1, 1, 1, -1)), ((2, 2, 2, 4), (1, 1, 1, -1)),
                                  ((4, 2, 2, 2), (1, 1, 1, -1)), ((2, 2, 4, 2), (1, 1, 1, 1))])
def test_free_field_spectrum(L, bc):
    M = oracle.dense_D(synth.unit_links(L), KAPPA, L, bc)
    ev = np.linalg.eigvals(M)
    assert _matched_max_err(ev, oracle.free_field_eigenvalues(L, KAPPA, bc)) < 1e-12


def test_free_field_spectrum_golden():
    """Closed-form spectrum stored in tests/golden (written by make_golden.py)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "free_field_spectrum_2x2x2x4_k0.12.txt")
    ref = np.loadtxt(path)
    ref = ref[:, 0] + 1j * ref[:, 1]
    L = (2, 2, 2, 4)
    ev = np.linalg.eigvals(oracle.dense_D(synth.unit_links(L), KAPPA, L))
    assert _matched_max_err(ev, ref) < 1e-12


def test_free_field_plane_wave(rng):
    L = (4, 4, 4, 6)
    ps = oracle.momenta(L)
    n = [rng.integers(0, L[m]) for m in range(4)]
    p = np.array([ps[m][n[m]] for m in range(4)])
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    x = oracle.coords(L)
    phase = np.exp(1j * (x @ p))
    psi = phase[:, None, None] * u[None]
    out = oracle.apply_D(synth.unit_links(L), psi, KAPPA, L)
    expect = phase[:, None, None] * (oracle.free_field_Dp(p, KAPPA) @ u)[None]
    assert np.abs(out - expect).max() < 1e-13


def test_constant_diagonal_links_shift_momentum(rng):
    L = (4, 4, 4, 4)
    phases = rng.uniform(-np.pi, np.pi, size=(4, 3))
    U = synth.constant_diagonal_links(L, phases)
    ps = oracle.momenta(L)
    p = np.array([ps[m][rng.integers(0, L[m])] for m in range(4)])
    x = oracle.coords(L)
    phase = np.exp(1j * (x @ p))
    for c in range(3):
        u = rng.normal(size=4) + 1j * rng.normal(size=4)
        psi = np.zeros((oracle.volume(L), 4, 3), dtype=np.complex128)
        psi[:, :, c] = phase[:, None] * u[None]
        out = oracle.apply_D(U, psi, KAPPA, L)
        expect = phase[:, None] * (oracle.free_field_Dp(p + phases[:, c], KAPPA) @ u)[None]
        assert np.abs(out[:, :, c] - expect).max() < 1e-13
        others = [d for d in range(3) if d != c]
        assert np.abs(out[:, :, others]).max() == 0.0


# --------------------------------------------------------------------------- adjoint
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_gamma5_hermiticity_and_adjoint(csw):
    L = (4, 4, 4, 4)
    U = synth.random_links(L)
    F = oracle.clover_field(U, KAPPA, csw, L) if csw else None
    psi, phi = _rand_spinor(L, 2), _rand_spinor(L, 3)
    Dpsi = oracle.apply_D(U, psi, KAPPA, L, F=F)
    Ddphi = oracle.apply_D(U, phi, KAPPA, L, F=F, dagger=True)
    # <phi, D psi> = <D^dag phi, psi>
    lhs, rhs = np.vdot(phi, Dpsi), np.vdot(Ddphi, psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # gamma5 D gamma5 = D^dag
    g5Dg5 = oracle.gamma5(oracle.apply_D(U, oracle.gamma5(phi), KAPPA, L, F=F))
    assert np.abs(g5Dg5 - Ddphi).max() < 1e-13


def test_schur_gamma5_hermiticity():
    L = (4, 4, 4, 4)
    U = synth.random_links(L)
    F = oracle.clover_field(U, KAPPA, 1.0, L)
    S = oracle.Schur(U, KAPPA, L, F=F)
    a = _rand_spinor(L, 2)[S.even]
    b = _rand_spinor(L, 3)[S.even]
    lhs = np.vdot(a, S.apply(b))
    rhs = np.vdot(S.apply(a, dagger=True), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert np.abs(oracle.gamma5(S.apply(oracle.gamma5(a))) - S.apply(a, dagger=True)).max() < 1e-13


# --------------------------------------------------------------------------- covariance
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_gauge_covariance(csw):
    L = (4, 4, 4, 6)
    U = synth.random_links(L)
    g = synth.random_gauge_transform(L)
    Ug = _gauge_transform_links(U, g, L)
    psi = _rand_spinor(L, 2)
    gpsi = np.einsum("vab,vsb->vsa", g, psi)
    F = oracle.clover_field(U, KAPPA, csw, L) if csw else None
    Fg = oracle.clover_field(Ug, KAPPA, csw, L) if csw else None
    lhs = oracle.apply_D(Ug, gpsi, KAPPA, L, F=Fg)
    rhs = np.einsum("vab,vsb->vsa", g, oracle.apply_D(U, psi, KAPPA, L, F=F))
    assert np.abs(lhs - rhs).max() < 1e-13


# --------------------------------------------------------------------------- clover
def test_clover_invariants():
    L = (4, 4, 4, 4)
    F = oracle.clover_field(synth.random_links(L), KAPPA, 1.0, L)
    assert np.abs(F - np.conj(np.swapaxes(F, 1, 2))).max() < 1e-15
    g5 = np.kron(oracle.GAMMA5, np.eye(3))
    assert np.abs(F @ g5 - g5 @ F).max() < 1e-15
    assert np.abs(F).max() > 1e-2
    F0 = oracle.clover_field(synth.unit_links(L), KAPPA, 1.0, L)
    assert np.abs(F0).max() == 0.0


@pytest.mark.parametrize("L,n", [((4, 4, 2, 2), 1), ((4, 6, 2, 4), 2)])
def test_abelian_flux_clover_spectrum(L, n):
    U = synth.abelian_flux_links(L, n)
    theta = 2 * np.pi * n / (L[0] * L[1])
    for s in [0, 5, oracle.volume(L) - 1]:
        Q = oracle.clover_leaf(U, L, 0, 1, s)
        assert np.abs(Q - 4 * np.exp(1j * theta) * np.eye(3)).max() < 1e-13
        for (mu, nu) in [(0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]:
            assert np.abs(oracle.clover_leaf(U, L, mu, nu, s) - 4 * np.eye(3)).max() < 1e-13
    csw = 1.0
    F = oracle.clover_field(U, KAPPA, csw, L)
    expect = np.sort(np.repeat([1 - KAPPA * csw * np.sin(theta), 1 + KAPPA * csw * np.sin(theta)], 6))
    for s in range(oracle.volume(L)):
        ev = np.sort(np.linalg.eigvalsh(np.eye(12) + F[s]))
        assert np.abs(ev - expect).max() < 1e-14


# --------------------------------------------------------------------------- solvers
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_dense_lu_2x4(csw):
    L = (2, 2, 2, 2)
    U = synth.random_links(L)
    F = oracle.clover_field(U, KAPPA, csw, L) if csw else None
    b = _rand_spinor(L, 2)
    x_lu = np.linalg.solve(oracle.dense_D(U, KAPPA, L, F=F), b.ravel()).reshape(b.shape)
    for method in ["bicgstab", "cgnr"]:
        x = oracle.solve(U, b, KAPPA, L, F=F, tol=1e-13, method=method)
        assert np.abs(x - x_lu).max() < 1e-11 * np.abs(x_lu).max()
    xd = oracle.solve(U, b, KAPPA, L, F=F, tol=1e-13, dagger=True)
    xd_lu = np.linalg.solve(oracle.dense_D(U, KAPPA, L, F=F).conj().T, b.ravel()).reshape(b.shape)
    assert np.abs(xd - xd_lu).max() < 1e-11 * np.abs(xd_lu).max()


def test_free_field_dft_inverse():
    L = (4, 4, 4, 6)
    U = synth.unit_links(L)
    b = _rand_spinor(L, 2)
    x_dft = oracle.free_field_solve_dft(b, KAPPA, L)
    x = oracle.solve(U, b, KAPPA, L, tol=1e-13)
    assert np.abs(x - x_dft).max() < 1e-10 * np.abs(x_dft).max()
    assert oracle.true_residual(U, b, x_dft, KAPPA, L) < 1e-13


def test_schur_equals_full_solve_residual():
    L = (4, 4, 4, 4)
    U = synth.random_links(L)
    F = oracle.clover_field(U, KAPPA, 1.0, L)
    b = _rand_spinor(L, 2)
    x = oracle.solve(U, b, KAPPA, L, F=F, tol=1e-12)
    assert oracle.true_residual(U, b, x, KAPPA, L, F=F) < 1e-12


def test_clover_field_sites_matches_full():
    L = (4, 4, 4, 6)
    U = synth.random_links(L)
    F = oracle.clover_field(U, KAPPA, 1.0, L)
    sites = np.array([0, 7, 100, oracle.volume(L) - 1])
    assert np.array_equal(oracle.clover_field_sites(U, KAPPA, 1.0, L, sites), F[sites])
    psi = _rand_spinor(L, 2)
    full = oracle.apply_D(U, psi, KAPPA, L, F=F)
    part = oracle.apply_D_sites_clover(U, psi, KAPPA, L, 1.0, sites)
    assert np.abs(part - full[sites]).max() < 1e-13
