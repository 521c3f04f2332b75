"""Pins of the oracle's gradient of L = Re<eta, D^{-1} b> to central finite differences.

grad_b = D^{-dag} eta; grad_U = kappa * bc * M^dag (unconstrained); the projected
force P satisfies dL/deps = tr(T P) for U -> exp(i eps T) U.  All derived from
dL = -Re<lam, dD x> with dD read off Eq. (1); checked here on 4^4 without
reference to that derivation.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
import synth

KAPPA = 0.12
L = (4, 4, 4, 4)
TOL = 1e-13


@pytest.fixture(scope="module")
def setup():
    U = synth.random_links(L)
    b = synth.gaussian_spinor(L, seed=2)
    eta = synth.gaussian_spinor(L, seed=3)
    x = oracle.solve(U, b, KAPPA, L, tol=TOL)
    lam = oracle.solve(U, eta, KAPPA, L, tol=TOL, dagger=True)
    G = oracle.link_gradient(x, lam, KAPPA, L)
    return U, b, eta, x, lam, G


def loss(U, b, eta):
    return np.vdot(eta, oracle.solve(U, b, KAPPA, L, tol=TOL)).real


def test_grad_b_fd(setup, rng):
    U, b, eta, x, lam, G = setup
    d = rng.normal(size=b.shape) + 1j * rng.normal(size=b.shape)
    h = 1e-3
    fd = (loss(U, b + h * d, eta) - loss(U, b - h * d, eta)) / (2 * h)
    assert abs(fd - np.vdot(lam, d).real) < 1e-9 * abs(fd)


def test_grad_U_unconstrained_fd(setup, rng):
    U, b, eta, x, lam, G = setup
    E = rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape)
    h = 1e-5
    fd = (loss(U + h * E, b, eta) - loss(U - h * E, b, eta)) / (2 * h)
    an = np.sum(np.conj(G) * E).real
    assert abs(fd - an) < 1e-6 * abs(an)


def _random_su3_algebra(rng):
    A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    T = 0.5 * (A + A.conj().T)
    return T - np.trace(T) / 3 * np.eye(3)


def test_projected_force_fd_links(setup, rng):
    U, b, eta, x, lam, G = setup
    P = oracle.projected_force(U, G)
    assert np.abs(np.trace(P, axis1=-2, axis2=-1)).max() < 1e-14
    assert np.abs(P - np.conj(np.swapaxes(P, -1, -2))).max() < 1e-14
    h = 1e-5
    V = oracle.volume(L)
    for _ in range(16):
        mu, s = rng.integers(0, 4), rng.integers(0, V)
        T = _random_su3_algebra(rng)
        Up, Um = U.copy(), U.copy()
        Up[mu, s] = expm(1j * h * T) @ U[mu, s]
        Um[mu, s] = expm(-1j * h * T) @ U[mu, s]
        fd = (loss(Up, b, eta) - loss(Um, b, eta)) / (2 * h)
        an = np.trace(T @ P[mu, s]).real
        assert abs(fd - an) < 1e-6 * max(abs(an), 1e-3), (mu, s, fd, an)


def test_projected_force_fd_full_direction(setup, rng):
    U, b, eta, x, lam, G = setup
    P = oracle.projected_force(U, G)
    V = oracle.volume(L)
    T = np.stack([[_random_su3_algebra(rng) for _ in range(V)] for _ in range(4)])
    h = 1e-5
    w, Q = np.linalg.eigh(T)
    ex = lambda e: (Q * np.exp(1j * e * w)[..., None, :]) @ np.conj(np.swapaxes(Q, -1, -2))
    fd = (loss(ex(h) @ U, b, eta) - loss(ex(-h) @ U, b, eta)) / (2 * h)
    an = np.einsum("mvab,mvba->", T, P).real
    assert abs(fd - an) < 1e-6 * abs(an)


# --------------------------------------------------------------------------- clover term
CSW = 1.0


@pytest.fixture(scope="module")
def setup_clover():
    U = synth.random_links(L, seed=11)
    b = synth.gaussian_spinor(L, seed=2)
    eta = synth.gaussian_spinor(L, seed=3)
    F = oracle.clover_field(U, KAPPA, CSW, L)
    x = oracle.solve(U, b, KAPPA, L, F=F, tol=TOL)
    lam = oracle.solve(U, eta, KAPPA, L, F=F, tol=TOL, dagger=True)
    G = oracle.link_gradient(x, lam, KAPPA, L, U=U, csw=CSW)
    return U, b, eta, G


def loss_clover(U, b, eta):
    F = oracle.clover_field(U, KAPPA, CSW, L)
    return np.vdot(eta, oracle.solve(U, b, KAPPA, L, F=F, tol=TOL)).real


def test_clover_grad_U_unconstrained_fd(setup_clover, rng):
    U, b, eta, G = setup_clover
    E = rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape)
    h = 1e-5
    fd = (loss_clover(U + h * E, b, eta) - loss_clover(U - h * E, b, eta)) / (2 * h)
    an = np.sum(np.conj(G) * E).real
    assert abs(fd - an) < 1e-6 * abs(an)


def test_clover_projected_force_fd(setup_clover, rng):
    U, b, eta, G = setup_clover
    P = oracle.projected_force(U, G)
    h = 1e-5
    V = oracle.volume(L)
    for _ in range(8):
        mu, s = rng.integers(0, 4), rng.integers(0, V)
        T = _random_su3_algebra(rng)
        Up, Um = U.copy(), U.copy()
        Up[mu, s] = expm(1j * h * T) @ U[mu, s]
        Um[mu, s] = expm(-1j * h * T) @ U[mu, s]
        fd = (loss_clover(Up, b, eta) - loss_clover(Um, b, eta)) / (2 * h)
        an = np.trace(T @ P[mu, s]).real
        assert abs(fd - an) < 1e-6 * max(abs(an), 1e-3), (mu, s, fd, an)
