"""Domain decomposition in x4 on one GPU (slabs with their own links, face
buffers exchanged by device copies): the decomposed hopping term and Schur
operator must equal the undecomposed ones bit for bit in every storage
format, parity and adjoint, for 2, 3 and 4 slabs (the antiperiodic boundary
then falls on a slab boundary); the decomposed FP64 solve must reach the
oracle's true residual, agree with the undecomposed solve, and give the same
bits with a host reducer that sums the slabs in the same order."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, KAPPA, gauge, lib, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _eighteen_real_links(monkeypatch):
    """The slabs read the 18-real links; the undecomposed kernel is compared
    in the same form (with two-row links FP32 differs by the rounding of the
    rebuilt third row)."""
    monkeypatch.setenv("BPP_LINK_COMPRESSION", "0")


CASES = [((4, 4, 4, 8), 2), ((6, 4, 2, 12), 3), ((4, 2, 4, 16), 4)]


@pytest.mark.parametrize("L,ndom", CASES)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_dd_dslash_bit_identical(L, ndom, prec):
    bpp = lib()
    g, U = gauge(L)
    dd = bpp.DomainDecomposition(to_dev(U), L, ndom, BC)
    Vh = oracle.volume(L) // 2
    dt = torch.complex128 if prec == 0 else torch.complex64
    psi = to_dev(synth.gaussian_spinor(L, seed=7, nrhs=2)[:, :Vh], dt)
    for parity in (0, 1):
        ref = bpp.dslash(g, psi, KAPPA, parity, prec)
        out = dd.dslash(psi, KAPPA, parity, prec)
        assert torch.equal(out, ref), (parity, (out - ref).abs().max().item())
    if prec == 0:
        full = synth.gaussian_spinor(L, seed=7, nrhs=2)[0, :Vh]
        assert rel_err(to_np(dd.dslash(psi[0], KAPPA, 0, 0)), oracle.hop_eo(U, full, KAPPA, L, 0)) <= 1e-13


@pytest.mark.parametrize("L,ndom", CASES[:2])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_dd_schur_bit_identical(L, ndom, prec, dagger):
    bpp = lib()
    g, U = gauge(L)
    dd = bpp.DomainDecomposition(to_dev(U), L, ndom, BC)
    Vh = oracle.volume(L) // 2
    dt = torch.complex128 if prec == 0 else torch.complex64
    x = to_dev(synth.gaussian_spinor(L, seed=8)[:Vh], dt)
    ref = bpp.schur_apply(g, x, KAPPA, 0.0, dagger, prec)
    out = dd.schur_apply(x, KAPPA, dagger, prec)
    assert torch.equal(out, ref)


def test_dd_periodic_time_boundary():
    """bc = +1 in time: no sign at the lattice's t boundary."""
    bpp = lib()
    L, bc = (4, 4, 4, 8), (1, 1, 1, 1)
    U = synth.random_links(L)
    g = bpp.Gauge(to_dev(U), L, bc)
    dd = bpp.DomainDecomposition(to_dev(U), L, 2, bc)
    Vh = oracle.volume(L) // 2
    psi = to_dev(synth.gaussian_spinor(L, seed=9)[:Vh])
    assert torch.equal(dd.dslash(psi, KAPPA, 1, 0), bpp.dslash(g, psi, KAPPA, 1, 0))


@pytest.mark.parametrize("L,ndom", CASES[:2])
def test_dd_solve(L, ndom):
    bpp = lib()
    g, U = gauge(L)
    dd = bpp.DomainDecomposition(to_dev(U), L, ndom, BC)
    b = synth.gaussian_spinor(L, seed=2, nrhs=2)
    x, st = dd.solve(to_dev(b), KAPPA, 1e-10)
    x = to_np(x)
    x_ref, _ = bpp.solve(g, to_dev(b), KAPPA, 0.0, 1e-10, bpp.solve_opts(inner_prec=0))
    for r in range(2):
        res = oracle.true_residual(U, b[r], x[r], KAPPA, L, BC)
        assert res <= 1e-10 and st[r]["converged"] == 1
        assert abs(st[r]["true_resid"] - res) <= 0.05 * res + 1e-15
        assert rel_err(x[r], to_np(x_ref[r])) <= 1e-9


def test_dd_solve_dagger():
    bpp = lib()
    L = (4, 4, 4, 8)
    g, U = gauge(L)
    dd = bpp.DomainDecomposition(to_dev(U), L, 2, BC)
    b = synth.gaussian_spinor(L, seed=4)
    x, st = dd.solve(to_dev(b), KAPPA, 1e-10, bpp.solve_opts(inner_prec=0, dagger=True))
    r = b - oracle.apply_D(U, to_np(x), KAPPA, L, BC, dagger=True)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10


def test_dd_host_reducer_same_bits():
    """A reducer registered from Python that sums the slabs in slab order gives
    the same solution bits as the library's device sum (same additions in the
    same order); a failing reducer is reported as an error."""
    bpp = lib()
    L = (4, 4, 2, 12)
    g, U = gauge(L)
    dd = bpp.DomainDecomposition(to_dev(U), L, 3, BC)
    b = to_dev(synth.gaussian_spinor(L, seed=2))
    x0, _ = dd.solve(b, KAPPA, 1e-10)
    calls = []

    def reducer(parts):
        calls.append(parts.shape)
        out = np.zeros(parts.shape[1])
        for k in range(parts.shape[0]):
            out += parts[k]
        return out
    dd.set_reducer(reducer)
    x1, _ = dd.solve(b, KAPPA, 1e-10)
    assert calls and all(c == (3, 4) for c in calls)
    assert torch.equal(x0, x1)
    dd.set_reducer(lambda parts: 1 / 0)
    with pytest.raises(bpp.BppError):
        dd.solve(b, KAPPA, 1e-10)
    dd.set_reducer(None)
    x2, _ = dd.solve(b, KAPPA, 1e-10)
    assert torch.equal(x0, x2)


def test_dd_rejects_bad_splits():
    bpp = lib()
    L = (4, 4, 4, 8)
    U = to_dev(synth.random_links(L))
    for ndom in (1, 3, 8):       # 8 / 3 not whole, 8 / 8 = 1 odd
        with pytest.raises(bpp.BppError) as e:
            bpp.DomainDecomposition(U, L, ndom, BC)
        assert e.value.code == -1
