"""Edge cases on the GPU: the 2^4 lattice (every forward and backward neighbour
coincide and both terms add), the largest batch, a zero right-hand side,
initial guesses, and the error paths of the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, KAPPA, gauge, lib, max_err, rel_err, round32, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6), (2, 5e-3), (3, 1e-12)])
def test_two_to_the_four(prec, tol):
    bpp = lib()
    L = (2, 2, 2, 2)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = synth.gaussian_spinor(L, seed=2)[:Vh]
    Uo = round32(U) if prec == 1 else U
    if prec == 1:
        psi = round32(psi)
        g, _ = gauge(L, Uo)
    dt = torch.complex128 if prec in (0, 3) else torch.complex64
    for parity in (0, 1):
        out = to_np(bpp.dslash(g, to_dev(psi, dt), KAPPA, parity, prec))
        assert rel_err(out, oracle.hop_eo(Uo, psi, KAPPA, L, parity, BC)) <= tol


def test_two_to_the_four_solve_dense():
    bpp = lib()
    L = (2, 2, 2, 2)
    g, U = gauge(L)
    g.clover_build(KAPPA, 1.0)
    F = oracle.clover_field(U, KAPPA, 1.0, L)
    b = synth.gaussian_spinor(L, seed=2)
    x_lu = np.linalg.solve(oracle.dense_D(U, KAPPA, L, BC, F), b.ravel()).reshape(b.shape)
    for inner in (0, 1, 2):
        x, st = bpp.solve(g, to_dev(b), KAPPA, 1.0, TOL, bpp.solve_opts(inner_prec=inner))
        assert rel_err(to_np(x), x_lu) <= 1e-9


def test_largest_batch_and_limit():
    bpp = lib()
    L = (4, 4, 2, 2)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2, nrhs=64)
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=1))
    for r in (0, 31, 63):
        assert oracle.true_residual(U, b[r], to_np(x[r]), KAPPA, L, BC) <= TOL
    with pytest.raises(bpp.BppError) as e:
        bpp.solve(g, to_dev(synth.gaussian_spinor(L, seed=2, nrhs=65)), KAPPA, 0.0, TOL)
    assert e.value.code == -1


def test_zero_rhs_and_mixed_batch():
    bpp = lib()
    L = (4, 4, 4, 4)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2, nrhs=3)
    b[1] = 0.0
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=2))
    xn = to_np(x)
    assert np.abs(xn[1]).max() == 0.0 and st[1]["converged"] == 1
    for r in (0, 2):
        assert oracle.true_residual(U, b[r], xn[r], KAPPA, L, BC) <= TOL


def test_initial_guess():
    bpp = lib()
    L = (4, 4, 4, 6)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2)
    x_ref = oracle.solve(U, b, KAPPA, L, BC, tol=1e-13)
    # the exact solution as the guess: no correction needed
    x0 = to_dev(x_ref)
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=1, use_x0=True), x=x0)
    assert st[0]["outer_iters"] == 0 and st[0]["true_resid"] <= TOL
    # a rough guess converges too
    xr = to_dev(x_ref + 0.1 * synth.gaussian_spinor(L, seed=9))
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=2, use_x0=True), x=xr)
    assert oracle.true_residual(U, b, to_np(x), KAPPA, L, BC) <= TOL


def test_host_buffers_multi_rhs():
    bpp = lib()
    L = (4, 4, 4, 4)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2, nrhs=3)
    x, st = bpp.solve(g, torch.from_numpy(b.copy()), KAPPA, 0.0, TOL)
    assert not x.is_cuda
    for r in range(3):
        assert oracle.true_residual(U, b[r], x[r].numpy(), KAPPA, L, BC) <= TOL


def test_error_paths():
    bpp = lib()
    L = (4, 4, 4, 4)
    g, U = gauge(L)
    x = to_dev(synth.gaussian_spinor(L, seed=2)[:128])
    # clover term used before it is built
    with pytest.raises(bpp.BppError) as e:
        bpp.schur_apply(g, x, KAPPA, 1.0)
    assert e.value.code == -2
    with pytest.raises(bpp.BppError) as e:
        bpp.clover_apply(g, x, 0)
    assert e.value.code == -2
    g.clover_build(KAPPA, 1.0)
    # kappa / csw differ from the ones the clover term was built with
    with pytest.raises(bpp.BppError) as e:
        bpp.schur_apply(g, x, 0.1, 1.0)
    assert e.value.code == -1
    # bad parity and precision
    rc = bpp._lib.bpp_dslash(g.handle, bpp._ptr(x), bpp._ptr(torch.empty_like(x)), KAPPA, 7, 0, 1, bpp._stream())
    assert rc == -1
    rc = bpp._lib.bpp_dslash(g.handle, bpp._ptr(x), bpp._ptr(torch.empty_like(x)), KAPPA, 0, 9, 1, bpp._stream())
    assert rc == -1
    # aliased input and output
    rc = bpp._lib.bpp_dslash(g.handle, bpp._ptr(x), bpp._ptr(x), KAPPA, 0, 0, 1, bpp._stream())
    assert rc == -1
    # the library still works after the errors
    out = to_np(bpp.dslash(g, x, KAPPA, 0, bpp.F64))
    assert rel_err(out, oracle.hop_eo(U, to_np(x), KAPPA, L, 0, BC)) <= 1e-13


@pytest.mark.parametrize("arith", [1, 2])
def test_prof_classes_cover_the_solve(arith):
    """With launch timing on, a host-driven mixed-precision solve credits the
    hopping kernels of the inner precision and the double-float outer loop (and
    the FP64 hop of the true-residual check with outer_arith 1, none with 2),
    the Krylov and outer-loop vector kernels, the layout conversion and the
    control kernels, each with time and (except control) algorithmic bytes."""
    bpp = lib()
    L = (4, 4, 4, 8)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2)
    bpp.prof_enable(True)
    for c in range(10):
        bpp.prof_read(c, reset=True)
    bpp.solve(g, to_dev(b), KAPPA, 0.0, 1e-10, bpp.solve_opts(inner_prec=bpp.F32, use_graph=0, outer_arith=arith))
    bpp.prof_enable(False)
    got = {c: bpp.prof_read(c, reset=True) for c in range(10)}
    for c in ((0,) if arith == 1 else ()) + (1, 3, 4, 5, 6, 7):
        n, ms, by = got[c]
        assert n > 0 and ms > 0.0, (c, got[c])
        assert (by > 0.0) == (c != 7), (c, got[c])
    if arith == 2:
        assert got[0][0] == 0
    assert got[9][0] == 0
