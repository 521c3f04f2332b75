"""GPU solves of D x = b (Sec. 2: the linear solve is the main bottleneck)
through the even-odd Schur complement, plain FP64 and mixed precision
(FP32 / FP16-storage inner, FP64 defect correction), BiCGStab and CGNR,
Wilson and clover, D and D^dag.  Every solve must reach a true FP64 residual
||b - D x|| / ||b|| <= 1e-10, recomputed here by the oracle's D, and agree with
the oracle's own solve to the accuracy the residual bound implies."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, KAPPA, gauge, lib, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def lat():
    L = (6, 6, 6, 10)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2)
    return L, g, U, b


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("inner", [0, 1, 2])
def test_solve_wilson(lat, solver, inner):
    bpp = lib()
    L, g, U, b = lat
    opts = bpp.solve_opts(solver=solver, inner_prec=inner)
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, opts)
    x = to_np(x)
    res = oracle.true_residual(U, b, x, KAPPA, L, BC)
    assert res <= TOL, (res, st)
    assert st[0]["converged"] == 1 and st[0]["true_resid"] <= TOL
    assert abs(st[0]["true_resid"] - res) <= 0.05 * res + 1e-15
    x_ref = oracle.solve(U, b, KAPPA, L, BC, tol=1e-12)
    assert rel_err(x, x_ref) <= 1e-7


def test_solve_dagger(lat):
    bpp = lib()
    L, g, U, b = lat
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(dagger=True))
    x = to_np(x)
    r = b - oracle.apply_D(U, x, KAPPA, L, BC, dagger=True)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= TOL


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_solve_clover(inner):
    bpp = lib()
    L = (4, 4, 4, 6)
    g, U = gauge(L)
    csw = 1.0
    g.clover_build(KAPPA, csw)
    F = oracle.clover_field(U, KAPPA, csw, L)
    b = synth.gaussian_spinor(L, seed=2, nrhs=2)
    x, st = bpp.solve(g, to_dev(b), KAPPA, csw, TOL, bpp.solve_opts(inner_prec=inner))
    x = to_np(x)
    for r in range(2):
        assert oracle.true_residual(U, b[r], x[r], KAPPA, L, BC, F) <= TOL


def test_solve_point_sources_12():
    """The 12 spin-colour point sources of a propagator (Fig. 1), one batched solve."""
    bpp = lib()
    L = (4, 4, 4, 8)
    g, U = gauge(L)
    b = np.stack([synth.point_source(L, idx) for idx in range(12)])
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=1))
    x = to_np(x)
    for idx in range(12):
        assert oracle.true_residual(U, b[idx], x[idx], KAPPA, L, BC) <= TOL


def test_solve_host_buffers(lat):
    bpp = lib()
    L, g, U, b = lat
    bt = torch.from_numpy(b.copy())
    x, st = bpp.solve(g, bt, KAPPA, 0.0, TOL)
    assert not x.is_cuda
    assert oracle.true_residual(U, b, x.numpy(), KAPPA, L, BC) <= TOL


def test_solve_not_converged_reports(lat):
    bpp = lib()
    L, g, U, b = lat
    opts = bpp.solve_opts(inner_prec=0, max_inner=2, max_outer=1)
    with pytest.raises(bpp.NotConverged):
        bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, opts)
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, opts, raise_on_fail=False)
    assert st[0]["converged"] == 0 and st[0]["status"] == -5


def test_solve_nonfinite_input(lat):
    bpp = lib()
    L, g, U, b = lat
    bb = b.copy()
    bb[3, 1, 2] = np.nan
    with pytest.raises(bpp.BppError):
        bpp.solve(g, to_dev(bb), KAPPA, 0.0, TOL)


@pytest.mark.parametrize("inner", [0, 1, 2])
@pytest.mark.parametrize("arith", [0, 1, 2])
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_solve_outer_arithmetic(inner, arith, csw):
    """Every outer-loop arithmetic (all FP64; double-float defects with the FP64
    check; double-float defects and check) reaches the true residual as the
    oracle computes it, reports it to 5%, and agrees with the oracle's x."""
    bpp = lib()
    L = (4, 4, 6, 8)
    g, U = gauge(L)
    F = None
    if csw:
        g.clover_build(KAPPA, csw)
        F = oracle.clover_field(U, KAPPA, csw, L)
    b = synth.gaussian_spinor(L, seed=2, nrhs=2)
    x, st = bpp.solve(g, to_dev(b), KAPPA, csw, TOL, bpp.solve_opts(inner_prec=inner, outer_arith=arith))
    x = to_np(x)
    for r in range(2):
        res = oracle.true_residual(U, b[r], x[r], KAPPA, L, BC, F)
        assert res <= TOL and st[r]["converged"] == 1
        assert abs(st[r]["true_resid"] - res) <= 0.05 * res + 1e-15
        assert rel_err(x[r], oracle.solve(U, b[r], KAPPA, L, BC, F=F, tol=1e-13)) <= 1e-8


def test_solve_outer_arith_rejects_bad_value(lat):
    bpp = lib()
    L, g, U, b = lat
    o = bpp.solve_opts()
    o.outer_arith = 3
    with pytest.raises(bpp.BppError) as e:
        bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, o)
    assert e.value.code == -1
    with pytest.raises(ValueError):
        bpp.solve_opts(outer_arith=5)


@pytest.mark.parametrize("scale", [1e-40, 1e-20, 1e20, 1e60])
@pytest.mark.parametrize("inner", [1, 2])
def test_solve_any_rhs_scale(scale, inner):
    """The solver normalises b, so the double-float outer loop (FP32 exponent
    range) works for right-hand sides of any magnitude; x scales with b."""
    bpp = lib()
    L = (4, 4, 4, 6)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2)
    x1, _ = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=inner))
    xs, st = bpp.solve(g, to_dev(b * scale), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=inner))
    assert st[0]["converged"] == 1
    assert oracle.true_residual(U, b * scale, to_np(xs), KAPPA, L, BC) <= TOL
    assert rel_err(to_np(xs) / scale, to_np(x1)) <= 1e-9


@pytest.mark.parametrize("scale", [1e-30, 1e-20, 1e20])
def test_dslash_f64df_scales(scale):
    """Double-float dslash across magnitudes (integer split fast path and the
    FP64 route for small values)."""
    bpp = lib()
    L = (4, 4, 4, 6)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = synth.gaussian_spinor(L, seed=2)[:Vh] * scale
    ref = oracle.hop_eo(U, psi, KAPPA, L, 0, BC)
    out = to_np(bpp.dslash(g, to_dev(psi), KAPPA, 0, bpp.F64DF))
    assert rel_err(out, ref) <= 1e-12
