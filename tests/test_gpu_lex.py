"""The lexical (full-lattice, no even-odd preconditioning) propagator solve of
Fig. 1 with its operator modes D, Ddag and DdagD, FP64 defect correction
around an FP32 or FP64 inner solve.  Every solve is checked by the oracle:
the residual of its own linear system ||b - A x|| / ||b|| <= 1e-10 with the
oracle's FP64 D, and x against the oracle's even-odd solve where A = D or
D^dag.  The 12-source propagator of Fig. 1 (point sources idx = ic + 3 id) is
compared with the even-odd solve."""
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
    L = (6, 4, 4, 10)
    g, U = gauge(L)
    b = synth.gaussian_spinor(L, seed=2, nrhs=2)
    return L, g, U, b


@pytest.mark.parametrize("inner", [0, 1])
@pytest.mark.parametrize("solver", [0, 1])
def test_lex_mode_D(lat, inner, solver):
    bpp = lib()
    L, g, U, b = lat
    opts = bpp.solve_opts(solver=solver, inner_prec=inner)
    x, st = bpp.solve_lex(g, to_dev(b), KAPPA, 0.0, TOL, bpp.LEX_D, opts)
    x = to_np(x)
    for r in range(2):
        res = oracle.true_residual(U, b[r], x[r], KAPPA, L, BC)
        assert res <= TOL and st[r]["converged"] == 1, (r, res, st[r])
        assert abs(st[r]["true_resid"] - res) <= 0.05 * res + 1e-15
        assert rel_err(x[r], oracle.solve(U, b[r], KAPPA, L, BC, tol=1e-12)) <= 1e-7


@pytest.mark.parametrize("solver", [0, 1])
def test_lex_mode_Ddag(lat, solver):
    bpp = lib()
    L, g, U, b = lat
    x, st = bpp.solve_lex(g, to_dev(b[0]), KAPPA, 0.0, TOL, bpp.LEX_DDAG,
                          bpp.solve_opts(solver=solver, inner_prec=bpp.F32))
    x = to_np(x)
    r = b[0] - oracle.apply_D(U, x, KAPPA, L, BC, dagger=True)
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= TOL
    assert rel_err(x, oracle.solve(U, b[0], KAPPA, L, BC, tol=1e-12, dagger=True)) <= 1e-7


@pytest.mark.parametrize("inner", [0, 1])
def test_lex_mode_DdagD(lat, inner):
    bpp = lib()
    L, g, U, b = lat
    x, st = bpp.solve_lex(g, to_dev(b[1]), KAPPA, 0.0, TOL, bpp.LEX_DDAGD, bpp.solve_opts(inner_prec=inner))
    x = to_np(x)
    Ax = oracle.apply_D(U, oracle.apply_D(U, x, KAPPA, L, BC), KAPPA, L, BC, dagger=True)
    res = np.linalg.norm(b[1] - Ax) / np.linalg.norm(b[1])
    assert res <= TOL and abs(st[0]["true_resid"] - res) <= 0.05 * res + 1e-15


def test_lex_clover():
    bpp = lib()
    L = (4, 4, 4, 6)
    csw = 1.0
    g, U = gauge(L)
    g.clover_build(KAPPA, csw)
    F = oracle.clover_field(U, KAPPA, csw, L)
    b = synth.gaussian_spinor(L, seed=3)
    for mode, dag in ((bpp.LEX_D, False), (bpp.LEX_DDAG, True)):
        x, st = bpp.solve_lex(g, to_dev(b), KAPPA, csw, TOL, mode, bpp.solve_opts(inner_prec=bpp.F32))
        r = b - oracle.apply_D(U, to_np(x), KAPPA, L, BC, F=F, dagger=dag)
        assert np.linalg.norm(r) / np.linalg.norm(b) <= TOL


def test_lex_propagator_twelve_sources_matches_eo():
    """Fig. 1's loop over idx = ic + Nc id: the lexical mixed-precision
    propagator (12 point sources in one call, CG on the normal equations)
    agrees with the even-odd solve to the accuracy the residuals allow."""
    bpp = lib()
    L = (4, 4, 4, 8)
    g, U = gauge(L)
    b = np.stack([synth.point_source(L, idx) for idx in range(12)])
    x_lex, st = bpp.solve_lex(g, to_dev(b), KAPPA, 0.0, TOL, bpp.LEX_D,
                              bpp.solve_opts(solver=bpp.CGNR, inner_prec=bpp.F32))
    x_eo, _ = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=bpp.F32))
    x_lex, x_eo = to_np(x_lex), to_np(x_eo)
    for idx in range(12):
        assert oracle.true_residual(U, b[idx], x_lex[idx], KAPPA, L, BC) <= TOL
        assert rel_err(x_lex[idx], x_eo[idx]) <= 1e-8


def test_lex_rejects_fp16_and_bad_mode(lat):
    bpp = lib()
    L, g, U, b = lat
    with pytest.raises(bpp.BppError) as e:
        bpp.solve_lex(g, to_dev(b[0]), KAPPA, 0.0, TOL, bpp.LEX_D, bpp.solve_opts(inner_prec=bpp.F16))
    assert e.value.code == -2
    with pytest.raises(bpp.BppError) as e:
        bpp.solve_lex(g, to_dev(b[0]), KAPPA, 0.0, TOL, 7)
    assert e.value.code == -1


def test_lex_host_buffers_and_zero_rhs(lat):
    bpp = lib()
    L, g, U, b = lat
    bh = torch.from_numpy(np.stack([b[0], np.zeros_like(b[0])]))
    x, st = bpp.solve_lex(g, bh, KAPPA, 0.0, TOL, bpp.LEX_D, bpp.solve_opts(inner_prec=bpp.F32))
    assert not x.is_cuda
    x = x.numpy()
    assert oracle.true_residual(U, b[0], x[0], KAPPA, L, BC) <= TOL
    assert np.count_nonzero(x[1]) == 0 and st[1]["converged"] == 1
