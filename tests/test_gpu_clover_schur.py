"""GPU parity of the clover term (Eq. 1: F is a 12x12 Hermitian matrix made
of links), its inverse, the even-odd Schur operator and the full FP64 D
(with and without clover, D and D^dag) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, KAPPA, eo_split, gauge, lib, max_err, rel_err, round32, to_dev, to_np

pytestmark = pytest.mark.gpu
CSW = 1.0


@pytest.fixture(scope="module", params=[(4, 4, 4, 4), (6, 6, 6, 10)])
def setup(request):
    L = request.param
    g, U = gauge(L)
    g.clover_build(KAPPA, CSW)
    F = oracle.clover_field(U, KAPPA, CSW, L)
    return L, g, U, F


@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("inverse", [False, True])
def test_clover_apply_f64(setup, parity, inverse):
    bpp = lib()
    L, g, U, F = setup
    A = oracle.clover_blocks(F, L, parity)
    if inverse:
        A = np.linalg.inv(A)
    x = synth.gaussian_spinor(L, seed=3)[: oracle.volume(L) // 2]
    ref = oracle.apply_site_matrix(A, x)
    out = to_np(bpp.clover_apply(g, to_dev(x), parity, inverse, bpp.F64))
    assert rel_err(out, ref) <= 1e-13
    assert max_err(out, ref) <= 1e-13


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (2, 5e-3)])
def test_clover_apply_low(setup, prec, tol):
    bpp = lib()
    L, g, U, F = setup
    A = oracle.clover_blocks(F, L, 0)
    x = round32(synth.gaussian_spinor(L, seed=3)[: oracle.volume(L) // 2])
    ref = oracle.apply_site_matrix(A, x)
    out = to_np(bpp.clover_apply(g, to_dev(x, torch.complex64), 0, False, prec))
    assert rel_err(out, ref) <= tol


@pytest.mark.parametrize("dagger", [False, True])
def test_schur_clover_f64(setup, dagger):
    bpp = lib()
    L, g, U, F = setup
    S = oracle.Schur(U, KAPPA, L, BC, F)
    x = synth.gaussian_spinor(L, seed=4)[S.even]
    ref = S.apply(x, dagger=dagger)
    out = to_np(bpp.schur_apply(g, to_dev(x), KAPPA, CSW, dagger, bpp.F64))
    assert rel_err(out, ref) <= 1e-13


@pytest.mark.parametrize("dagger", [False, True])
def test_schur_wilson_f64(setup, dagger):
    bpp = lib()
    L, g, U, F = setup
    S = oracle.Schur(U, KAPPA, L, BC, None)
    x = synth.gaussian_spinor(L, seed=4)[S.even]
    ref = S.apply(x, dagger=dagger)
    out = to_np(bpp.schur_apply(g, to_dev(x), KAPPA, 0.0, dagger, bpp.F64))
    assert rel_err(out, ref) <= 1e-13
    assert max_err(out, ref) <= 1e-13


def test_schur_f32(setup):
    bpp = lib()
    L, g, U, F = setup
    S = oracle.Schur(round32(U), KAPPA, L, BC, None)
    x = round32(synth.gaussian_spinor(L, seed=4)[S.even])
    ref = S.apply(x)
    out = to_np(bpp.schur_apply(g, to_dev(x, torch.complex64), KAPPA, 0.0, False, bpp.F32))
    assert rel_err(out, ref) <= 1e-6


@pytest.mark.parametrize("csw", [0.0, CSW])
@pytest.mark.parametrize("dagger", [False, True])
def test_dirac_full_f64(setup, csw, dagger):
    bpp = lib()
    L, g, U, F = setup
    x = synth.gaussian_spinor(L, seed=5)
    ref = oracle.apply_D(U, x, KAPPA, L, BC, F if csw else None, dagger=dagger)
    out = to_np(bpp.dirac_apply(g, to_dev(x), KAPPA, csw, dagger))
    assert rel_err(out, ref) <= 1e-13
    assert max_err(out, ref) <= 1e-13


def test_clover_abelian_flux_spectrum():
    """Uniform abelian flux: A = 1 + F has eigenvalues 1 -/+ kappa c_SW sin(theta)."""
    bpp = lib()
    L = (4, 4, 2, 2)
    U = synth.abelian_flux_links(L, 1)
    g, _ = gauge(L, U)
    g.clover_build(KAPPA, CSW)
    theta = 2 * np.pi / 16
    Vh = oracle.volume(L) // 2
    # apply A to the 12 unit vectors at every site: columns of the per-site matrix
    cols = []
    for k in range(12):
        e = np.zeros((Vh, 12), dtype=np.complex128)
        e[:, k] = 1.0
        cols.append(to_np(bpp.clover_apply(g, to_dev(e.reshape(Vh, 4, 3)), 0, False, bpp.F64)).reshape(Vh, 12))
    A = np.stack(cols, axis=2)
    expect = np.sort(np.repeat([1 - KAPPA * CSW * np.sin(theta), 1 + KAPPA * CSW * np.sin(theta)], 6))
    for s in range(Vh):
        assert np.abs(np.sort(np.linalg.eigvalsh(A[s])) - expect).max() < 1e-14


@pytest.mark.parametrize("csw", [0.0, CSW])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_f64df(setup, csw, dagger):
    """Schur operator in double-float arithmetic (the outer loop's defects): bar 1e-12."""
    bpp = lib()
    L, g, U, F = setup
    S = oracle.Schur(U, KAPPA, L, BC, F if csw else None)
    x = synth.gaussian_spinor(L, seed=4)[S.even]
    ref = S.apply(x, dagger=dagger)
    out = to_np(bpp.schur_apply(g, to_dev(x), KAPPA, csw, dagger, bpp.F64DF))
    assert rel_err(out, ref) <= 1e-12
