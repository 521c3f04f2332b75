"""GPU parity of the even-odd hopping term (Eq. 1, Sec. 3) against the FP64 oracle.

Bars: FP64 <= 1e-13 (norm-relative and element-wise relative to the largest
element); FP32 <= 1e-6 with the inputs (spinor and links) rounded to FP32
before the oracle sees them; FP16 storage: error reported, bound 5e-3.
Lattices span several thread blocks with a ragged tail (Vh not a multiple of
the block) and asymmetric extents, including L_mu = 2.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, KAPPA, gauge, lib, max_err, rel_err, round32, to_dev, to_np

pytestmark = pytest.mark.gpu

LATTICES = [(4, 4, 4, 4), (6, 6, 6, 10), (8, 8, 8, 8), (4, 6, 8, 10), (2, 4, 2, 6)]


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_f64(L, parity):
    bpp = lib()
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = synth.gaussian_spinor(L, seed=2)[:Vh]          # any half field
    ref = oracle.hop_eo(U, psi, KAPPA, L, parity, BC)
    out = to_np(bpp.dslash(g, to_dev(psi), KAPPA, parity, bpp.F64))
    assert rel_err(out, ref) <= 1e-13
    assert max_err(out, ref) <= 1e-13


@pytest.mark.parametrize("L", [(6, 6, 6, 10), (8, 8, 8, 8)])
@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_f32(L, parity):
    bpp = lib()
    U = round32(synth.random_links(L))
    g, _ = gauge(L, U)
    Vh = oracle.volume(L) // 2
    psi = round32(synth.gaussian_spinor(L, seed=2)[:Vh])
    ref = oracle.hop_eo(U, psi, KAPPA, L, parity, BC)
    out = to_np(bpp.dslash(g, to_dev(psi, torch.complex64), KAPPA, parity, bpp.F32))
    assert rel_err(out, ref) <= 1e-6


@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_f16(parity):
    bpp = lib()
    L = (8, 8, 8, 8)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = synth.gaussian_spinor(L, seed=2)[:Vh]
    ref = oracle.hop_eo(U, psi, KAPPA, L, parity, BC)
    out = to_np(bpp.dslash(g, to_dev(psi, torch.complex64), KAPPA, parity, bpp.F16))
    err = rel_err(out, ref)
    print(f"FP16-storage dslash norm-relative error {err:.2e}")
    assert err <= 5e-3


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 6, 10)])
def test_dslash_full_f64(L):
    bpp = lib()
    g, U = gauge(L)
    psi = synth.gaussian_spinor(L, seed=2)
    ref = oracle.apply_D(U, psi, KAPPA, L, BC)
    out = to_np(bpp.dslash(g, to_dev(psi), KAPPA, bpp.FULL, bpp.F64))
    assert rel_err(out, ref) <= 1e-13
    assert max_err(out, ref) <= 1e-13


def test_dslash_multi_rhs_matches_single():
    bpp = lib()
    L = (6, 6, 6, 10)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psis = synth.gaussian_spinor(L, seed=2, nrhs=3)[:, :Vh]
    out = to_np(bpp.dslash(g, to_dev(psis), KAPPA, 0, bpp.F64))
    for r in range(3):
        one = to_np(bpp.dslash(g, to_dev(psis[r]), KAPPA, 0, bpp.F64))
        assert np.array_equal(out[r], one)
        assert rel_err(one, oracle.hop_eo(U, psis[r], KAPPA, L, 0, BC)) <= 1e-13


def test_dslash_free_field_plane_wave():
    """U = 1: a plane wave with allowed momentum is an eigenvector of the full D."""
    bpp = lib()
    L = (8, 4, 4, 6)
    g, U = gauge(L, synth.unit_links(L))
    ps = oracle.momenta(L, BC)
    p = np.array([ps[0][1], ps[1][2], ps[2][3], ps[3][0]])
    u = np.arange(12).reshape(4, 3) * (0.3 + 0.1j) + 1.0
    x = oracle.coords(L)
    phase = np.exp(1j * (x @ p))
    psi = phase[:, None, None] * u[None]
    out = to_np(bpp.dslash(g, to_dev(psi), KAPPA, bpp.FULL, bpp.F64))
    expect = phase[:, None, None] * (oracle.free_field_Dp(p, KAPPA) @ u)[None]
    assert np.abs(out - expect).max() < 1e-13 * np.abs(expect).max()


@pytest.mark.parametrize("L", [(6, 6, 6, 10), (8, 8, 8, 8), (2, 4, 2, 6)])
@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_f64df(L, parity):
    """FP64 values with double-float arithmetic (~48-bit significands): bar 1e-12."""
    bpp = lib()
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = synth.gaussian_spinor(L, seed=2)[:Vh]
    ref = oracle.hop_eo(U, psi, KAPPA, L, parity, BC)
    out = to_np(bpp.dslash(g, to_dev(psi), KAPPA, parity, bpp.F64DF))
    err = rel_err(out, ref)
    print(f"double-float dslash norm-relative error {err:.2e}")
    assert err <= 1e-12
    assert max_err(out, ref) <= 1e-12


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("nrhs", [2, 4, 6, 12])
def test_dslash_multi_rhs_low_precision(prec, nrhs):
    """Right-hand sides of one gauge field (the register-blocked path shares each
    link load): every RHS matches its own single-RHS result and the oracle."""
    bpp = lib()
    L = (8, 8, 8, 8)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psis = synth.gaussian_spinor(L, seed=5, nrhs=nrhs)[:, :Vh]
    if prec == 1:
        psis = round32(psis)
    dev = to_dev(psis, torch.complex64)
    for parity in (0, 1):
        out = to_np(bpp.dslash(g, dev, KAPPA, parity, prec))
        for r in range(nrhs):
            one = to_np(bpp.dslash(g, dev[r].contiguous(), KAPPA, parity, prec))
            assert rel_err(out[r], one) <= (1e-6 if prec == 1 else 5e-3)
        ref = oracle.hop_eo(round32(U) if prec == 1 else U, psis[nrhs - 1], KAPPA, L, parity, BC)
        assert rel_err(out[nrhs - 1], ref) <= (1e-6 if prec == 1 else 5e-3)


@pytest.mark.parametrize("L", [(6, 6, 6, 10), (2, 4, 2, 6)])
def test_dslash_two_row_links(L, monkeypatch):
    """Exact SU(3) links: the FP32 hop reads the two-row form (row 3 rebuilt
    as conj(row1 x row2); 48 B per link in the work counter), agrees with the
    oracle on the FP64 links to 1e-6 and with the 18-real form; links that are
    not SU(3) to 1e-10 keep the 18-real form, and FP16 always does."""
    bpp = lib()
    prec, tol, spin, full = 1, 1e-6, 96, 72
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = synth.gaussian_spinor(L, seed=2)[:Vh]
    ref = oracle.hop_eo(U, psi, KAPPA, L, 0, BC)
    bpp.work_read(prec, reset=True)
    out = to_np(bpp.dslash(g, to_dev(psi, torch.complex64), KAPPA, 0, prec))
    assert bpp.work_read(prec, reset=True)[1] == Vh * (8 * 48 + 2 * spin)
    assert rel_err(out, ref) <= tol
    monkeypatch.setenv("BPP_LINK_COMPRESSION", "0")
    out18 = to_np(bpp.dslash(g, to_dev(psi, torch.complex64), KAPPA, 0, prec))
    assert bpp.work_read(prec, reset=True)[1] == Vh * (8 * full + 2 * spin)
    assert rel_err(out, out18) <= tol
    monkeypatch.delenv("BPP_LINK_COMPRESSION")
    g32, _ = gauge(L, round32(U))          # FP32-rounded: unitary only to ~1e-7
    bpp.dslash(g32, to_dev(psi, torch.complex64), KAPPA, 0, prec)
    assert bpp.work_read(prec, reset=True)[1] == Vh * (8 * full + 2 * spin)
    bpp.work_read(2, reset=True)
    bpp.dslash(g, to_dev(psi, torch.complex64), KAPPA, 0, 2)
    assert bpp.work_read(2, reset=True)[1] == Vh * (8 * 36 + 2 * 52)
