"""Parity at the workloads' full sizes, in the configuration the benchmark times.

The oracle cannot apply D to every site of these lattices in seconds, so it is
evaluated at sampled sites (plain loops, one site at a time), and solves are
checked by their true residual: with the oracle's full FP64 D where that takes
a few seconds (32^3x64, 24^3x48, the uneven batch), and at 48^3x96 by the
library's FP64 D (itself parity-tested against the oracle) plus the oracle at
sampled sites."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, KAPPA, lib, rel_err, round32, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _sample(n, count, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=count, replace=False))


@pytest.fixture(scope="module")
def big32():
    bpp = lib()
    L = (32, 32, 32, 64)
    U = synth.random_links(L, seed=1)
    g = bpp.Gauge(to_dev(U), L)
    return L, U, g


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6), (2, 5e-3)])
def test_dslash_32x64_sampled(big32, prec, tol):
    bpp = lib()
    L, U, g = big32
    Vh = oracle.volume(L) // 2
    psi = synth.gaussian_spinor(L, seed=2)[:Vh]
    Uo = U
    if prec == 1:
        psi = round32(psi)
        Uo = round32(U)
    dt = torch.complex128 if prec == 0 else torch.complex64
    out = to_np(bpp.dslash(g, to_dev(psi, dt), KAPPA, 0, prec))
    even = oracle.parity_sites(L, 0)
    k = _sample(Vh, 4096, 5)                       # sampled output sites (half-lattice index)
    full = oracle.embed(L, psi, 1)
    ref = oracle.apply_D(Uo, full, KAPPA, L, BC, sites=even[k])
    assert rel_err(out[k], ref) <= tol
    if prec == 0:
        assert np.abs(out[k] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_plain_fp64_8x8x8x8():
    """The plain FP64 workload on 8^4 (seed-1 links, kappa 0.12, one Gaussian
    source): one FP64 dslash against the oracle at 1e-13, then the FP64
    even-odd BiCGStab (no reduced precision anywhere) to a relative residual of
    the Schur system of 1e-12, recomputed by the oracle; the full-D residual is
    reported and x agrees with the oracle's own solve."""
    bpp = lib()
    L = (8, 8, 8, 8)
    U = synth.random_links(L, seed=1)
    g = bpp.Gauge(to_dev(U), L)
    b = synth.gaussian_spinor(L, seed=2)
    Vh = oracle.volume(L) // 2
    psi_o = b[oracle.parity_sites(L, 1)]
    out = to_np(bpp.dslash(g, to_dev(psi_o), KAPPA, 0, bpp.F64))
    ref = oracle.hop_eo(U, psi_o, KAPPA, L, 0)
    assert out.shape == (Vh, 4, 3)
    assert rel_err(out, ref) <= 1e-13
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()
    S = oracle.Schur(U, KAPPA, L, BC)
    bhat = S.prepare(b)
    bn, bhn = np.linalg.norm(b), np.linalg.norm(bhat)
    # the library stops on the full-D residual, which equals the Schur residual
    # times ||bhat|| / ||b|| (the odd half is exact after the reconstruction)
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, 1e-12 * bhn / bn, bpp.solve_opts(inner_prec=bpp.F64))
    x = to_np(x)
    even = oracle.parity_sites(L, 0)
    schur_res = np.linalg.norm(bhat - S.apply(x[even])) / bhn
    full_res = oracle.true_residual(U, b, x, KAPPA, L, BC)
    print(f"8^4 FP64: Schur residual {schur_res:.3e}, full-D residual {full_res:.3e}, "
          f"{st[0]['inner_iters']} BiCGStab iterations")
    assert schur_res <= 1e-12
    assert full_res <= 1e-12
    x_ref = oracle.solve(U, b, KAPPA, L, BC, tol=1e-13)
    assert rel_err(x, x_ref) <= 1e-10


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_solve_32x64_bench_config(big32, inner):
    bpp = lib()
    L, U, g = big32
    b = synth.gaussian_spinor(L, seed=2)
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=inner))
    res = oracle.true_residual(U, b, to_np(x), KAPPA, L, BC)
    assert res <= TOL and st[0]["converged"] == 1
    assert abs(st[0]["true_resid"] - res) <= 0.05 * res


def test_batch_24x48_twelve_point_sources():
    bpp = lib()
    L = (24, 24, 24, 48)
    U = synth.random_links(L, seed=1)
    g = bpp.Gauge(to_dev(U), L)
    b = np.stack([synth.point_source(L, idx) for idx in range(12)])
    x, st = bpp.solve(g, to_dev(b), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=bpp.F32))
    assert all(s["converged"] == 1 and s["true_resid"] <= TOL for s in st)
    xn = to_np(x)
    for idx in range(12):
        res = oracle.true_residual(U, b[idx], xn[idx], KAPPA, L, BC)
        assert res <= TOL, (idx, res)
        assert abs(st[idx]["true_resid"] - res) <= 0.05 * res, (idx, res, st[idx]["true_resid"])


def test_uneven_batch_six_lattices():
    bpp = lib()
    lats = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (16, 16, 16, 32), (20, 20, 20, 40), (24, 24, 24, 48)]
    kappas = synth.uniform_kappas(len(lats), seed=4)
    gs, Us, bs = [], [], []
    for i, L in enumerate(lats):
        U = synth.random_links(L, seed=1)
        gs.append(bpp.Gauge(to_dev(U), L))
        Us.append(U)
        bs.append(to_dev(synth.gaussian_spinor(L, seed=2 + i)))
    opts = bpp.solve_opts(inner_prec=bpp.F32)
    xs, st = bpp.solve_batch(gs, bs, kappas, TOL, opts)
    for i, L in enumerate(lats):
        assert st[i]["converged"] == 1
        assert oracle.true_residual(Us[i], to_np(bs[i]), to_np(xs[i]), kappas[i], L, BC) <= TOL
    for i in (0, 5):
        x1, _ = bpp.solve(gs[i], bs[i], kappas[i], 0.0, TOL, opts)
        assert torch.equal(x1, xs[i])


def test_clover_48x96_four_rhs_fp16_grad_b():
    """Wilson-clover c_SW = 1 on 48^3x96, 4 RHS, FP16-storage inner, FP64 outer to
    1e-10, with the adjoint gradient with respect to b."""
    bpp = lib()
    from paper_2111_04457_b300.autograd import solve_fn
    L = (48, 48, 48, 96)
    csw = 1.0
    U = synth.random_links(L, seed=1)
    g = bpp.Gauge(to_dev(U), L)
    g.clover_build(KAPPA, csw)
    V = oracle.volume(L)
    b = to_dev(synth.gaussian_spinor(L, seed=2, nrhs=4)).requires_grad_(True)
    x = solve_fn(None, b, L, KAPPA, csw=csw, tol=TOL, inner_prec=bpp.F16, gauge=g)
    eta = to_dev(synth.gaussian_spinor(L, seed=3, nrhs=4))
    torch.vdot(eta.reshape(-1), x.reshape(-1)).real.backward()
    lam = b.grad
    with torch.no_grad():
        for r in range(4):
            # true residual of the forward solve with the library's FP64 D (parity-tested)
            Dx = bpp.dirac_apply(g, x[r].detach(), KAPPA, csw)
            assert (torch.linalg.vector_norm(b[r] - Dx) / torch.linalg.vector_norm(b[r])).item() <= TOL
            Dl = bpp.dirac_apply(g, lam[r], KAPPA, csw, dagger=True)
            assert (torch.linalg.vector_norm(eta[r] - Dl) / torch.linalg.vector_norm(eta[r])).item() <= TOL
        # the oracle at sampled sites: D x = b and D^dag lam = eta there
        sites = _sample(V, 256, 9)
        xs = to_np(x[0].detach())
        ls = to_np(lam[0])
        Dx_o = oracle.apply_D_sites_clover(U, xs, KAPPA, L, csw, sites)
        b0 = to_np(b[0].detach())
        assert np.abs(Dx_o - b0[sites]).max() <= 1e-10 * np.linalg.norm(b0)
        Dl_o = oracle.apply_D_sites_clover(U, ls, KAPPA, L, csw, sites, dagger=True)
        e0 = to_np(eta[0])
        assert np.abs(Dl_o - e0[sites]).max() <= 1e-10 * np.linalg.norm(e0)
