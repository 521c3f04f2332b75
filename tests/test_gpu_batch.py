"""Batching (the 12 spin-colour sources of a propagator, Fig. 1; lattices of
uneven sizes) and the graph-captured inner loop.  A system's result does not
depend on the batch it runs in, nor on graph versus eager execution: the
kernels, block-to-site maps of each system and reduction orders are the same,
so results must be bit-identical."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, gauge, lib, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_graph_equals_eager(solver, csw):
    """Host-driven loops, the inner-loop graph and the whole-solve graph (first
    call host-driven, then replayed) give bit-identical results."""
    bpp = lib()
    L = (6, 6, 6, 10)
    g, U = gauge(L)
    if csw:
        g.clover_build(0.12, csw)
    b = to_dev(synth.gaussian_spinor(L, seed=2))
    for inner in [bpp.F32, bpp.F16, bpp.F64]:
        xe, se = bpp.solve(g, b, 0.12, csw, TOL, bpp.solve_opts(solver=solver, inner_prec=inner, use_graph=0))
        for mode in (1, 2, 2, 2):
            xg, sg = bpp.solve(g, b, 0.12, csw, TOL, bpp.solve_opts(solver=solver, inner_prec=inner, use_graph=mode))
            assert torch.equal(xe, xg), (inner, mode)
            assert se[0]["inner_iters"] == sg[0]["inner_iters"]
            assert se[0]["outer_iters"] == sg[0]["outer_iters"]
            assert sg[0]["converged"] == 1


def test_uneven_batch_matches_single():
    bpp = lib()
    lats = [(4, 4, 4, 4), (6, 6, 6, 6), (4, 4, 4, 8), (8, 4, 4, 6)]
    kappas = synth.uniform_kappas(len(lats))
    gs, Us, bs = [], [], []
    for i, L in enumerate(lats):
        g, U = gauge(L, seed=1 + i)
        gs.append(g)
        Us.append(U)
        bs.append(to_dev(synth.gaussian_spinor(L, seed=2 + i)))
    for inner, mode in [(bpp.F32, 1), (bpp.F16, 1), (bpp.F32, 2), (bpp.F16, 2)]:
        opts = bpp.solve_opts(inner_prec=inner, use_graph=mode)
        bpp.solve_batch(gs, bs, kappas, TOL, opts)          # first call of a configuration: host-driven
        xs, st = bpp.solve_batch(gs, bs, kappas, TOL, opts)
        for i, L in enumerate(lats):
            x1, s1 = bpp.solve(gs[i], bs[i], kappas[i], 0.0, TOL, opts)
            assert torch.equal(xs[i], x1), (L, inner)
            assert st[i]["inner_iters"] == s1[0]["inner_iters"]
            res = oracle.true_residual(Us[i], to_np(bs[i]), to_np(xs[i]), kappas[i], L, BC)
            assert res <= TOL


@pytest.mark.parametrize("L", [(4, 4, 4, 8), (8, 8, 8, 16)])
def test_twelve_sources_match_single(L):
    """Each source of a 12-source batch gives the same bits as its own solve
    (the vector kernels' partition depends on the lattice, not on the number
    of right-hand sides; at 8^3x16 the batch holds 12 x 4096 sites)."""
    bpp = lib()
    g, U = gauge(L)
    b = np.stack([synth.point_source(L, idx) for idx in range(12)])
    opts = bpp.solve_opts(inner_prec=bpp.F32)
    x, st = bpp.solve(g, to_dev(b), 0.12, 0.0, TOL, opts)
    for idx in [0, 5, 11]:
        x1, _ = bpp.solve(g, to_dev(b[idx]), 0.12, 0.0, TOL, opts)
        assert torch.equal(x[idx], x1[0] if x1.dim() == 4 else x1)


def test_launch_count_grows():
    bpp = lib()
    L = (4, 4, 4, 4)
    g, U = gauge(L)
    b = to_dev(synth.gaussian_spinor(L, seed=2))
    bpp.launch_count(reset=True)
    bpp.solve(g, b, 0.12, 0.0, TOL)
    n = bpp.launch_count()
    assert n > 10


def test_clover_batch_uneven():
    """Wilson-clover lattices of different sizes and kappas in one batched solve."""
    bpp = lib()
    lats = [(4, 4, 4, 4), (6, 4, 4, 8), (4, 6, 6, 6)]
    kappas = synth.uniform_kappas(len(lats))
    csw = 1.0
    gs, Us, bs, Fs = [], [], [], []
    for i, L in enumerate(lats):
        g, U = gauge(L, seed=3 + i)
        g.clover_build(kappas[i], csw)
        gs.append(g)
        Us.append(U)
        Fs.append(oracle.clover_field(U, kappas[i], csw, L))
        bs.append(to_dev(synth.gaussian_spinor(L, seed=7 + i)))
    for inner in (bpp.F32, bpp.F16):
        xs, st = bpp.solve_batch(gs, bs, kappas, TOL, bpp.solve_opts(inner_prec=inner), csw=csw)
        for i, L in enumerate(lats):
            assert oracle.true_residual(Us[i], to_np(bs[i]), to_np(xs[i]), kappas[i], L, BC, Fs[i]) <= TOL


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (6, 6, 6, 10), (8, 8, 8, 8)])
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_fused_inner_products_match_separate(L, csw, monkeypatch):
    """BiCGStab's <rhat, v>, <t, s> and ||t||^2 formed by the second hop of
    each Schur application (the default; per-warp sums, partial warps on
    these lattices: Vh = 8, 1080, 2048) and by separate vector kernels
    (BPP_FUSED_DOTS=0, read when a solve plan is built) group the same terms
    differently: both solves meet the tolerance by the oracle's residual, in
    every inner precision, and their solutions agree to the solve's accuracy."""
    bpp = lib()
    b_np = synth.gaussian_spinor(L, seed=2)
    F = oracle.clover_field(synth.random_links(L, seed=1), 0.12, csw, L) if csw else None
    xs = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("BPP_FUSED_DOTS", fused)
        g, U = gauge(L)          # a new gauge handle: new plans under this setting
        if csw:
            g.clover_build(0.12, csw)
        b = to_dev(b_np)
        for inner in (bpp.F64, bpp.F32, bpp.F16):
            x, st = bpp.solve(g, b, 0.12, csw, TOL, bpp.solve_opts(inner_prec=inner))
            assert st[0]["converged"] == 1
            xn = to_np(x)
            res = oracle.true_residual(U, b_np, xn, 0.12, L, BC, F)
            assert res <= TOL, (fused, inner, res)
            xs[(fused, inner)] = xn
        del g
    for inner in (bpp.F64, bpp.F32, bpp.F16):
        a, c = xs[("1", inner)], xs[("0", inner)]
        assert np.linalg.norm(a - c) / np.linalg.norm(c) <= 1e-8, inner
