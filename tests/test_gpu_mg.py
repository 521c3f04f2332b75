"""Two-level multigrid on the GPU against the oracle's definitions: the
prolongator and restriction (P c, P^dag f), R P = 1, the Galerkin coarse
operator D_c = P^dag D P (random links, antiperiodic time, Wilson and clover;
the free field against its closed form through the oracle), all in FP32 (the
preconditioner's precision) to 2e-5 relative; the multigrid-preconditioned
solve to the oracle's true residual 1e-10 and x against the oracle's solve."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import BC, KAPPA, gauge, lib, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu
TOLF = 2e-5


def _vecs(L, seed=60):
    return np.stack([synth.gaussian_spinor(L, seed=seed + k) for k in range(6)])


def _coarse_rand(n, Vc, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n, Vc, 12)) + 1j * rng.normal(size=(n, Vc, 12))).astype(np.complex64)


@pytest.fixture(scope="module")
def setup():
    bpp = lib()
    L, block = (8, 4, 4, 8), (2, 2, 2, 4)
    g, U = gauge(L)
    v = _vecs(L)
    mg = bpp.Multigrid(g, KAPPA, to_dev(v), block)
    P = oracle.mg_prolongator(v, L, block)
    return L, block, g, U, v, mg, P


def test_mg_prolong_restrict(setup):
    L, block, g, U, v, mg, P = setup
    V, Vc = oracle.volume(L), mg.Vc
    c = _coarse_rand(2, Vc, 1)
    f = to_np(mg.prolong(torch.from_numpy(c).cuda()))
    for r in range(2):
        ref = (P @ c[r].reshape(-1).astype(np.complex128)).reshape(V, 4, 3)
        assert rel_err(f[r], ref) <= TOLF
    x = synth.gaussian_spinor(L, seed=5, nrhs=2).astype(np.complex64)
    rc = to_np(mg.restrict(torch.from_numpy(x).cuda()))
    for r in range(2):
        ref = (P.conj().T @ x[r].reshape(-1).astype(np.complex128)).reshape(Vc, 12)
        assert rel_err(rc[r], ref) <= TOLF
    # R P = 1
    back = to_np(mg.restrict(mg.prolong(torch.from_numpy(c).cuda())))
    assert rel_err(back, c.astype(np.complex128)) <= TOLF


def test_mg_coarse_operator_wilson(setup):
    L, block, g, U, v, mg, P = setup
    Dc = oracle.mg_coarse_operator(U, KAPPA, L, P, BC)
    c = _coarse_rand(2, mg.Vc, 2)
    out = to_np(mg.coarse(torch.from_numpy(c).cuda()))
    for r in range(2):
        ref = (Dc @ c[r].reshape(-1).astype(np.complex128)).reshape(mg.Vc, 12)
        assert rel_err(out[r], ref) <= TOLF


def test_mg_coarse_operator_clover():
    bpp = lib()
    L, block, csw = (4, 4, 4, 8), (2, 2, 2, 4), 1.0
    g, U = gauge(L)
    g.clover_build(KAPPA, csw)
    v = _vecs(L, 70)
    mg = bpp.Multigrid(g, KAPPA, to_dev(v), block, csw=csw)
    P = oracle.mg_prolongator(v, L, block)
    Dc = oracle.mg_coarse_operator(U, KAPPA, L, P, BC, F=oracle.clover_field(U, KAPPA, csw, L))
    c = _coarse_rand(1, mg.Vc, 3)
    out = to_np(mg.coarse(torch.from_numpy(c).cuda()))
    assert rel_err(out[0], (Dc @ c[0].reshape(-1).astype(np.complex128)).reshape(mg.Vc, 12)) <= TOLF


def test_mg_coarse_free_field_closed_form():
    """Unit links, periodic, block-constant basis: the GPU coarse operator
    against the oracle's (itself pinned to the closed form)."""
    bpp = lib()
    L, block, bc = (8, 4, 4, 8), (2, 2, 2, 4), (1, 1, 1, 1)
    U = synth.unit_links(L)
    g = bpp.Gauge(to_dev(U), L, bc)
    V = oracle.volume(L)
    v = np.zeros((6, V, 4, 3), dtype=np.complex128)
    for k in range(6):
        v[k, :, k // 3, k % 3] = 1.0
        v[k, :, 2 + k // 3, k % 3] = 1.0
    mg = bpp.Multigrid(g, KAPPA, to_dev(v), block)
    P = oracle.mg_prolongator(v, L, block)
    Dc = oracle.mg_coarse_operator(U, KAPPA, L, P, bc)
    c = _coarse_rand(1, mg.Vc, 4)
    out = to_np(mg.coarse(torch.from_numpy(c).cuda()))
    assert rel_err(out[0], (Dc @ c[0].reshape(-1).astype(np.complex128)).reshape(mg.Vc, 12)) <= TOLF


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_mg_solve(csw):
    bpp = lib()
    L, block = (8, 8, 8, 8), (4, 4, 4, 4)
    g, U = gauge(L)
    F = None
    if csw:
        g.clover_build(KAPPA, csw)
        F = oracle.clover_field(U, KAPPA, csw, L)
    mg = bpp.Multigrid(g, KAPPA, to_dev(_vecs(L, 80)), block, csw=csw, refine=1)
    b = synth.gaussian_spinor(L, seed=2, nrhs=2)
    x, st = mg.solve(to_dev(b), 1e-10)
    x = to_np(x)
    print("multigrid solve stats", [(s["outer_iters"], s["inner_iters"], s["true_resid"]) for s in st])
    for r in range(2):
        res = oracle.true_residual(U, b[r], x[r], KAPPA, L, BC, F)
        assert res <= 1e-10 and st[r]["converged"] == 1
        assert abs(st[r]["true_resid"] - res) <= 0.05 * res + 1e-15
        assert rel_err(x[r], oracle.solve(U, b[r], KAPPA, L, BC, F=F, tol=1e-12)) <= 1e-7


def test_mg_solve_dagger_and_vcycle():
    bpp = lib()
    L, block = (8, 8, 8, 8), (4, 4, 4, 4)
    g, U = gauge(L)
    mg = bpp.Multigrid(g, KAPPA, to_dev(_vecs(L, 90)), block, refine=1)
    b = synth.gaussian_spinor(L, seed=3)
    x, st = mg.solve(to_dev(b), 1e-10, bpp.solve_opts(dagger=True, max_inner=200))
    r = b - oracle.apply_D(U, to_np(x), KAPPA, L, BC, dagger=True)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    # the V-cycle is a useful approximate inverse: |1 - D M| reduces a residual
    f = synth.gaussian_spinor(L, seed=4).astype(np.complex64)
    z = to_np(mg.vcycle(torch.from_numpy(f).cuda()[None]))[0]
    red = np.linalg.norm(f - oracle.apply_D(U, z, KAPPA, L, BC)) / np.linalg.norm(f)
    print("V-cycle residual reduction", red)
    assert red < 0.5


def test_mg_rejects_bad_blocks():
    bpp = lib()
    L = (8, 8, 8, 8)
    g, U = gauge(L)
    v = to_dev(_vecs(L))
    for block in ((3, 4, 4, 4), (2, 2, 2, 2), (8, 8, 4, 4)):   # not dividing, 16 sites, 1024 sites
        with pytest.raises(bpp.BppError) as e:
            bpp.Multigrid(g, KAPPA, v, block)
        assert e.value.code == -1
