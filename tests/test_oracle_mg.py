"""Pins of the oracle's multigrid construction (prolongator P and Galerkin
coarse operator D_c = P^dag D P): P has orthonormal columns, reproduces every
near-null vector (P P^dag v_k = v_k), and for the free field with constant
near-null vectors D_c equals its closed form: inside a block every hop pair
contributes 2 (the gamma parts of the forward and backward hops cancel), across
a block face in direction mu the coupling is -(kappa / b_mu)(1 -+ gamma_mu)
restricted to the basis spinors."""
import numpy as np

import oracle
import synth

KAPPA = 0.12


def _gauss_vecs(L, seed):
    return np.stack([synth.gaussian_spinor(L, seed=seed + k) for k in range(6)])


def test_prolongator_orthonormal_and_reproduces_vectors():
    L, block = (4, 4, 4, 8), (2, 2, 2, 4)
    v = _gauss_vecs(L, 40)
    P = oracle.mg_prolongator(v, L, block)
    assert np.abs(P.conj().T @ P - np.eye(P.shape[1])).max() < 1e-13
    for k in range(6):
        vk = v[k].reshape(-1)
        assert np.linalg.norm(P @ (P.conj().T @ vk) - vk) <= 1e-12 * np.linalg.norm(vk)
    # Gram-Schmidt order: the first column of each aggregate is the first vector normalised there
    bidx, _ = oracle.mg_block_index(L, block)
    s0 = np.flatnonzero(bidx == 3)
    seg = v[0][s0][:, 2:4, :].reshape(-1)
    col = P.reshape(oracle.volume(L), 4, 3, -1)[s0][:, 2:4, :, 3 * 12 + 6].reshape(-1)
    assert np.abs(col - seg / np.linalg.norm(seg)).max() < 1e-13


def _free_coarse_closed_form(L, block, kappa):
    """D_c of the free field (periodic) with block-constant basis spinors
    e_(chi, k) = spin 2 chi + k // 3, colour k % 3."""
    Lc = [L[m] // block[m] for m in range(4)]
    Vc = int(np.prod(Lc))
    g = oracle.GAMMA
    # basis index i = 6 chi + k -> spin-colour (2 chi + k // 3, k % 3)
    spin = np.array([2 * (i // 6) + (i % 6) // 3 for i in range(12)])
    col = np.array([i % 6 % 3 for i in range(12)])
    same_col = (col[:, None] == col[None, :]).astype(float)

    def gam(mu):
        return g[mu][spin[:, None], spin[None, :]] * same_col

    Dc = np.zeros((Vc, 12, Vc, 12), dtype=np.complex128)
    bc_coords = np.stack(np.meshgrid(*[np.arange(n) for n in Lc], indexing="ij"), axis=-1).reshape(-1, 4)
    idx = lambda b: b[0] + Lc[0] * (b[1] + Lc[1] * (b[2] + Lc[2] * b[3]))
    bv = int(np.prod(block))
    for b in bc_coords:
        B = idx(b)
        Dc[B, :, B, :] += np.eye(12)
        for mu in range(4):
            inner = bv * (block[mu] - 1) / block[mu] if Lc[mu] > 1 else bv   # hops that stay in the block
            if Lc[mu] == 1:
                Dc[B, :, B, :] += -kappa * (inner / bv) * 2 * np.eye(12)
                continue
            Dc[B, :, B, :] += -kappa * (inner / bv) * 2 * np.eye(12)
            face = 1.0 / block[mu]                                         # face sites / bv
            bf, bb = b.copy(), b.copy()
            bf[mu] = (b[mu] + 1) % Lc[mu]
            bb[mu] = (b[mu] - 1) % Lc[mu]
            Dc[B, :, idx(bf), :] += -kappa * face * (np.eye(12) - gam(mu))
            Dc[B, :, idx(bb), :] += -kappa * face * (np.eye(12) + gam(mu))
    return Dc.reshape(Vc * 12, Vc * 12)


def test_coarse_operator_free_field_closed_form():
    L, block = (8, 4, 4, 8), (2, 2, 2, 4)
    bc = (1, 1, 1, 1)
    U = synth.unit_links(L)
    V = oracle.volume(L)
    v = np.zeros((6, V, 4, 3), dtype=np.complex128)
    for k in range(6):
        v[k, :, k // 3, k % 3] = 1.0
        v[k, :, 2 + k // 3, k % 3] = 1.0
    P = oracle.mg_prolongator(v, L, block)
    Dc = oracle.mg_coarse_operator(U, KAPPA, L, P, bc)
    ref = _free_coarse_closed_form(L, block, KAPPA)
    assert np.abs(Dc - ref).max() < 1e-13


def test_coarse_operator_is_the_galerkin_product():
    """Random links: <P a, D P b> = <a, D_c b> for random coarse a, b, with D
    applied by the oracle's D directly on the prolongated field."""
    L, block = (4, 4, 4, 8), (2, 2, 2, 4)
    U = synth.random_links(L, seed=1)
    P = oracle.mg_prolongator(_gauss_vecs(L, 50), L, block)
    Dc = oracle.mg_coarse_operator(U, KAPPA, L, P)
    rng = np.random.default_rng(3)
    a = rng.normal(size=P.shape[1]) + 1j * rng.normal(size=P.shape[1])
    b = rng.normal(size=P.shape[1]) + 1j * rng.normal(size=P.shape[1])
    lhs = np.vdot(P @ a, oracle.apply_D(U, (P @ b).reshape(-1, 4, 3), KAPPA, L).reshape(-1))
    assert abs(lhs - np.vdot(a, Dc @ b)) < 1e-12 * abs(lhs)
