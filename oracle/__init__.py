"""FP64 CPU ORACLE -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct restatement of what the CUDA library computes,
written from the paper "General purpose lattice QCD code set Bridge++ 2.0 for
high performance computing" (arXiv:2111.04457).  Only tests/, the smoke check
and the benchmark's CPU-baseline leg may import it; the CUDA library never
does, and the two share no code.  The operator application lives in dirac.c
(plain loops); the algorithms on top of it (even-odd Schur complement,
BiCGStab, CGNR, dense assembly, DFT inverse of the free field, the projected
force) are plain numpy here, each step in the order its definition gives.

Conventions (readings of points the paper leaves open):
  * gamma matrices: Euclidean, Hermitian, chiral basis
      gamma_k = [[0, i sigma_k], [-i sigma_k, 0]] (k = 1,2,3),
      gamma_4 = [[0, 1], [1, 0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4.
  * directions mu = 0..3 are x1..x4 (x, y, z, t); site index
    x1 + L1*(x2 + L2*(x3 + L3*x4)); parity (x1+x2+x3+x4) mod 2, even = 0.
  * boundary: a hop across the boundary in direction mu is multiplied by
    bc[mu]; the workloads use bc = (1, 1, 1, -1) (antiperiodic in time).
  * clover term: F = i kappa c_SW sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu},
    sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], Fhat = (Q - Q^dag)/8.
  * even-odd: Mhat = D_ee - D_eo D_oo^{-1} D_oe on the even sites.
  * gradient: L = Re<eta, x>, x = D^{-1} b; grad_b = D^{-dag} eta,
    grad_U = kappa * bc * M^dag (dirac.c), projected force
    P = (i/2)(U G^dag - G U^dag) minus its trace, so that for U -> exp(i eps T) U
    with T Hermitian traceless, dL/deps = tr(T P).

Parity pinning: every function here is checked in tests/test_oracle_*.py
against closed forms, invariants and brute force (free-field spectrum and
plane waves, constant abelian phases, gamma5-hermiticity, gauge covariance,
dense LU on 2^4, DFT inverse of the free field, uniform abelian flux for the
clover normalisation, central finite differences for the gradient).  The sign
convention of the clover term is pinned only by invariants and by the
abelian-flux spectrum, which is symmetric under the sign: parity unpinned for
that sign.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

# ---------------------------------------------------------------------------
# gamma matrices (chiral basis)
_s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_z2 = np.zeros((2, 2), dtype=np.complex128)
_i2 = np.eye(2, dtype=np.complex128)


def _chiral(a):
    return np.block([[_z2, a], [a.conj().T, _z2]])


GAMMA = np.stack([_chiral(1j * _s1), _chiral(1j * _s2), _chiral(1j * _s3), _chiral(_i2)])
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
DEFAULT_BC = (1, 1, 1, -1)


# ---------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile dirac.c into liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "dirac.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        p, d, i, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
        lib.oracle_dirac_apply.argtypes = [p, p, p, p, p, d, i, p, p, i64, p]
        lib.oracle_clover_field.argtypes = [p, p, p, d, d, p]
        lib.oracle_clover_field_sites.argtypes = [p, p, p, d, d, p, i64, p]
        lib.oracle_clover_leaf.argtypes = [p, p, i, i, i64, p]
        lib.oracle_link_gradient.argtypes = [p, p, p, p, p, d, p]
        lib.oracle_clover_gradient.argtypes = [p, p, p, p, p, d, d, p]
        _lib = lib
    return _lib


def _ivec(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def volume(L) -> int:
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


# ---------------------------------------------------------------------------
# Eq. (1)
def apply_D(U, psi, kappa, L, bc=DEFAULT_BC, F=None, dagger=False, sites=None):
    """D psi (or D^dag psi) by Eq. (1); psi (V,4,3); F (V,12,12) or None (Wilson).
    With sites given, returns D psi at those sites only, shape (len(sites),4,3)."""
    lib = _load()
    Lv, bv = _ivec(L), _ivec(bc)
    U, psi = _c128(U), _c128(psi)
    Fp = None if F is None else _c128(F)
    if sites is None:
        out = np.empty((volume(L), 4, 3), dtype=np.complex128)
        lib.oracle_dirac_apply(Lv.ctypes.data, bv.ctypes.data, GAMMA.ctypes.data, U.ctypes.data,
                               None if Fp is None else Fp.ctypes.data, float(kappa), int(dagger),
                               psi.ctypes.data, out.ctypes.data, 0, None)
    else:
        sv = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
        out = np.empty((len(sv), 4, 3), dtype=np.complex128)
        lib.oracle_dirac_apply(Lv.ctypes.data, bv.ctypes.data, GAMMA.ctypes.data, U.ctypes.data,
                               None if Fp is None else Fp.ctypes.data, float(kappa), int(dagger),
                               psi.ctypes.data, out.ctypes.data, len(sv), sv.ctypes.data)
    return out


def clover_leaf(U, L, mu, nu, site):
    """Q_{mu nu}(x): the sum of the four same-orientation plaquettes at x."""
    Q = np.empty((3, 3), dtype=np.complex128)
    U, Lv = _c128(U), _ivec(L)
    _load().oracle_clover_leaf(Lv.ctypes.data, U.ctypes.data, mu, nu, site, Q.ctypes.data)
    return Q


def clover_field(U, kappa, csw, L):
    """F(x), the 12x12 Hermitian clover term per site, shape (V,12,12)."""
    F = np.empty((volume(L), 12, 12), dtype=np.complex128)
    U, Lv = _c128(U), _ivec(L)
    _load().oracle_clover_field(Lv.ctypes.data, GAMMA.ctypes.data, U.ctypes.data,
                                float(kappa), float(csw), F.ctypes.data)
    return F


def clover_field_sites(U, kappa, csw, L, sites):
    """F(x) at the listed sites only, shape (len(sites),12,12)."""
    sv = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    F = np.empty((len(sv), 12, 12), dtype=np.complex128)
    U, Lv = _c128(U), _ivec(L)
    _load().oracle_clover_field_sites(Lv.ctypes.data, GAMMA.ctypes.data, U.ctypes.data, float(kappa), float(csw),
                                      F.ctypes.data, len(sv), sv.ctypes.data)
    return F


def apply_D_sites_clover(U, psi, kappa, L, csw, sites, bc=DEFAULT_BC, dagger=False):
    """D psi (or D^dag psi) with the clover term at the listed sites only: the
    hopping part from Eq. (1) plus F(x) psi(x) with F built at those sites."""
    sv = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = apply_D(U, psi, kappa, L, bc, None, dagger, sites=sv)
    if csw != 0.0:
        F = clover_field_sites(U, kappa, csw, L, sv)
        out = out + np.einsum("nij,nj->ni", F, psi[sv].reshape(len(sv), 12)).reshape(out.shape)
    return out


def link_gradient(x, lam, kappa, L, bc=DEFAULT_BC, U=None, csw=0.0):
    """Unconstrained grad_U of L = Re<eta, D^{-1} b> given x and lam = D^{-dag} eta:
    the hopping term's part, plus the clover term's part when csw != 0 (needs U)."""
    G = np.empty((4, volume(L), 3, 3), dtype=np.complex128)
    x, lam, Lv, bv = _c128(x), _c128(lam), _ivec(L), _ivec(bc)
    _load().oracle_link_gradient(Lv.ctypes.data, bv.ctypes.data, GAMMA.ctypes.data,
                                 x.ctypes.data, lam.ctypes.data, float(kappa), G.ctypes.data)
    if csw != 0.0:
        Uc = _c128(U)
        _load().oracle_clover_gradient(Lv.ctypes.data, GAMMA.ctypes.data, Uc.ctypes.data, x.ctypes.data,
                                       lam.ctypes.data, float(kappa), float(csw), G.ctypes.data)
    return G


def projected_force(U, G):
    """P_mu(x) = (i/2)(U G^dag - G U^dag) minus trace/3: dL/deps = tr(T P) for U -> e^{i eps T} U."""
    Gd = np.conj(np.swapaxes(G, -1, -2))
    Ud = np.conj(np.swapaxes(U, -1, -2))
    Z = 0.5j * (U @ Gd - G @ Ud)
    tr = np.trace(Z, axis1=-2, axis2=-1) / 3.0
    return Z - tr[..., None, None] * np.eye(3)


# ---------------------------------------------------------------------------
# lattice bookkeeping
def coords(L):
    V = volume(L)
    s = np.arange(V, dtype=np.int64)
    return np.stack([s % L[0], (s // L[0]) % L[1], (s // (L[0] * L[1])) % L[2],
                     s // (L[0] * L[1] * L[2])], axis=1)


def parity(L):
    """(x1+x2+x3+x4) mod 2 of every site, in lexicographic order."""
    return coords(L).sum(axis=1) % 2


def parity_sites(L, p):
    """Lexicographic indices of the sites of parity p, in lexicographic order
    (this is the even-odd ordering of half-volume fields)."""
    return np.nonzero(parity(L) == p)[0]


def embed(L, half, p):
    """Full-lattice field that equals `half` on parity p and 0 elsewhere."""
    out = np.zeros((volume(L),) + half.shape[1:], dtype=np.complex128)
    out[parity_sites(L, p)] = half
    return out


def hop_eo(U, psi_half, kappa, L, p, bc=DEFAULT_BC):
    """-kappa H_{p,pbar} psi_pbar: the hopping term of Eq. (1) from the sites of
    parity 1-p to the sites of parity p (the diagonal term vanishes there)."""
    full = embed(L, psi_half, 1 - p)
    return apply_D(U, full, kappa, L, bc)[parity_sites(L, p)]


def clover_blocks(F, L, p):
    """A_pp = 1 + F on the sites of parity p, shape (Vh,12,12)."""
    return np.eye(12) + F[parity_sites(L, p)]


def apply_site_matrix(A, v):
    """Per-site 12x12 matrix on a (n,4,3) field."""
    return np.einsum("nij,nj->ni", A, v.reshape(len(v), 12)).reshape(v.shape)


class Schur:
    """Mhat = D_ee - D_eo D_oo^{-1} D_oe on the even sites, with D_oo^{-1}
    from a per-site 12x12 inverse of the odd diagonal block."""

    def __init__(self, U, kappa, L, bc=DEFAULT_BC, F=None):
        self.U, self.kappa, self.L, self.bc, self.F = U, kappa, tuple(L), tuple(bc), F
        self.even = parity_sites(L, 0)
        self.odd = parity_sites(L, 1)
        if F is None:
            self.Doo_inv = None
        else:
            self.Doo_inv = np.linalg.inv(clover_blocks(F, L, 1))

    def D(self, v, dagger=False):
        return apply_D(self.U, v, self.kappa, self.L, self.bc, self.F, dagger)

    def Doo_inverse(self, v_odd, dagger=False):
        if self.Doo_inv is None:
            return v_odd.copy()
        A = np.conj(np.swapaxes(self.Doo_inv, -1, -2)) if dagger else self.Doo_inv
        return apply_site_matrix(A, v_odd)

    def apply(self, x_e, dagger=False):
        y = self.D(embed(self.L, x_e, 0), dagger)           # y_e = D_ee x_e, y_o = D_oe x_e
        z_o = self.Doo_inverse(y[self.odd], dagger)
        w = self.D(embed(self.L, z_o, 1), dagger)           # w_e = D_eo z_o
        return y[self.even] - w[self.even]

    def prepare(self, b):
        """bhat_e = b_e - D_eo D_oo^{-1} b_o."""
        z_o = self.Doo_inverse(b[self.odd])
        w = self.D(embed(self.L, z_o, 1))
        return b[self.even] - w[self.even]

    def reconstruct(self, x_e, b):
        """x_o = D_oo^{-1} (b_o - D_oe x_e); returns the full-lattice x."""
        y = self.D(embed(self.L, x_e, 0))
        x_o = self.Doo_inverse(b[self.odd] - y[self.odd])
        x = np.zeros((volume(self.L), 4, 3), dtype=np.complex128)
        x[self.even] = x_e
        x[self.odd] = x_o
        return x


# ---------------------------------------------------------------------------
# Krylov solvers (plain textbook forms, complex inner product <a,b> = sum conj(a) b)
def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _norm(a):
    return np.sqrt(np.vdot(a.ravel(), a.ravel()).real)


def bicgstab(op, b, tol=1e-12, maxiter=10000, x0=None):
    """BiCGStab (van der Vorst 1992) for op(x) = b; stops when ||b - op x|| / ||b|| <= tol
    (recursive residual, confirmed with the true residual).  Returns (x, iterations)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - op(x) if x0 is not None else b.copy()
    bnorm = _norm(b)
    if bnorm == 0.0:
        return x, 0
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxiter + 1):
        rho = _dot(rhat, r)
        if abs(rho) < 1e-300:
            rhat = r.copy()
            rho = _dot(rhat, r)
            p = np.zeros_like(b)
            v = np.zeros_like(b)
            rho_old = alpha = omega = 1.0 + 0j
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = op(p)
        alpha = rho / _dot(rhat, v)
        s = r - alpha * v
        t = op(s)
        tt = _dot(t, t).real
        omega = _dot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        if _norm(r) <= tol * bnorm:
            rt = b - op(x)
            if _norm(rt) <= tol * bnorm:
                return x, it
            r = rt
    raise RuntimeError("oracle BiCGStab did not converge")


def cg(op, b, tol=1e-12, maxiter=20000, x0=None):
    """Conjugate gradient (Hestenes-Stiefel) for a Hermitian positive-definite op."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - op(x) if x0 is not None else b.copy()
    bnorm = _norm(b)
    if bnorm == 0.0:
        return x, 0
    p = r.copy()
    rr = _dot(r, r).real
    for it in range(1, maxiter + 1):
        q = op(p)
        alpha = rr / _dot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = _dot(r, r).real
        if np.sqrt(rr_new) <= tol * bnorm:
            return x, it
        p = r + (rr_new / rr) * p
        rr = rr_new
    raise RuntimeError("oracle CG did not converge")


def cgnr(op, op_dag, b, tol=1e-12, maxiter=20000):
    """CGNR (CG on the normal equations op^dag op x = op^dag b), stopping when the
    residual of the original system, ||b - op x|| / ||b||, reaches tol."""
    x = np.zeros_like(b)
    r = b.copy()
    z = op_dag(r)
    p = z.copy()
    zz = _dot(z, z).real
    bnorm = _norm(b)
    if bnorm == 0.0:
        return x, 0
    for it in range(1, maxiter + 1):
        w = op(p)
        alpha = zz / _dot(w, w).real
        x = x + alpha * p
        r = r - alpha * w
        if _norm(r) <= tol * bnorm:
            return x, it
        z = op_dag(r)
        zz_new = _dot(z, z).real
        p = z + (zz_new / zz) * p
        zz = zz_new
    raise RuntimeError("oracle CGNR did not converge")


def gamma5(psi):
    """gamma_5 psi on a (..., 4, 3) field."""
    return np.einsum("st,...tc->...sc", GAMMA5, psi)


def solve(U, b, kappa, L, bc=DEFAULT_BC, F=None, tol=1e-12, method="bicgstab", dagger=False):
    """x = D^{-1} b (or D^{-dag} b) through the even-odd Schur complement.
    D^dag is applied through gamma5-hermiticity: D^{-dag} b = g5 D^{-1} g5 b."""
    if dagger:
        return gamma5(solve(U, gamma5(b), kappa, L, bc, F, tol, method, dagger=False))
    S = Schur(U, kappa, L, bc, F)
    bhat = S.prepare(b)
    bn = _norm(b)
    # the full residual equals the Schur residual on the even sites (odd part is exact)
    stol = tol * bn / max(_norm(bhat), 1e-300)
    if method == "bicgstab":
        xe, _ = bicgstab(S.apply, bhat, tol=stol)
    elif method == "cgnr":
        xe, _ = cgnr(S.apply, lambda v: S.apply(v, dagger=True), bhat, tol=stol)
    else:
        raise ValueError(method)
    return S.reconstruct(xe, b)


def true_residual(U, b, x, kappa, L, bc=DEFAULT_BC, F=None):
    """||b - D x|| / ||b|| with the full FP64 D of Eq. (1)."""
    r = b - apply_D(U, x, kappa, L, bc, F)
    return _norm(r) / _norm(b)


# ---------------------------------------------------------------------------
# brute force and closed forms
def dense_D(U, kappa, L, bc=DEFAULT_BC, F=None):
    """The (12V x 12V) matrix of Eq. (1), assembled column by column."""
    n = 12 * volume(L)
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        M[:, j] = apply_D(U, e.reshape(-1, 4, 3), kappa, L, bc, F).ravel()
    return M


def momenta(L, bc=DEFAULT_BC):
    """Allowed momenta per direction: p = (2 pi n + theta)/L with theta = 0 (periodic)
    or pi (antiperiodic)."""
    out = []
    for mu in range(4):
        theta = 0.0 if bc[mu] == 1 else np.pi
        out.append((2.0 * np.pi * np.arange(L[mu]) + theta) / L[mu])
    return out


def free_field_eigenvalues(L, kappa, bc=DEFAULT_BC):
    """Closed-form spectrum of D at U = 1, F = 0: for every momentum,
    1 - 2 kappa sum cos p +- 2 i kappa sqrt(sum sin^2 p), each twice (spin) times 3 (colour)."""
    ps = momenta(L, bc)
    P = np.meshgrid(*ps, indexing="ij")
    c = sum(np.cos(p) for p in P).ravel()
    s = np.sqrt(sum(np.sin(p) ** 2 for p in P)).ravel()
    lam = np.concatenate([1 - 2 * kappa * c + 2j * kappa * s, 1 - 2 * kappa * c - 2j * kappa * s])
    return np.repeat(lam, 6)


def free_field_Dp(p, kappa):
    """D(p) = 1 - 2 kappa sum cos p_mu + 2 i kappa sum gamma_mu sin p_mu (4x4, colour-blind)."""
    return ((1 - 2 * kappa * np.sum(np.cos(p))) * np.eye(4)
            + 2j * kappa * np.einsum("m,mst->st", np.sin(p), GAMMA))


def free_field_solve_dft(b, kappa, L, bc=DEFAULT_BC):
    """x = D^{-1} b at U = 1 by a plain discrete Fourier transform written out as
    one explicit DFT matrix per axis (no FFT library)."""
    ps = momenta(L, bc)
    xs = [np.arange(L[mu]) for mu in range(4)]
    E = [np.exp(-1j * np.outer(ps[mu], xs[mu])) for mu in range(4)]    # E[mu][n, x]
    # b indexed [x4, x3, x2, x1, spin, colour]
    bt = b.reshape(L[3], L[2], L[1], L[0], 4, 3)
    bt = np.einsum("ax,xyzwsc->ayzwsc", E[3], bt)
    bt = np.einsum("ay,xyzwsc->xazwsc", E[2], bt)
    bt = np.einsum("az,xyzwsc->xyawsc", E[1], bt)
    bt = np.einsum("aw,xyzwsc->xyzasc", E[0], bt)
    out = np.empty_like(bt)
    for n4 in range(L[3]):
        for n3 in range(L[2]):
            for n2 in range(L[1]):
                for n1 in range(L[0]):
                    p = np.array([ps[0][n1], ps[1][n2], ps[2][n3], ps[3][n4]])
                    out[n4, n3, n2, n1] = np.linalg.solve(free_field_Dp(p, kappa), bt[n4, n3, n2, n1])
    Ei = [np.conj(e).T / L[mu] for mu, e in enumerate(E)]              # Ei[mu][x, n]
    out = np.einsum("xa,ayzwsc->xyzwsc", Ei[3], out)
    out = np.einsum("ya,xazwsc->xyzwsc", Ei[2], out)
    out = np.einsum("za,xyawsc->xyzwsc", Ei[1], out)
    out = np.einsum("wa,xyzasc->xyzwsc", Ei[0], out)
    return out.reshape(volume(L), 4, 3)


# ---------------------------------------------------------------------------
# Two-level aggregation multigrid (the multi-grid solver named in Sec. 1 and
# Sec. 4; the paper gives no construction, the reading is the standard
# aggregation with chirality-split blocks): the prolongator and the Galerkin
# coarse operator, by their definitions, as dense matrices (small lattices).
def mg_block_index(L, block):
    """Block index of every lexicographic site, b0 + Lc0 (b1 + Lc1 (b2 + Lc2 b3)),
    and the block-lattice extents Lc."""
    Lc = [L[m] // block[m] for m in range(4)]
    b = coords(L) // np.asarray(block)
    return b[:, 0] + Lc[0] * (b[:, 1] + Lc[1] * (b[:, 2] + Lc[2] * b[:, 3])), Lc


def mg_prolongator(vecs, L, block):
    """P as a dense (12 V) x (12 Vc) matrix.  Column (B, 6 chi + k) is the k-th
    vector of the Gram-Schmidt orthonormalisation, in the order k = 0..5, of the
    six vectors vecs[k] restricted to block B and chirality chi (spins 2 chi,
    2 chi + 1).  Gram-Schmidt in order is the QR factorisation whose R has a
    positive real diagonal."""
    vecs = np.asarray(vecs)
    V = volume(L)
    bidx, Lc = mg_block_index(L, block)
    Vc = int(np.prod(Lc))
    P = np.zeros((V, 4, 3, Vc, 12), dtype=np.complex128)
    for B in range(Vc):
        sites = np.flatnonzero(bidx == B)
        for chi in range(2):
            A = vecs[:, sites][:, :, 2 * chi:2 * chi + 2, :].reshape(6, -1).T
            Q, R = np.linalg.qr(A)
            d = np.diag(R)
            Q = Q * (d / np.abs(d))[None, :]
            P[sites, 2 * chi:2 * chi + 2, :, B, 6 * chi:6 * chi + 6] = Q.reshape(len(sites), 2, 3, 6)
    return P.reshape(V * 12, Vc * 12)


def mg_coarse_operator(U, kappa, L, P, bc=DEFAULT_BC, F=None):
    """D_c = P^dag D P with D of Eq. (1) applied to every column of P."""
    V = volume(L)
    DP = np.empty_like(P)
    for j in range(P.shape[1]):
        DP[:, j] = apply_D(U, P[:, j].reshape(V, 4, 3), kappa, L, bc, F).reshape(-1)
    return P.conj().T @ DP
