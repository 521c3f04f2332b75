"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

The module draws the random fields the paper's workloads are made of (random
SU(3) gauge links, complex Gaussian sources, point sources, random gauge
transformations) and a few constructed link fields with known physics (free
field, constant abelian phases, a uniform abelian flux).  It holds none of the
fermion matrix's arithmetic: both the FP64 oracle and the CUDA library receive
these arrays as plain inputs.

Canonical layouts (complex128, lexicographic site index x1 + L1*(x2 + L2*(x3 + L3*x4))):
    links  U[mu, site, a, b]        shape (4, V, 3, 3)
    spinor psi[site, spin, colour]  shape (V, 4, 3) (or (nrhs, V, 4, 3))

The generator is splitmix64 used as a counter-based stream, with Box-Muller
normals (see gen.c); seeds follow the workload recipe: links 1, sources 2,
eta 3, kappas of the uneven batch 4, gauge transformations 5.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "gen.c")
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
        u64, i64, dbl, ptr = ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        lib.synth_normal_pairs.argtypes = [u64, u64, i64, ptr]
        lib.synth_uniforms.argtypes = [u64, u64, i64, ptr]
        lib.synth_su3_links.argtypes = [u64, i64, dbl, ptr]
        lib.synth_su3_sites.argtypes = [u64, i64, dbl, ptr]
        _lib = lib
    return _lib


def volume(L) -> int:
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def coords(L) -> np.ndarray:
    """(V, 4) integer coordinates (x1, x2, x3, x4) of every site in lexicographic order."""
    V = volume(L)
    s = np.arange(V, dtype=np.int64)
    x1 = s % L[0]
    x2 = (s // L[0]) % L[1]
    x3 = (s // (L[0] * L[1])) % L[2]
    x4 = s // (L[0] * L[1] * L[2])
    return np.stack([x1, x2, x3, x4], axis=1)


def complex_normals(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n complex numbers with Re and Im iid N(0,1) from pairs offset .. offset+n-1."""
    out = np.empty(2 * n, dtype=np.float64)
    _load().synth_normal_pairs(ctypes.c_uint64(seed), ctypes.c_uint64(offset), n,
                               out.ctypes.data)
    return out.view(np.complex128)


def random_links(L, seed: int = 1, eps: float = 0.3) -> np.ndarray:
    """Random SU(3) links U_mu(x) = exp(i*eps*H) reunitarised, shape (4, V, 3, 3)."""
    V = volume(L)
    out = np.empty((4, V, 3, 3), dtype=np.complex128)
    _load().synth_su3_links(ctypes.c_uint64(seed), V, float(eps), out.ctypes.data)
    return out


def random_gauge_transform(L, seed: int = 5, eps: float = 1.0) -> np.ndarray:
    """One random SU(3) matrix g(x) per site, shape (V, 3, 3)."""
    V = volume(L)
    out = np.empty((V, 3, 3), dtype=np.complex128)
    _load().synth_su3_sites(ctypes.c_uint64(seed), V, float(eps), out.ctypes.data)
    return out


def gaussian_spinor(L, seed: int = 2, nrhs: int | None = None, offset: int = 0) -> np.ndarray:
    """Complex Gaussian spinor field(s): shape (V, 4, 3), or (nrhs, V, 4, 3)."""
    V = volume(L)
    n = 1 if nrhs is None else nrhs
    z = complex_normals(seed, n * V * 12, offset=offset)
    return z.reshape(V, 4, 3) if nrhs is None else z.reshape(n, V, 4, 3)


def point_source(L, idx: int, site: int = 0) -> np.ndarray:
    """Local source b = delta_{x,site} e_{spin id, colour ic} with idx = ic + 3*id."""
    V = volume(L)
    b = np.zeros((V, 4, 3), dtype=np.complex128)
    b[site, idx // 3, idx % 3] = 1.0
    return b


def uniforms(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in (0,1] from counters offset .. offset+n-1."""
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniforms(ctypes.c_uint64(seed), ctypes.c_uint64(offset), n, out.ctypes.data)
    return out


def uniform_kappas(n: int, seed: int = 4, lo: float = 0.10, hi: float = 0.12) -> np.ndarray:
    """n hopping parameters drawn uniformly in [lo, hi]."""
    return lo + (hi - lo) * uniforms(seed, n)


def unit_links(L) -> np.ndarray:
    """Free field U_mu(x) = 1."""
    V = volume(L)
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1.0
    return U


def constant_diagonal_links(L, phases) -> np.ndarray:
    """U_mu(x) = diag(exp(i*phases[mu, c])) on every site; phases has shape (4, 3)."""
    V = volume(L)
    ph = np.asarray(phases, dtype=np.float64)
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)
    for mu in range(4):
        for c in range(3):
            U[mu, :, c, c] = np.exp(1j * ph[mu, c])
    return U


def abelian_flux_links(L, n_flux: int = 1) -> np.ndarray:
    """Uniform abelian flux in the (1,2) plane: every 12-plaquette equals exp(i*theta),
    theta = 2*pi*n_flux/(L1*L2), with the 't Hooft twist on the x1 = L1-1 links.
    U_2(x) = exp(i*theta*x1); U_1(x) = 1 except U_1(L1-1, x2, ...) = exp(-i*theta*L1*x2);
    U_3 = U_4 = 1.  Colour structure is the identity."""
    V = volume(L)
    x = coords(L)
    theta = 2.0 * np.pi * n_flux / (L[0] * L[1])
    ph1 = np.where(x[:, 0] == L[0] - 1, -theta * L[0] * x[:, 1], 0.0)
    ph2 = theta * x[:, 0]
    U = unit_links(L)
    for c in range(3):
        U[0, :, c, c] = np.exp(1j * ph1)
        U[1, :, c, c] = np.exp(1j * ph2)
    return U
