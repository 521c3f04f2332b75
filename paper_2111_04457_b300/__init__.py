"""B300 Wilson / Wilson-clover fermion matrix and solver (arXiv:2111.04457, Eq. 1).

Thin Python binding over the C ABI in include/bpp.h (libbpp.so): argument
marshalling only.  Every step of the computation runs in the library's CUDA
kernels; PyTorch supplies device memory and streams.  There is no CPU path:
importing this module fails loudly when libbpp.so is missing, and every call
needs CUDA tensors (the solve also accepts host tensors, copied inside the
call).

Canonical layouts (see include/bpp.h): spinors complex [nrhs][V][4][3] (half
fields [nrhs][Vh][4][3], sites of one parity in lexicographic order), links
complex128 [4][V][3][3], lexicographic site index x1 + L1*(x2 + L2*(x3 + L3*x4)).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libbpp.so")

if not os.path.exists(_SO):
    raise ImportError(f"libbpp.so not found at {_SO}: build it with "
                      "`python paper_2111_04457_b300/build.py` (nvcc, sm_103a)")

_lib = ctypes.CDLL(_SO)

F64, F32, F16, F64DF = 0, 1, 2, 3
LEX_D, LEX_DDAG, LEX_DDAGD = 0, 1, 2
EVEN, ODD, FULL = 0, 1, 2
BICGSTAB, CGNR = 0, 1
_ERR = {0: "OK", -1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "CUDA", -4: "OOM", -5: "NOT_CONVERGED",
        -6: "NONFINITE", -7: "TIMEOUT"}


class BppError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR.get(code, code)}: {msg}")
        self.code = code


class NotConverged(BppError):
    pass


class _Lattice(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("bc", ctypes.c_int * 4)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("inner_prec", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_inner", ctypes.c_int), ("max_outer", ctypes.c_int), ("use_x0", ctypes.c_int),
                ("dagger", ctypes.c_int), ("check_every", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("outer_arith", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("status", ctypes.c_int), ("true_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("hop_bytes", ctypes.c_double), ("hop_gbs", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_p, _i, _d, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
_SIGS = {
    "bpp_version": ([], _i),
    "bpp_last_error": ([ctypes.c_char_p, ctypes.c_size_t], _i),
    "bpp_gauge_create": ([ctypes.POINTER(_Lattice), _p, _p, ctypes.POINTER(_p)], _i),
    "bpp_gauge_destroy": ([_p], _i),
    "bpp_clover_build": ([_p, _d, _d, _p], _i),
    "bpp_dslash": ([_p, _p, _p, _d, _i, _i, _i, _p], _i),
    "bpp_dslash_noalloc": ([_p, _p, _p, _d, _i, _i, _i, _p], _i),
    "bpp_clover_apply": ([_p, _p, _p, _i, _i, _i, _i, _p], _i),
    "bpp_schur_apply": ([_p, _p, _p, _d, _d, _i, _i, _i, _p], _i),
    "bpp_dirac_apply": ([_p, _p, _p, _d, _d, _i, _i, _p], _i),
    "bpp_solve_opts_default": ([ctypes.POINTER(SolveOpts)], None),
    "bpp_solve": ([_p, _p, _p, _d, _d, _d, _i, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _p], _i),
    "bpp_solve_lex": ([_p, _p, _p, _d, _d, _d, _i, _i, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _p], _i),
    "bpp_solve_batch": ([_i, ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.POINTER(_d), _d, _d,
                         ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _p], _i),
    "bpp_force": ([_p, _p, _p, _d, _d, _i, _p, _i, _p], _i),
    "bpp_dd_create": ([ctypes.POINTER(_Lattice), _p, _i, _p, ctypes.POINTER(_p)], _i),
    "bpp_dd_destroy": ([_p], _i),
    "bpp_dd_set_reducer": ([_p, _p, _p], _i),
    "bpp_dd_dslash": ([_p, _p, _p, _d, _i, _i, _i, _p], _i),
    "bpp_dd_schur_apply": ([_p, _p, _p, _d, _i, _i, _i, _p], _i),
    "bpp_dd_solve": ([_p, _p, _p, _d, _d, _i, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _p], _i),
    "bpp_mg_params_default": ([_p], None),
    "bpp_mg_create": ([_p, _d, _d, ctypes.POINTER(_i), _p, _i, _p, _p, ctypes.POINTER(_p)], _i),
    "bpp_mg_destroy": ([_p], _i),
    "bpp_mg_apply": ([_p, _i, _p, _p, _i, _p], _i),
    "bpp_mg_solve": ([_p, _p, _p, _d, _i, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _p], _i),
    "bpp_launch_count": ([_i], _i64),
    "bpp_prof_enable": ([_i], _i),
    "bpp_prof_read": ([_i, ctypes.POINTER(_i64), ctypes.POINTER(_d), ctypes.POINTER(_d), _i], _i),
    "bpp_work_read": ([_i, ctypes.POINTER(_i64), ctypes.POINTER(_d), _i], _i),
    "bpp_release_workspace": ([], _i),
    "bpp_fma_peak": ([_i, ctypes.POINTER(_d), _p], _i),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _check(rc):
    if rc != 0:
        buf = ctypes.create_string_buffer(1024)
        _lib.bpp_last_error(buf, 1024)
        cls = NotConverged if rc == -5 else BppError
        raise cls(rc, buf.value.decode(errors="replace"))


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _cuda(t: torch.Tensor, what):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (the library has no CPU path)")


def _cdtype(prec):
    return torch.complex128 if prec in (F64, F64DF) else torch.complex64


def version() -> int:
    return _lib.bpp_version()


def launch_count(reset: bool = False) -> int:
    return int(_lib.bpp_launch_count(int(reset)))


def prof_enable(on: bool = True):
    _check(_lib.bpp_prof_enable(int(on)))


def prof_read(prec: int, reset: bool = True):
    """(launches, total_ms, total_algorithmic_bytes) of the hopping kernels of precision prec."""
    n, ms, by = _i64(), _d(), _d()
    _check(_lib.bpp_prof_read(prec, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), int(reset)))
    return n.value, ms.value, by.value


def work_read(prec: int, reset: bool = True):
    """(launches, algorithmic bytes) of the hopping kernels of precision prec, graph work included."""
    n, by = _i64(), _d()
    _check(_lib.bpp_work_read(prec, ctypes.byref(n), ctypes.byref(by), int(reset)))
    return n.value, by.value


def release_workspace():
    _check(_lib.bpp_release_workspace())


def fma_peak(prec: int, stream=None) -> float:
    """Measured FMA-pipe throughput in TFLOP/s of prec (F64 or F32), bpp_fma_peak."""
    t = ctypes.c_double()
    _check(_lib.bpp_fma_peak(int(prec), ctypes.byref(t), _stream(stream)))
    return t.value


@dataclass(frozen=True)
class Lattice:
    L: tuple
    bc: tuple = (1, 1, 1, -1)

    @property
    def V(self):
        return self.L[0] * self.L[1] * self.L[2] * self.L[3]

    @property
    def Vh(self):
        return self.V // 2


class Gauge:
    """Gauge field U_mu(x) on the device in the library's internal layout.

    U: complex128 tensor [4][V][3][3] (CUDA or CPU; copied)."""

    def __init__(self, U: torch.Tensor, L, bc=(1, 1, 1, -1), stream=None):
        self.lattice = Lattice(tuple(int(v) for v in L), tuple(int(v) for v in bc))
        if U.dtype != torch.complex128 or tuple(U.shape) != (4, self.lattice.V, 3, 3):
            raise ValueError("U must be complex128 of shape (4, V, 3, 3)")
        U = U.contiguous()
        lat = _Lattice((ctypes.c_int * 4)(*self.lattice.L), (ctypes.c_int * 4)(*self.lattice.bc))
        h = _p()
        _check(_lib.bpp_gauge_create(ctypes.byref(lat), _ptr(U), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.clover = None
        # a few links of the source field, for matches() (a check, not a copy)
        V = self.lattice.V
        self._probe_sites = torch.tensor(sorted({0, V // 3, V // 2, (2 * V) // 3, V - 1}), dtype=torch.long)
        self._probe = U[:, self._probe_sites.to(U.device)].detach().to("cpu", copy=True)

    def matches(self, U: torch.Tensor) -> bool:
        """True when U has this field's shape and equals its source field at the
        probe sites (catches a gauge handle built from another field)."""
        if U.dtype != torch.complex128 or tuple(U.shape) != (4, self.lattice.V, 3, 3):
            return False
        return bool(torch.equal(U.detach()[:, self._probe_sites.to(U.device)].cpu(), self._probe))

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("gauge handle destroyed")
        return self._h

    def clover_build(self, kappa: float, csw: float, stream=None):
        _check(_lib.bpp_clover_build(self.handle, float(kappa), float(csw), _stream(stream)))
        self.clover = (float(kappa), float(csw))

    def destroy(self):
        if getattr(self, "_h", None) is not None:
            _lib.bpp_gauge_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _nrhs(t, per):
    n = t.numel() // per
    if n * per != t.numel() or n < 1:
        raise ValueError("field size is not a multiple of the per-RHS size")
    return n


def dslash(g: Gauge, psi: torch.Tensor, kappa: float, parity: int, prec: int = F64, stream=None):
    """parity EVEN/ODD: out_p = -kappa H_{p,pbar} psi_pbar on half fields [nrhs][Vh][4][3];
    parity FULL: out = D_W psi (clover-free) on full fields [nrhs][V][4][3]."""
    _cuda(psi, "psi")
    if psi.dtype != _cdtype(prec):
        raise ValueError(f"psi must be {_cdtype(prec)} for precision {prec}")
    per = 12 * (g.lattice.V if parity == FULL else g.lattice.Vh)
    n = _nrhs(psi, per)
    psi = psi.contiguous()
    out = torch.empty_like(psi)
    _check(_lib.bpp_dslash(g.handle, _ptr(psi), _ptr(out), float(kappa), parity, prec, n, _stream(stream)))
    return out


def dslash_noalloc(g: Gauge, psi: torch.Tensor, kappa: float, parity: int, prec: int = F64, out=None, stream=None):
    """The EVEN/ODD hopping term of dslash() without any device allocation by
    the library: for callers whose device memory is owned by another manager.
    The library's working storage is a fixed 32 MiB device array, placed on the
    device when the gauge field was created (requests that need more raise
    BppError); concurrent calls on unordered streams race.  out, if given, must
    be a contiguous CUDA tensor of psi's dtype, size and device that does not
    overlap psi (ValueError otherwise)."""
    _cuda(psi, "psi")
    if psi.dtype != _cdtype(prec):
        raise ValueError(f"psi must be {_cdtype(prec)} for precision {prec}")
    n = _nrhs(psi, 12 * g.lattice.Vh)
    psi = psi.contiguous()
    if out is None:
        out = torch.empty_like(psi)
    else:
        # the library writes n * Vh * 12 elements of complex<prec> through out
        if out.dtype != psi.dtype:
            raise ValueError(f"out must be {psi.dtype} for precision {prec}")
        if out.numel() != psi.numel():
            raise ValueError("out must have as many elements as psi")
        if not out.is_cuda or out.device != psi.device:
            raise ValueError("out must be a CUDA tensor on psi's device")
        if not out.is_contiguous():
            raise ValueError("out must be contiguous")
        o0, o1 = out.data_ptr(), out.data_ptr() + out.numel() * out.element_size()
        p0, p1 = psi.data_ptr(), psi.data_ptr() + psi.numel() * psi.element_size()
        if o0 < p1 and p0 < o1:
            raise ValueError("out must not overlap psi")
    _check(_lib.bpp_dslash_noalloc(g.handle, _ptr(psi), _ptr(out), float(kappa), parity, prec, n, _stream(stream)))
    return out


def clover_apply(g: Gauge, x: torch.Tensor, parity: int, inverse: bool = False, prec: int = F64, stream=None):
    """(1 + F) x or (1 + F)^-1 x on half fields of parity EVEN/ODD."""
    _cuda(x, "x")
    if x.dtype != _cdtype(prec):
        raise ValueError(f"x must be {_cdtype(prec)}")
    x = x.contiguous()
    n = _nrhs(x, 12 * g.lattice.Vh)
    out = torch.empty_like(x)
    _check(_lib.bpp_clover_apply(g.handle, _ptr(x), _ptr(out), parity, int(inverse), prec, n, _stream(stream)))
    return out


def schur_apply(g: Gauge, x: torch.Tensor, kappa: float, csw: float = 0.0, dagger: bool = False, prec: int = F64,
                stream=None):
    """Mhat x_e = A_ee x_e - kappa^2 H_eo A_oo^-1 H_oe x_e (or its adjoint) on even half fields."""
    _cuda(x, "x")
    if x.dtype != _cdtype(prec):
        raise ValueError(f"x must be {_cdtype(prec)}")
    x = x.contiguous()
    n = _nrhs(x, 12 * g.lattice.Vh)
    out = torch.empty_like(x)
    _check(_lib.bpp_schur_apply(g.handle, _ptr(x), _ptr(out), float(kappa), float(csw), int(dagger), prec, n,
                                _stream(stream)))
    return out


def dirac_apply(g: Gauge, x: torch.Tensor, kappa: float, csw: float = 0.0, dagger: bool = False, stream=None):
    """D x (or D^dag x) of Eq. (1) in FP64 on full complex128 fields [nrhs][V][4][3]."""
    _cuda(x, "x")
    if x.dtype != torch.complex128:
        raise ValueError("x must be complex128")
    x = x.contiguous()
    n = _nrhs(x, 12 * g.lattice.V)
    out = torch.empty_like(x)
    _check(_lib.bpp_dirac_apply(g.handle, _ptr(x), _ptr(out), float(kappa), float(csw), int(dagger), n,
                                _stream(stream)))
    return out


def solve_opts(solver=BICGSTAB, inner_prec=F32, inner_tol=None, max_inner=20000, max_outer=50, dagger=False,
               check_every=4, use_x0=False, use_graph=2, outer_df64=True, outer_arith=None) -> SolveOpts:
    """Solver options (bpp_solve_opts).  use_graph: 0 host-driven, 1 inner loop as
    a CUDA graph, 2 whole correction loop as one graph launch (default).
    outer_arith: 0 every outer-loop operator in FP64; 1 the preparation and the
    intermediate defects in double-float arithmetic, the true-residual check and
    the solution accumulation in FP64; 2 the check and the iterate in
    double-float too (the returned x is the checked iterate).
    None keeps the library default (2); outer_df64=False is outer_arith=0."""
    o = SolveOpts()
    _lib.bpp_solve_opts_default(ctypes.byref(o))
    o.solver = solver
    o.inner_prec = inner_prec
    if inner_tol is not None:
        o.inner_tol = inner_tol
    o.max_inner = max_inner
    o.max_outer = max_outer
    o.dagger = int(dagger)
    o.check_every = check_every
    o.use_x0 = int(use_x0)
    o.use_graph = int(use_graph)
    if outer_arith is not None:
        if int(outer_arith) not in (0, 1, 2):
            raise ValueError("outer_arith must be 0, 1 or 2")
        o.outer_arith = int(outer_arith)
    elif not outer_df64:
        o.outer_arith = 0
    return o


def solve(g: Gauge, b: torch.Tensor, kappa: float, csw: float = 0.0, tol: float = 1e-10, opts: SolveOpts = None,
          x: torch.Tensor = None, stream=None, raise_on_fail: bool = True):
    """x = D^-1 b (or D^-dag b with opts.dagger) to ||b - D x|| / ||b|| <= tol per RHS.
    b: complex128 [nrhs][V][4][3] (or [V][4][3]) on the device or the host.
    Returns (x, [stats dict per RHS])."""
    if b.dtype != torch.complex128:
        raise ValueError("b must be complex128")
    b = b.contiguous()
    n = _nrhs(b, 12 * g.lattice.V)
    if x is None:
        x = torch.empty_like(b)
    o = opts if opts is not None else solve_opts()
    st = (SolveStats * n)()
    rc = _lib.bpp_solve(g.handle, _ptr(b), _ptr(x), float(kappa), float(csw), float(tol), n, ctypes.byref(o), st,
                        _stream(stream))
    stats = [s.as_dict() for s in st]
    if raise_on_fail:
        _check(rc)
    return x, stats


def solve_lex(g: Gauge, b: torch.Tensor, kappa: float, csw: float = 0.0, tol: float = 1e-10, mode: int = LEX_D,
              opts: SolveOpts = None, x: torch.Tensor = None, stream=None, raise_on_fail: bool = True):
    """Full-lattice (lexical) solve of A x = b with A = D (mode LEX_D), D^dag
    (LEX_DDAG) or D^dag D (LEX_DDAGD, CG); with opts.solver = CGNR and mode
    LEX_D, x = D^-1 b through CG on the normal equations.  FP64 defect
    correction around an FP32 (or FP64) inner solve to |b - A x| / |b| <= tol.
    b: complex128 [nrhs][V][4][3] (or [V][4][3]), device or host.
    Returns (x, [stats dict per RHS])."""
    if b.dtype != torch.complex128:
        raise ValueError("b must be complex128")
    b = b.contiguous()
    n = _nrhs(b, 12 * g.lattice.V)
    if x is None:
        x = torch.empty_like(b)
    o = opts if opts is not None else solve_opts()
    st = (SolveStats * n)()
    rc = _lib.bpp_solve_lex(g.handle, _ptr(b), _ptr(x), float(kappa), float(csw), float(tol), n, int(mode),
                            ctypes.byref(o), st, _stream(stream))
    stats = [s.as_dict() for s in st]
    if raise_on_fail:
        _check(rc)
    return x, stats


def solve_batch(gauges, bs, kappas, tol: float = 1e-10, opts: SolveOpts = None, xs=None, stream=None,
                raise_on_fail: bool = True, csw: float = 0.0):
    """Independent solves on several lattices run together in every launch
    (csw != 0: each gauge holds its clover term for its own kappa and this csw)."""
    n = len(gauges)
    xs = [torch.empty_like(b) for b in bs] if xs is None else xs
    for b in bs:
        _cuda(b, "b")
    H = (_p * n)(*[g.handle for g in gauges])
    B = (_p * n)(*[_ptr(b).value for b in bs])
    X = (_p * n)(*[_ptr(x).value for x in xs])
    K = (_d * n)(*[float(k) for k in kappas])
    o = opts if opts is not None else solve_opts()
    st = (SolveStats * n)()
    rc = _lib.bpp_solve_batch(n, H, B, X, K, float(csw), float(tol), ctypes.byref(o), st, _stream(stream))
    stats = [s.as_dict() for s in st]
    if raise_on_fail:
        _check(rc)
    return xs, stats


def force(g: Gauge, x: torch.Tensor, lam: torch.Tensor, kappa: float, project: bool = False, csw: float = 0.0,
          stream=None):
    """Link gradient G (project=False) or projected force P (project=True) of
    L = Re<eta, D^-1 b>, given x = D^-1 b and lam = D^-dag eta (complex128
    [V][4][3] or [nrhs][V][4][3], summed over the right-hand sides); csw != 0
    adds the clover term's part."""
    _cuda(x, "x")
    _cuda(lam, "lam")
    if x.dtype != torch.complex128 or lam.dtype != torch.complex128:
        raise ValueError("x and lam must be complex128")
    if x.shape != lam.shape:
        raise ValueError("x and lam must have the same shape")
    x, lam = x.contiguous(), lam.contiguous()
    n = _nrhs(x, 12 * g.lattice.V)
    out = torch.empty((4, g.lattice.V, 3, 3), dtype=torch.complex128, device=x.device)
    _check(_lib.bpp_force(g.handle, _ptr(x), _ptr(lam), float(kappa), float(csw), n, _ptr(out), int(project),
                          _stream(stream)))
    return out


# Reducer of the decomposed solve's sums: (in, out, nparts, n, ctx) -> int
DD_REDUCER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                              ctypes.c_int, ctypes.c_int, ctypes.c_void_p)


class DomainDecomposition:
    """The lattice cut in x4 into ndom slabs (L4 / ndom even), each slab
    holding its own links, all on the current GPU (bpp_dd_*).  The decomposed
    hopping term and Schur operator equal dslash() and schur_apply() bit for
    bit; solve() is FP64 BiCGStab on the Schur system with per-slab
    reductions combined across slabs.

    U: complex128 [4][V][3][3] (CUDA or CPU)."""

    def __init__(self, U: torch.Tensor, L, ndom: int, bc=(1, 1, 1, -1), stream=None):
        self.lattice = Lattice(tuple(int(v) for v in L), tuple(int(v) for v in bc))
        if U.dtype != torch.complex128 or tuple(U.shape) != (4, self.lattice.V, 3, 3):
            raise ValueError("U must be complex128 of shape (4, V, 3, 3)")
        U = U.contiguous()
        lat = _Lattice((ctypes.c_int * 4)(*self.lattice.L), (ctypes.c_int * 4)(*self.lattice.bc))
        h = _p()
        _check(_lib.bpp_dd_create(ctypes.byref(lat), _ptr(U), int(ndom), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.ndom = int(ndom)
        self._reducer = None

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("decomposition handle destroyed")
        return self._h

    def set_reducer(self, fn=None):
        """fn(parts: numpy [nparts, n] float64) -> numpy [n] float64 combines the
        per-slab sums (None: the library's device sum in slab order)."""
        if fn is None:
            self._reducer = None
            _check(_lib.bpp_dd_set_reducer(self.handle, None, None))
            return
        import numpy as np

        def cb(pin, pout, nparts, n, ctx):
            try:
                parts = np.ctypeslib.as_array(pin, shape=(nparts * n,)).reshape(nparts, n).copy()
                res = np.asarray(fn(parts), dtype=np.float64).reshape(n)
                np.ctypeslib.as_array(pout, shape=(n,))[:] = res
                return 0
            except Exception:
                return 1
        self._reducer = DD_REDUCER(cb)     # kept alive with the handle
        _check(_lib.bpp_dd_set_reducer(self.handle, ctypes.cast(self._reducer, _p), None))

    def dslash(self, psi: torch.Tensor, kappa: float, parity: int, prec: int = F64, stream=None):
        _cuda(psi, "psi")
        if psi.dtype != _cdtype(prec):
            raise ValueError(f"psi must be {_cdtype(prec)} for precision {prec}")
        psi = psi.contiguous()
        n = _nrhs(psi, 12 * self.lattice.Vh)
        out = torch.empty_like(psi)
        _check(_lib.bpp_dd_dslash(self.handle, _ptr(psi), _ptr(out), float(kappa), parity, prec, n, _stream(stream)))
        return out

    def schur_apply(self, x: torch.Tensor, kappa: float, dagger: bool = False, prec: int = F64, stream=None):
        _cuda(x, "x")
        if x.dtype != _cdtype(prec):
            raise ValueError(f"x must be {_cdtype(prec)}")
        x = x.contiguous()
        n = _nrhs(x, 12 * self.lattice.Vh)
        out = torch.empty_like(x)
        _check(_lib.bpp_dd_schur_apply(self.handle, _ptr(x), _ptr(out), float(kappa), int(dagger), prec, n,
                                       _stream(stream)))
        return out

    def solve(self, b: torch.Tensor, kappa: float, tol: float = 1e-10, opts: SolveOpts = None, stream=None,
              raise_on_fail: bool = True):
        _cuda(b, "b")
        if b.dtype != torch.complex128:
            raise ValueError("b must be complex128")
        b = b.contiguous()
        n = _nrhs(b, 12 * self.lattice.V)
        x = torch.empty_like(b)
        o = opts if opts is not None else solve_opts(inner_prec=F64)
        st = (SolveStats * n)()
        rc = _lib.bpp_dd_solve(self.handle, _ptr(b), _ptr(x), float(kappa), float(tol), n, ctypes.byref(o), st,
                               _stream(stream))
        stats = [s.as_dict() for s in st]
        if raise_on_fail:
            _check(rc)
        return x, stats

    def destroy(self):
        if getattr(self, "_h", None) is not None:
            _lib.bpp_dd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class MGParams(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("coarse_tol", ctypes.c_double),
                ("coarse_maxiter", ctypes.c_int), ("gcr_restart", ctypes.c_int), ("setup_tol", ctypes.c_double)]


MG_PROLONG, MG_RESTRICT, MG_COARSE, MG_VCYCLE = 0, 1, 2, 3


def mg_params(**kw) -> MGParams:
    p = MGParams()
    _lib.bpp_mg_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Multigrid:
    """Two-level aggregation multigrid for the full-lattice D (bpp_mg_*).

    vectors: complex128 [6][V][4][3] near-null (or starting) vectors, CUDA or
    CPU; refine: inverse-iteration passes applied to them; block: the
    aggregate extents.  The gauge g (with its clover term for csw != 0) must
    outlive this object."""

    def __init__(self, g: Gauge, kappa: float, vectors: torch.Tensor, block, csw: float = 0.0, refine: int = 0,
                 params: MGParams = None, stream=None):
        if vectors.dtype != torch.complex128 or tuple(vectors.shape) != (6, g.lattice.V, 4, 3):
            raise ValueError("vectors must be complex128 of shape (6, V, 4, 3)")
        vectors = vectors.contiguous()
        self.gauge = g
        self.kappa, self.csw = float(kappa), float(csw)
        self.block = tuple(int(b) for b in block)
        self.Lc = tuple(g.lattice.L[m] // self.block[m] for m in range(4))
        self.Vc = self.Lc[0] * self.Lc[1] * self.Lc[2] * self.Lc[3]
        h = _p()
        bs = (ctypes.c_int * 4)(*self.block)
        _check(_lib.bpp_mg_create(g.handle, self.kappa, self.csw, bs, _ptr(vectors), int(refine),
                                  ctypes.byref(params) if params is not None else None, _stream(stream),
                                  ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("multigrid handle destroyed")
        return self._h

    def _apply(self, op, x, out_shape, stream=None):
        _cuda(x, "input")
        if x.dtype != torch.complex64:
            raise ValueError("multigrid operators take complex64 fields")
        x = x.contiguous()
        per = 12 * (self.Vc if op in (MG_PROLONG, MG_COARSE) else self.gauge.lattice.V)
        n = _nrhs(x, per)
        out = torch.empty((n,) + out_shape, dtype=torch.complex64, device=x.device)
        _check(_lib.bpp_mg_apply(self.handle, op, _ptr(x), _ptr(out), n, _stream(stream)))
        return out

    def prolong(self, c, stream=None):
        """P c: coarse [nrhs][Vc][12] -> full [nrhs][V][4][3]."""
        return self._apply(MG_PROLONG, c, (self.gauge.lattice.V, 4, 3), stream)

    def restrict(self, f, stream=None):
        """P^dag f: full [nrhs][V][4][3] -> coarse [nrhs][Vc][12]."""
        return self._apply(MG_RESTRICT, f, (self.Vc, 12), stream)

    def coarse(self, c, stream=None):
        """D_c c on coarse fields."""
        return self._apply(MG_COARSE, c, (self.Vc, 12), stream)

    def vcycle(self, f, stream=None):
        """M f (the preconditioner) on full fields."""
        return self._apply(MG_VCYCLE, f, (self.gauge.lattice.V, 4, 3), stream)

    def solve(self, b: torch.Tensor, tol: float = 1e-10, opts: SolveOpts = None, stream=None, raise_on_fail=True):
        _cuda(b, "b")
        if b.dtype != torch.complex128:
            raise ValueError("b must be complex128")
        b = b.contiguous()
        n = _nrhs(b, 12 * self.gauge.lattice.V)
        x = torch.empty_like(b)
        o = opts if opts is not None else solve_opts(max_inner=200)
        st = (SolveStats * n)()
        rc = _lib.bpp_mg_solve(self.handle, _ptr(b), _ptr(x), float(tol), n, ctypes.byref(o), st, _stream(stream))
        stats = [s.as_dict() for s in st]
        if raise_on_fail:
            _check(rc)
        return x, stats

    def destroy(self):
        if getattr(self, "_h", None) is not None:
            _lib.bpp_mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def exported_symbols():
    """Names of the C functions this binding binds (all declared in include/bpp.h)."""
    return sorted(_SIGS)
