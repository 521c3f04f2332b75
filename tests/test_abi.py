"""The C ABI library loads on a machine without a GPU and exports every
function include/bpp.h declares; the binding binds exactly those (no compute
calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bpp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bpp_dslash", "bpp_clover_apply", "bpp_solve", "bpp_gauge_create", "bpp_force",
                     "bpp_solve_batch", "bpp_schur_apply", "bpp_dirac_apply", "bpp_clover_build"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2111_04457_b300 as bpp
    lib = ctypes.CDLL(os.path.join(os.path.dirname(bpp.__file__), "libbpp.so"))
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(bpp.exported_symbols()) == declared_functions()


def test_version_and_error_without_gpu():
    import paper_2111_04457_b300 as bpp
    assert bpp.version() >= 10000
    # an invalid call fails with a status code, never a crash or an exception across the ABI
    rc = bpp._lib.bpp_gauge_destroy(None)
    assert rc == 0
    buf = ctypes.create_string_buffer(256)
    rc = bpp._lib.bpp_dslash(None, None, None, 0.1, 0, 0, 1, None)
    assert rc == -1
    assert bpp._lib.bpp_last_error(buf, 256) == -1
    assert b"NULL" in buf.value


def test_gauge_create_rejects_bad_lattices_before_touching_the_gpu():
    import paper_2111_04457_b300 as bpp
    lib = bpp._lib
    h = ctypes.c_void_p()
    dummy = ctypes.create_string_buffer(16)
    for L, bc in [((4, 3, 4, 4), (1, 1, 1, -1)),     # odd extent: not bipartite
                  ((3, 4, 4, 4), (1, 1, 1, -1)),
                  ((4, 4, 4, 0), (1, 1, 1, -1)),
                  ((4, 4, 4, 4), (1, 1, 1, 2))]:       # bc must be +-1
        lat = bpp._Lattice((ctypes.c_int * 4)(*L), (ctypes.c_int * 4)(*bc))
        rc = lib.bpp_gauge_create(ctypes.byref(lat), dummy, None, ctypes.byref(h))
        assert rc == -1, (L, bc)
    rc = lib.bpp_gauge_create(None, dummy, None, ctypes.byref(h))
    assert rc == -1


def test_prof_classes_without_gpu():
    """Every documented kernel class (0..9) reads back as zero launches before
    any launch; a class out of range is refused with INVALID_ARG."""
    import pytest

    import paper_2111_04457_b300 as bpp
    for c in range(10):
        n, ms, by = bpp.prof_read(c, reset=True)
        assert n == 0 and ms == 0.0 and by == 0.0
    for c in (-1, 10):
        with pytest.raises(bpp.BppError) as e:
            bpp.prof_read(c)
        assert e.value.code == -1


def test_solve_opts_defaults_without_gpu():
    """The documented defaults of bpp_solve_opts_default (header), read back
    through the binding: BiCGStab, FP32 inner, per-precision inner tolerance,
    whole-solve graph, double-float outer loop with its own check."""
    import paper_2111_04457_b300 as bpp
    o = bpp.SolveOpts()
    bpp._lib.bpp_solve_opts_default(ctypes.byref(o))
    assert (o.solver, o.inner_prec, o.inner_tol, o.max_inner, o.max_outer) == (bpp.BICGSTAB, bpp.F32, 0.0, 20000, 50)
    assert (o.use_x0, o.dagger, o.check_every, o.use_graph, o.outer_arith) == (0, 0, 4, 2, 2)
    assert bpp.solve_opts(outer_df64=False).outer_arith == 0
    assert bpp.solve_opts(outer_arith=1).outer_arith == 1
