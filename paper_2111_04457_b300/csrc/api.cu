// C ABI of the library (include/bpp.h): argument checks, boundary layout
// conversion and dispatch; no C++ exception crosses this file's functions.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "blas.h"
#include "gauge.h"
#include "kernels.h"
#include "solver.h"
#include "dd.h"
#include "mg.h"

namespace bpp {
int prof_enable(int on);
int prof_read(int prec, int64_t* n, double* ms, double* bytes, int reset);
int64_t launch_count(int reset);
int work_read(int prec, int64_t* n, double* bytes, int reset);
int release_workspace();
int noalloc_prepare(int dev, cudaStream_t st, std::string* err, void** ptr);
}  // namespace bpp

using namespace bpp;

static thread_local std::string t_err;
static thread_local int t_code = BPP_OK;

static int fail(int code, const std::string& m) {
    t_err = m;
    t_code = code;
    return code;
}

namespace bpp {
// Records an error for bpp_last_error from entry points defined in other files.
int set_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace bpp

template <class F>
static int guard(const char* fn, F f) {
    try {
        return (int)f();
    } catch (const Error& e) {
        return fail(e.code, std::string(fn) + ": " + e.what());
    } catch (const std::exception& e) {
        return fail(BPP_ERR_CUDA, std::string(fn) + ": " + e.what());
    } catch (...) {
        return fail(BPP_ERR_CUDA, std::string(fn) + ": unknown failure");
    }
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void check_gauge(const Gauge* G) { BPP_REQUIRE(G != nullptr, BPP_ERR_INVALID_ARG, "NULL gauge handle"); }
static void check_prec(int prec, bool allow_df = false) {
    BPP_REQUIRE(prec == BPP_F64 || prec == BPP_F32 || prec == BPP_F16 || (allow_df && prec == BPP_F64DF),
                BPP_ERR_INVALID_ARG, "unknown precision");
}
static int canon_is_f64(int prec) { return prec == BPP_F64 || prec == BPP_F64DF; }
static void check_clover(const Gauge& G, double kappa, double csw) {
    if (csw == 0.0) return;
    BPP_REQUIRE(G.has_clover, BPP_ERR_UNSUPPORTED, "clover term not built (call bpp_clover_build)");
    BPP_REQUIRE(std::fabs(G.clov_kappa - kappa) <= 1e-14 * std::fabs(kappa) &&
                    std::fabs(G.clov_csw - csw) <= 1e-14 * std::fabs(csw),
                BPP_ERR_INVALID_ARG, "kappa/csw differ from the ones bpp_clover_build used");
}

static void build_batch(Batch& b, const Gauge& G, int prec, double kappa, bool clover, int nrhs, cudaStream_t st) {
    b.prec = prec;
    b.comp = link_compression(G, prec);
    for (int r = 0; r < nrhs; ++r) batch_add(b, G, kappa, clover);
    b.upload(st);
}

extern "C" {

int bpp_version(void) { return 10000; }

int bpp_last_error(char* buf, size_t n) {
    if (buf && n) {
        std::strncpy(buf, t_err.c_str(), n - 1);
        buf[n - 1] = '\0';
    }
    return t_code;
}

int bpp_gauge_create(const bpp_lattice* lat, const void* U_lex, bpp_stream stream, bpp_gauge* out) {
    return guard("bpp_gauge_create", [&]() -> int {
        BPP_REQUIRE(lat && U_lex && out, BPP_ERR_INVALID_ARG, "NULL argument");
        for (int mu = 0; mu < 4; ++mu) {
            BPP_REQUIRE(lat->L[mu] >= 2, BPP_ERR_INVALID_ARG, "every L[mu] must be >= 2");
            BPP_REQUIRE(lat->bc[mu] == 1 || lat->bc[mu] == -1, BPP_ERR_INVALID_ARG, "bc[mu] must be +1 or -1");
        }
        // even-odd preconditioning needs a bipartite lattice: every extent even
        for (int mu = 0; mu < 4; ++mu)
            BPP_REQUIRE(lat->L[mu] % 2 == 0, BPP_ERR_INVALID_ARG, "every L[mu] must be even (even-odd decomposition)");
        const int64_t V = (int64_t)lat->L[0] * lat->L[1] * lat->L[2] * lat->L[3];
        BPP_REQUIRE(V / 2 < (int64_t)1 << 30, BPP_ERR_INVALID_ARG, "lattice too large");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        Gauge* G = new Gauge();
        try {
            for (int mu = 0; mu < 4; ++mu) { G->g.L[mu] = lat->L[mu]; G->g.bc[mu] = lat->bc[mu]; }
            G->g.Lh = lat->L[0] / 2;
            G->g.Vh = (int)(V / 2);
            G->V = V;
            G->Vh = V / 2;
            G->stride = pad_stride(G->Vh);
            BPP_CUDA(cudaGetDevice(&G->device));
            // places the fixed scratch array of bpp_dslash_noalloc on this
            // device now, so that entry point never causes an allocation
            {
                std::string err;
                const int rc = noalloc_prepare(G->device, st, &err, nullptr);
                BPP_REQUIRE(rc == BPP_OK, rc, err);
            }
            for (int p = 0; p < NPREC; ++p) BPP_CUDA(cudaMalloc(&G->links[p], 8 * link_alloc_bytes(p, G->stride)));
            const size_t bytes = (size_t)V * 4 * 9 * 16;
            if (is_device_ptr(U_lex)) {
                links_to_internal(*G, U_lex, st);
            } else {
                DevBuf tmp(bytes, st);
                BPP_CUDA(cudaMemcpyAsync(tmp.p, U_lex, bytes, cudaMemcpyHostToDevice, st));
                links_to_internal(*G, tmp.p, st);
            }
            BPP_CUDA(cudaStreamSynchronize(st));
        } catch (...) {
            for (int p = 0; p < NPREC; ++p) {
                if (G->links[p]) cudaFree(G->links[p]);
                if (G->links12[p]) cudaFree(G->links12[p]);
            }
            delete G;
            throw;
        }
        *out = G;
        return BPP_OK;
    });
}

int bpp_gauge_destroy(bpp_gauge g) {
    return guard("bpp_gauge_destroy", [&]() -> int {
        if (!g) return BPP_OK;
        drop_plans(g);
        cudaDeviceSynchronize();
        for (int p = 0; p < NPREC; ++p) {
            if (g->links[p]) cudaFree(g->links[p]);
            if (g->links12[p]) cudaFree(g->links12[p]);
            if (g->clover[p]) cudaFree(g->clover[p]);
        }
        delete g;
        return BPP_OK;
    });
}

int bpp_clover_build(bpp_gauge g, double kappa, double csw, bpp_stream stream) {
    return guard("bpp_clover_build", [&]() -> int {
        check_gauge(g);
        BPP_REQUIRE(std::isfinite(kappa) && std::isfinite(csw), BPP_ERR_INVALID_ARG, "kappa and csw must be finite");
        clover_build(*g, kappa, csw, reinterpret_cast<cudaStream_t>(stream));
        return BPP_OK;
    });
}

int bpp_dslash(bpp_gauge U, const void* psi, void* out, double kappa, int parity, int prec, int nrhs,
               bpp_stream stream) {
    return guard("bpp_dslash", [&]() -> int {
        check_gauge(U);
        check_prec(prec, true);
        BPP_REQUIRE(psi && out && psi != out, BPP_ERR_INVALID_ARG, "NULL or aliased field");
        BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
        BPP_REQUIRE(parity == BPP_EVEN || parity == BPP_ODD || parity == BPP_FULL, BPP_ERR_INVALID_ARG, "bad parity");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        Batch b;
        build_batch(b, *U, prec, kappa, false, nrhs, st);
        const int f64 = canon_is_f64(prec);
        DevBuf vin(b.vec_bytes, st), vout(b.vec_bytes, st);
        if (parity != BPP_FULL) {
            half_to_int(b, psi, f64, vin.as<char>(), st);
            hop(b, parity, 0, HOP_PLAIN, -1.0, vin.as<char>(), vout.as<char>(), nullptr, st);
            int_to_half(b, vout.as<char>(), out, f64, st);
        } else {
            DevBuf ve(b.vec_bytes, st), vo(b.vec_bytes, st);
            full_to_eo(b, 0, nrhs, psi, f64, U->V * 12, vin.as<char>(), vout.as<char>(), 0, st);
            hop(b, 0, 0, HOP_XPAY, -1.0, vout.as<char>(), ve.as<char>(), vin.as<char>(), st);
            hop(b, 1, 0, HOP_XPAY, -1.0, vin.as<char>(), vo.as<char>(), vout.as<char>(), st);
            eo_to_full(b, 0, nrhs, ve.as<char>(), vo.as<char>(), out, f64, U->V * 12, 0, st);
        }
        return BPP_OK;
    });
}

int bpp_clover_apply(bpp_gauge U, const void* in, void* out, int parity, int inverse, int prec, int nrhs,
                     bpp_stream stream) {
    return guard("bpp_clover_apply", [&]() -> int {
        check_gauge(U);
        check_prec(prec);
        BPP_REQUIRE(in && out, BPP_ERR_INVALID_ARG, "NULL field");
        BPP_REQUIRE(parity == BPP_EVEN || parity == BPP_ODD, BPP_ERR_INVALID_ARG, "parity must be EVEN or ODD");
        BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
        BPP_REQUIRE(U->has_clover, BPP_ERR_UNSUPPORTED, "clover term not built (call bpp_clover_build)");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        Batch b;
        build_batch(b, *U, prec, U->clov_kappa, true, nrhs, st);
        const int f64 = prec == BPP_F64;
        DevBuf vin(b.vec_bytes, st), vout(b.vec_bytes, st);
        half_to_int(b, in, f64, vin.as<char>(), st);
        clover_apply(b, parity, inverse ? 1 : 0, vin.as<char>(), vout.as<char>(), st);
        int_to_half(b, vout.as<char>(), out, f64, st);
        return BPP_OK;
    });
}

int bpp_schur_apply(bpp_gauge U, const void* in, void* out, double kappa, double csw, int dagger, int prec,
                    int nrhs, bpp_stream stream) {
    return guard("bpp_schur_apply", [&]() -> int {
        check_gauge(U);
        check_prec(prec, true);
        check_clover(*U, kappa, csw);
        BPP_REQUIRE(in && out && in != out, BPP_ERR_INVALID_ARG, "NULL or aliased field");
        BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        Batch b;
        build_batch(b, *U, prec, kappa, csw != 0.0, nrhs, st);
        const int f64 = canon_is_f64(prec);
        DevBuf vin(b.vec_bytes, st), vout(b.vec_bytes, st), tmp(b.vec_bytes, st);
        half_to_int(b, in, f64, vin.as<char>(), st);
        schur(b, csw != 0.0, dagger ? 1 : 0, vin.as<char>(), vout.as<char>(), tmp.as<char>(), st);
        int_to_half(b, vout.as<char>(), out, f64, st);
        return BPP_OK;
    });
}

int bpp_dirac_apply(bpp_gauge U, const void* in, void* out, double kappa, double csw, int dagger, int nrhs,
                    bpp_stream stream) {
    return guard("bpp_dirac_apply", [&]() -> int {
        check_gauge(U);
        check_clover(*U, kappa, csw);
        BPP_REQUIRE(in && out && in != out, BPP_ERR_INVALID_ARG, "NULL or aliased field");
        BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        const bool cl = csw != 0.0;
        Batch b;
        build_batch(b, *U, P64, kappa, cl, nrhs, st);
        DevBuf xe(b.vec_bytes, st), xo(b.vec_bytes, st), ye(b.vec_bytes, st), yo(b.vec_bytes, st);
        full_to_eo(b, 0, nrhs, in, 1, U->V * 12, xe.as<char>(), xo.as<char>(), 0, st);
        const int mode = cl ? HOP_CLOV_XPAY : HOP_XPAY;
        const int dag = dagger ? 1 : 0;
        hop(b, 0, dag, mode, -1.0, xo.as<char>(), ye.as<char>(), xe.as<char>(), st);
        hop(b, 1, dag, mode, -1.0, xe.as<char>(), yo.as<char>(), xo.as<char>(), st);
        eo_to_full(b, 0, nrhs, ye.as<char>(), yo.as<char>(), out, 1, U->V * 12, 0, st);
        return BPP_OK;
    });
}

void bpp_solve_opts_default(bpp_solve_opts* o) {
    if (!o) return;
    o->solver = BPP_BICGSTAB;
    o->inner_prec = BPP_F32;
    o->inner_tol = 0.0;
    o->max_inner = 20000;
    o->max_outer = 50;
    o->use_x0 = 0;
    o->dagger = 0;
    o->check_every = 4;
    o->use_graph = 2;
    o->outer_arith = 2;
}

int bpp_solve(bpp_gauge U, const void* b, void* x, double kappa, double csw, double tol, int nrhs,
              const bpp_solve_opts* opts, bpp_solve_stats* stats, bpp_stream stream) {
    return guard("bpp_solve", [&]() -> int {
        check_gauge(U);
        check_clover(*U, kappa, csw);
        BPP_REQUIRE(b && x, BPP_ERR_INVALID_ARG, "NULL field");
        BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
        BPP_REQUIRE(std::isfinite(kappa), BPP_ERR_INVALID_ARG, "kappa must be finite");
        bpp_solve_opts o;
        bpp_solve_opts_default(&o);
        if (opts) o = *opts;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        const size_t field = (size_t)U->V * 12 * 16;
        const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
        DevBuf bbuf, xbuf;
        const char* bp = static_cast<const char*>(b);
        char* xp = static_cast<char*>(x);
        if (!bdev) {
            bbuf.alloc(field * nrhs, st);
            BPP_CUDA(cudaMemcpyAsync(bbuf.p, b, field * nrhs, cudaMemcpyHostToDevice, st));
            bp = bbuf.as<char>();
        }
        if (!xdev) {
            xbuf.alloc(field * nrhs, st);
            if (o.use_x0) BPP_CUDA(cudaMemcpyAsync(xbuf.p, x, field * nrhs, cudaMemcpyHostToDevice, st));
            xp = xbuf.as<char>();
        }
        std::vector<const Gauge*> G(nrhs, U);
        std::vector<double> k(nrhs, kappa);
        std::vector<const void*> bv(nrhs);
        std::vector<void*> xv(nrhs);
        for (int r = 0; r < nrhs; ++r) {
            bv[r] = bp + field * r;
            xv[r] = xp + field * r;
        }
        int rc = solve_batch(G, k, csw != 0.0, bv, xv, tol, o, stats, st);
        if (!xdev) {
            BPP_CUDA(cudaMemcpyAsync(x, xp, field * nrhs, cudaMemcpyDeviceToHost, st));
            BPP_CUDA(cudaStreamSynchronize(st));
        }
        if (rc != BPP_OK) return fail(rc, "bpp_solve: a right-hand side did not reach the tolerance (see stats)");
        return BPP_OK;
    });
}

int bpp_solve_lex(bpp_gauge U, const void* b, void* x, double kappa, double csw, double tol, int nrhs, int mode,
                  const bpp_solve_opts* opts, bpp_solve_stats* stats, bpp_stream stream) {
    return guard("bpp_solve_lex", [&]() -> int {
        check_gauge(U);
        check_clover(*U, kappa, csw);
        BPP_REQUIRE(b && x, BPP_ERR_INVALID_ARG, "NULL field");
        BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
        BPP_REQUIRE(std::isfinite(kappa), BPP_ERR_INVALID_ARG, "kappa must be finite");
        bpp_solve_opts o;
        bpp_solve_opts_default(&o);
        if (opts) o = *opts;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        const size_t field = (size_t)U->V * 12 * 16;
        const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
        DevBuf bbuf, xbuf;
        const char* bp = static_cast<const char*>(b);
        char* xp = static_cast<char*>(x);
        if (!bdev) {
            bbuf.alloc(field * nrhs, st);
            BPP_CUDA(cudaMemcpyAsync(bbuf.p, b, field * nrhs, cudaMemcpyHostToDevice, st));
            bp = bbuf.as<char>();
        }
        if (!xdev) {
            xbuf.alloc(field * nrhs, st);
            if (o.use_x0) BPP_CUDA(cudaMemcpyAsync(xbuf.p, x, field * nrhs, cudaMemcpyHostToDevice, st));
            xp = xbuf.as<char>();
        }
        std::vector<const void*> bv(nrhs);
        std::vector<void*> xv(nrhs);
        for (int r = 0; r < nrhs; ++r) {
            bv[r] = bp + field * r;
            xv[r] = xp + field * r;
        }
        int rc = solve_lex(*U, kappa, csw != 0.0, bv, xv, mode, tol, o, stats, st);
        if (!xdev) {
            BPP_CUDA(cudaMemcpyAsync(x, xp, field * nrhs, cudaMemcpyDeviceToHost, st));
            BPP_CUDA(cudaStreamSynchronize(st));
        }
        if (rc != BPP_OK) return fail(rc, "bpp_solve_lex: a right-hand side did not reach the tolerance (see stats)");
        return BPP_OK;
    });
}

int bpp_solve_batch(int nlat, const bpp_gauge* U, const void* const* b, void* const* x, const double* kappa,
                    double csw, double tol, const bpp_solve_opts* opts, bpp_solve_stats* stats, bpp_stream stream) {
    return guard("bpp_solve_batch", [&]() -> int {
        BPP_REQUIRE(nlat >= 1 && nlat <= MAXSYS && U && b && x && kappa, BPP_ERR_INVALID_ARG, "bad batch arguments");
        bpp_solve_opts o;
        bpp_solve_opts_default(&o);
        if (opts) o = *opts;
        std::vector<const Gauge*> G(nlat);
        std::vector<double> k(nlat);
        std::vector<const void*> bv(nlat);
        std::vector<void*> xv(nlat);
        for (int i = 0; i < nlat; ++i) {
            check_gauge(U[i]);
            check_clover(*U[i], kappa[i], csw);
            BPP_REQUIRE(b[i] && x[i] && is_device_ptr(b[i]) && is_device_ptr(x[i]), BPP_ERR_INVALID_ARG,
                        "batched solve fields must be device pointers");
            G[i] = U[i];
            k[i] = kappa[i];
            bv[i] = b[i];
            xv[i] = x[i];
        }
        int rc = solve_batch(G, k, csw != 0.0, bv, xv, tol, o, stats, reinterpret_cast<cudaStream_t>(stream));
        if (rc != BPP_OK) return fail(rc, "bpp_solve_batch: a lattice did not reach the tolerance (see stats)");
        return BPP_OK;
    });
}

int bpp_force(bpp_gauge U, const void* x, const void* lam, double kappa, double csw, int nrhs, void* dU,
              int project_su3, bpp_stream stream) {
    return guard("bpp_force", [&]() -> int {
        check_gauge(U);
        BPP_REQUIRE(x && lam && dU, BPP_ERR_INVALID_ARG, "NULL field");
        BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
        BPP_REQUIRE(std::isfinite(kappa) && std::isfinite(csw), BPP_ERR_INVALID_ARG, "kappa and csw must be finite");
        BPP_REQUIRE(is_device_ptr(x) && is_device_ptr(lam) && is_device_ptr(dU), BPP_ERR_INVALID_ARG,
                    "x, lam and dU must be device memory");
        force(*U, x, lam, kappa, csw, nrhs, dU, project_su3 ? 1 : 0, reinterpret_cast<cudaStream_t>(stream));
        return BPP_OK;
    });
}

int bpp_dd_create(const bpp_lattice* lat, const void* U_lex, int ndom, bpp_stream stream, bpp_dd* out) {
    return guard("bpp_dd_create", [&]() -> int {
        dd_create(lat, U_lex, ndom, reinterpret_cast<cudaStream_t>(stream), out);
        return BPP_OK;
    });
}

int bpp_dd_destroy(bpp_dd dd) {
    return guard("bpp_dd_destroy", [&]() -> int {
        dd_destroy(dd);
        return BPP_OK;
    });
}

int bpp_dd_set_reducer(bpp_dd dd, bpp_dd_reducer fn, void* ctx) {
    return guard("bpp_dd_set_reducer", [&]() -> int {
        dd_set_reducer(dd, fn, ctx);
        return BPP_OK;
    });
}

int bpp_dd_dslash(bpp_dd dd, const void* psi, void* out, double kappa, int parity, int prec, int nrhs,
                  bpp_stream stream) {
    return guard("bpp_dd_dslash", [&]() -> int {
        BPP_REQUIRE(psi && out && psi != out, BPP_ERR_INVALID_ARG, "NULL or aliased field");
        dd_dslash(dd, psi, out, kappa, parity, prec, nrhs, reinterpret_cast<cudaStream_t>(stream));
        return BPP_OK;
    });
}

int bpp_dd_schur_apply(bpp_dd dd, const void* in, void* out, double kappa, int dagger, int prec, int nrhs,
                       bpp_stream stream) {
    return guard("bpp_dd_schur_apply", [&]() -> int {
        BPP_REQUIRE(in && out && in != out, BPP_ERR_INVALID_ARG, "NULL or aliased field");
        dd_schur(dd, in, out, kappa, dagger ? 1 : 0, prec, nrhs, reinterpret_cast<cudaStream_t>(stream));
        return BPP_OK;
    });
}

int bpp_dd_solve(bpp_dd dd, const void* b, void* x, double kappa, double tol, int nrhs, const bpp_solve_opts* opts,
                 bpp_solve_stats* stats, bpp_stream stream) {
    return guard("bpp_dd_solve", [&]() -> int {
        BPP_REQUIRE(b && x && is_device_ptr(b) && is_device_ptr(x), BPP_ERR_INVALID_ARG, "b and x must be device memory");
        BPP_REQUIRE(std::isfinite(kappa), BPP_ERR_INVALID_ARG, "kappa must be finite");
        bpp_solve_opts o;
        bpp_solve_opts_default(&o);
        o.inner_prec = BPP_F64;
        if (opts) o = *opts;
        const int rc = dd_solve(dd, b, x, kappa, tol, nrhs, o, stats, reinterpret_cast<cudaStream_t>(stream));
        if (rc != BPP_OK) return fail(rc, "bpp_dd_solve: a right-hand side did not reach the tolerance (see stats)");
        return BPP_OK;
    });
}

void bpp_mg_params_default(bpp_mg_params* p) {
    if (!p) return;
    p->nu_pre = 4;
    p->nu_post = 4;
    p->coarse_tol = 0.2;
    p->coarse_maxiter = 15;
    p->gcr_restart = 12;
    p->setup_tol = 0.05;
}

int bpp_mg_create(bpp_gauge U, double kappa, double csw, const int block[4], const void* vectors, int refine,
                  const bpp_mg_params* params, bpp_stream stream, bpp_mg* out) {
    return guard("bpp_mg_create", [&]() -> int {
        check_gauge(U);
        BPP_REQUIRE(std::isfinite(kappa) && std::isfinite(csw), BPP_ERR_INVALID_ARG, "kappa and csw must be finite");
        BPP_REQUIRE(refine >= 0 && refine <= 8, BPP_ERR_INVALID_ARG, "refine must be 0..8");
        mg_create(U, kappa, csw, block, vectors, refine, params, reinterpret_cast<cudaStream_t>(stream), out);
        return BPP_OK;
    });
}

int bpp_mg_destroy(bpp_mg mg) {
    return guard("bpp_mg_destroy", [&]() -> int {
        mg_destroy(mg);
        return BPP_OK;
    });
}

int bpp_mg_apply(bpp_mg mg, int op, const void* in, void* out, int nrhs, bpp_stream stream) {
    return guard("bpp_mg_apply", [&]() -> int {
        BPP_REQUIRE(in && out && in != out && is_device_ptr(in) && is_device_ptr(out), BPP_ERR_INVALID_ARG,
                    "in and out must be distinct device buffers");
        mg_apply_op(mg, op, in, out, nrhs, reinterpret_cast<cudaStream_t>(stream));
        return BPP_OK;
    });
}

int bpp_mg_solve(bpp_mg mg, const void* b, void* x, double tol, int nrhs, const bpp_solve_opts* opts,
                 bpp_solve_stats* stats, bpp_stream stream) {
    return guard("bpp_mg_solve", [&]() -> int {
        BPP_REQUIRE(b && x && is_device_ptr(b) && is_device_ptr(x), BPP_ERR_INVALID_ARG, "b and x must be device memory");
        bpp_solve_opts o;
        bpp_solve_opts_default(&o);
        o.max_inner = 200;
        if (opts) o = *opts;
        const int rc = mg_solve(mg, b, x, tol, nrhs, o, stats, reinterpret_cast<cudaStream_t>(stream));
        if (rc != BPP_OK) return fail(rc, "bpp_mg_solve: a right-hand side did not reach the tolerance (see stats)");
        return BPP_OK;
    });
}

int64_t bpp_launch_count(int reset) { return launch_count(reset); }

int bpp_prof_enable(int enable) { return prof_enable(enable); }

int bpp_prof_read(int prec, int64_t* launches, double* ms, double* bytes, int reset) {
    return guard("bpp_prof_read", [&]() -> int { return prof_read(prec, launches, ms, bytes, reset); });
}

int bpp_work_read(int prec, int64_t* launches, double* bytes, int reset) {
    return guard("bpp_work_read", [&]() -> int { return work_read(prec, launches, bytes, reset); });
}

int bpp_fma_peak(int prec, double* tflops, bpp_stream stream) {
    return guard("bpp_fma_peak", [&]() -> int {
        BPP_REQUIRE(tflops, BPP_ERR_INVALID_ARG, "tflops is NULL");
        *tflops = fma_peak(prec, (cudaStream_t)stream);
        return BPP_OK;
    });
}

int bpp_release_workspace(void) {
    return guard("bpp_release_workspace", [&]() -> int {
        drop_plans(nullptr);
        return release_workspace();
    });
}

}  // extern "C"
