// Solve on the full lattice without even-odd preconditioning: the lexical
// propagator of Fig. 1 (Fprop_Standard_lex with a double/float mixed-precision
// solver, Sec. 2), with the operator modes D, Ddag and DdagD (Fig. 1: "mode
// is D, Ddag, DdagD, ...").
//
//   mode D:      D x = b       (BiCGStab on D, or CG on D^dag D with right-hand
//                               side D^dag b: the normal-equation propagator)
//   mode Ddag:   D^dag x = b   (the same on D^dag)
//   mode DdagD:  D^dag D x = b (CG; D^dag D is Hermitian positive definite)
//
// Outer loop: FP64 defect correction r = b - A x with the full FP64 operator A,
// an inner Krylov solve of A e = r/|r| in FP32 (or FP64: the plain solve), and
// x += |r| e, until |b - A x| / |b| <= tol.
//
// Layout: a full field is one structure-of-arrays vector whose planes hold
// 2 * stride entries, the even sites (lexicographic order of their parity) in
// the first half of every plane and the odd sites in the second half.  The
// even-odd hopping kernels see each half as a half field with plane stride
// 2 * stride, so A x is two launches (out_e = A_ee x_e - kappa H_eo x_o and
// out_o likewise); the vector kernels see one field of 2 * stride sites (the
// padding entries are zero and stay zero).  FP16 storage keeps a per-site
// scale plane of 4-byte entries, which this split does not fit: the lexical
// solve takes FP64 and FP32 inner precisions.
#include <chrono>
#include <cmath>
#include <vector>

#include "blas.h"
#include "kernels.h"
#include "lex.h"
#include "solver.h"

namespace bpp {

int work_read(int prec, int64_t* n, double* bytes, int reset);

namespace {

struct LexVec {
    DevBuf buf;
    char* p() const { return buf.as<char>(); }
};

void alloc_zero(LexVec& v, size_t bytes, cudaStream_t st) {
    v.buf.alloc(bytes, st);
    BPP_CUDA(cudaMemsetAsync(v.buf.p, 0, bytes, st));
}

}  // namespace

void lex_batches(LexBatches& lb, const Gauge& G, int prec, double kappa, bool clover, int nrhs, cudaStream_t st) {
    lb.hop.prec = lb.vec.prec = prec;
    const int64_t S2 = 2 * G.stride;
    const size_t fbytes = spinor_alloc_bytes(prec, S2);
    for (int r = 0; r < nrhs; ++r) {
        SysDesc d;
        d.g = G.g;
        for (int p = 0; p < 2; ++p) {
            for (int mu = 0; mu < 4; ++mu) d.U[p][mu] = link_view(G, prec, p, mu);
            d.A[p] = clover ? clover_view(G, prec, 0, p) : CloverView{nullptr, G.stride};
            d.Ainv[p] = clover ? clover_view(G, prec, 1, p) : CloverView{nullptr, G.stride};
        }
        d.kappa = kappa;
        d.stride = S2;
        d.vec_off = (int64_t)(r * fbytes);
        lb.hop.sys.push_back(d);
        SysDesc v = d;
        v.g.Vh = (int)S2;
        lb.vec.sys.push_back(v);
    }
    lb.hop.vec_bytes = lb.vec.vec_bytes = fbytes * nrhs;
    lb.hop.Vh_max = G.g.Vh;
    lb.vec.Vh_max = (int)S2;
    lb.hop.uniform = lb.vec.uniform = true;
    lb.hop.upload(st);
    lb.vec.upload(st);
    lb.half_off = (size_t)G.stride * 16;   // 16-byte plane entries (double2 / float4)
}

void lex_apply(const LexBatches& lb, bool clover, int dag, char* in, char* out, cudaStream_t st, const int* done,
               int ds) {
    const int mode = clover ? HOP_CLOV_XPAY : HOP_XPAY;
    char* in_o = in + lb.half_off;
    char* out_o = out + lb.half_off;
    hop(lb.hop, 0, dag, mode, -1.0, in_o, out, in, st, done, ds);
    hop(lb.hop, 1, dag, mode, -1.0, in, out_o, in_o, st, done, ds);
}

int solve_lex(const Gauge& G, double kappa, bool clover, const std::vector<const void*>& b_canon,
              const std::vector<void*>& x_canon, int mode, double tol, const bpp_solve_opts& o,
              bpp_solve_stats* stats, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    double work0 = 0.0;
    for (int q = 0; q < NPREC; ++q) {
        double by = 0.0;
        work_read(q, nullptr, &by, 0);
        work0 += by;
    }
    const int n = (int)b_canon.size();
    BPP_REQUIRE(n >= 1 && n <= MAXSYS, BPP_ERR_INVALID_ARG, "number of right-hand sides must be 1..64");
    BPP_REQUIRE(tol > 0.0, BPP_ERR_INVALID_ARG, "tol must be positive");
    BPP_REQUIRE(mode >= BPP_LEX_D && mode <= BPP_LEX_DDAGD, BPP_ERR_INVALID_ARG, "unknown operator mode");
    BPP_REQUIRE(o.solver == BPP_BICGSTAB || o.solver == BPP_CGNR, BPP_ERR_INVALID_ARG, "unknown solver");
    BPP_REQUIRE(o.inner_prec == BPP_F64 || o.inner_prec == BPP_F32, BPP_ERR_UNSUPPORTED,
                "the lexical solve takes FP64 or FP32 inner precision");
    BPP_REQUIRE(o.max_inner > 0 && o.max_outer > 0 && o.check_every > 0, BPP_ERR_INVALID_ARG,
                "iteration caps must be positive");
    const int prec = o.inner_prec;
    // DdagD is Hermitian positive definite: CG; otherwise the requested solver
    const bool normal = mode == BPP_LEX_DDAGD;
    const bool cgnr = !normal && o.solver == BPP_CGNR;
    const int dag = mode == BPP_LEX_DDAG ? 1 : 0;

    LexBatches L64, LP;
    lex_batches(L64, G, P64, kappa, clover, n, st);
    lex_batches(LP, G, prec, kappa, clover, n, st);
    const size_t b64 = L64.vec.vec_bytes, bP = LP.vec.vec_bytes;
    LexVec B, X, R, T64;
    for (LexVec* v : {&B, &X, &R, &T64}) alloc_zero(*v, b64, st);
    LexVec W[8];
    for (auto& w : W) alloc_zero(w, bP, st);
    RedBuf rb;
    DevBuf d64(n * sizeof(KScal), st), dP(n * sizeof(KScal), st);
    BPP_CUDA(cudaMemsetAsync(d64.p, 0, n * sizeof(KScal), st));
    BPP_CUDA(cudaMemsetAsync(dP.p, 0, n * sizeof(KScal), st));
    KScal* sc64 = d64.as<KScal>();
    KScal* scP = dP.as<KScal>();
    std::vector<KScal> h64(n), hP(n);
    auto read = [&](const DevBuf& d, std::vector<KScal>& h) {
        BPP_CUDA(cudaMemcpyAsync(h.data(), d.p, n * sizeof(KScal), cudaMemcpyDeviceToHost, st));
        BPP_CUDA(cudaStreamSynchronize(st));
    };
    auto write = [&](DevBuf& d, const std::vector<KScal>& h) {
        BPP_CUDA(cudaMemcpyAsync(d.p, h.data(), n * sizeof(KScal), cudaMemcpyHostToDevice, st));
    };

    for (int s = 0; s < n; ++s) full_to_eo(L64.hop, s, 1, b_canon[s], 1, 0, B.p(), B.p() + L64.half_off, 0, st);
    if (o.use_x0)
        for (int s = 0; s < n; ++s) full_to_eo(L64.hop, s, 1, x_canon[s], 1, 0, X.p(), X.p() + L64.half_off, 0, st);
    std::vector<double> bnorm2(n);
    {
        BlasVecs v;
        v.x = B.p();
        blas(L64.vec, B_NORM2, v, sc64, rb, st);
        read(d64, h64);
        for (int s = 0; s < n; ++s) bnorm2[s] = h64[s].bb;
    }
    for (int s = 0; s < n; ++s) BPP_REQUIRE(std::isfinite(bnorm2[s]), BPP_ERR_NONFINITE, "non-finite right-hand side");

    // A x in FP64 into R (A = D, D^dag or D^dag D)
    auto apply64 = [&](char* in, char* out) {
        if (normal) {
            lex_apply(L64, clover, 0, in, T64.p(), st);
            lex_apply(L64, clover, 1, T64.p(), out, st);
        } else {
            lex_apply(L64, clover, dag, in, out, st);
        }
    };
    auto defect = [&]() {   // R = B - A X, ||R||^2 and ||R|| per system
        apply64(X.p(), R.p());
        outer_residual(L64.vec, B.p(), R.p(), sc64, rb, st);
        read(d64, h64);
    };

    std::vector<int> outer(n, 0), inner_it(n, 0), conv(n, 0), status(n, BPP_OK);
    std::vector<double> true_res(n, 0.0);
    const int* doneP = &scP[0].done;
    const int ds = (int)(sizeof(KScal) / sizeof(int));
    // inner operator in the inner precision, skipping converged systems
    auto applyP = [&](int adj, char* in, char* out) {
        if (normal) {
            lex_apply(LP, clover, 0, in, W[7].p(), st, doneP, ds);
            lex_apply(LP, clover, 1, W[7].p(), out, st, doneP, ds);
        } else {
            lex_apply(LP, clover, dag ^ adj, in, out, st, doneP, ds);
        }
    };

    defect();
    for (int pass = 0;; ++pass) {
        bool any = false;
        for (int s = 0; s < n; ++s) {
            if (status[s] != BPP_OK || conv[s]) { h64[s].scale = 0.0; continue; }
            const double rr = h64[s].rr;
            if (!std::isfinite(rr)) { status[s] = BPP_ERR_NONFINITE; h64[s].scale = 0.0; continue; }
            true_res[s] = bnorm2[s] > 0.0 ? std::sqrt(rr / bnorm2[s]) : 0.0;
            if (true_res[s] <= tol) { conv[s] = 1; h64[s].scale = 0.0; continue; }
            if (outer[s] >= o.max_outer) { h64[s].scale = 0.0; continue; }
            any = true;
            // inner tolerance: the per-precision default, never tighter than
            // needed to reach tol in this correction
            const double need = 0.5 * tol * std::sqrt(bnorm2[s] / rr);
            const double itol = prec == P64 ? need : std::max(o.inner_tol > 0.0 ? o.inner_tol : 1e-6, need);
            KScal k = {};
            k.tol2 = itol * itol;
            k.max_iter = o.max_inner;
            hP[s] = k;
        }
        if (!any) break;
        for (int s = 0; s < n; ++s)
            if (h64[s].scale == 0.0) { hP[s] = KScal{}; hP[s].max_iter = 1; }
        write(d64, h64);
        write(dP, hP);
        outer_downcast(L64.vec, LP.vec, R.p(), W[0].p(), sc64, st);
        // inner solve of A e = W0 into W1
        BlasVecs v;
        if (!normal && !cgnr) {
            v.b = W[0].p(); v.x = W[1].p(); v.r = W[2].p(); v.rhat = W[3].p(); v.p = W[4].p();
            v.v = W[5].p(); v.s = W[6].p(); v.t = W[7].p();
            blas(LP.vec, B_INIT_BICG, v, scP, rb, st);
        } else {
            v.b = W[0].p(); v.x = W[1].p(); v.r = W[2].p(); v.z = W[3].p(); v.p = W[4].p(); v.w = W[5].p();
            blas(LP.vec, B_CG_INIT, v, scP, rb, st);
            if (cgnr) applyP(1, v.r, v.z);   // z = A^dag r
            BlasVecs vz = v;
            if (normal) vz.z = v.r;          // CG: p = r
            blas(LP.vec, B_CG_PZ, vz, scP, rb, st);
        }
        const int max_chunks = o.max_inner / o.check_every + 2;
        for (int chunk = 0; chunk < max_chunks; ++chunk) {
            for (int it = 0; it < o.check_every; ++it) {
                if (!normal && !cgnr) {
                    applyP(0, v.p, v.v);
                    blas(LP.vec, B_ALPHA, v, scP, rb, st);
                    blas(LP.vec, B_S, v, scP, rb, st);
                    applyP(0, v.s, v.t);
                    blas(LP.vec, B_OMEGA, v, scP, rb, st);
                    blas(LP.vec, B_XR, v, scP, rb, st);
                    blas(LP.vec, B_P, v, scP, rb, st);
                } else if (cgnr) {
                    applyP(0, v.p, v.w);
                    blas(LP.vec, B_CG_ALPHA, v, scP, rb, st);
                    blas(LP.vec, B_CG_XR, v, scP, rb, st);
                    applyP(1, v.r, v.z);
                    blas(LP.vec, B_CG_BETA, v, scP, rb, st);
                } else {
                    // CG on D^dag D: with t = D p, <p, A p> = ||t||^2 and A p = D^dag t
                    BlasVecs va = v;
                    va.w = W[6].p();
                    lex_apply(LP, clover, 0, v.p, W[6].p(), st, doneP, ds);
                    blas(LP.vec, B_CG_ALPHA, va, scP, rb, st);
                    lex_apply(LP, clover, 1, W[6].p(), v.w, st, doneP, ds);
                    blas(LP.vec, B_CG_XR, v, scP, rb, st);
                    BlasVecs vb = v;
                    vb.z = v.r;
                    blas(LP.vec, B_CG_BETA, vb, scP, rb, st);
                }
            }
            read(dP, hP);
            bool all = true;
            for (auto& k : hP) all = all && k.done;
            if (all) break;
        }
        outer_accumulate(L64.vec, LP.vec, X.p(), W[1].p(), sc64, st);
        for (int s = 0; s < n; ++s)
            if (h64[s].scale != 0.0) {
                outer[s] += 1;
                inner_it[s] += hP[s].iter;
            }
        defect();
        (void)pass;
    }
    for (int s = 0; s < n; ++s) {
        const double rr = h64[s].rr;
        if (status[s] == BPP_OK) {
            true_res[s] = bnorm2[s] > 0.0 ? std::sqrt(rr / bnorm2[s]) : 0.0;
            if (!std::isfinite(true_res[s])) status[s] = BPP_ERR_NONFINITE;
            conv[s] = true_res[s] <= tol;
        }
    }
    for (int s = 0; s < n; ++s) eo_to_full(L64.hop, s, 1, X.p(), X.p() + L64.half_off, x_canon[s], 1, 0, 0, st);
    BPP_CUDA(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    double work1 = 0.0;
    for (int q = 0; q < NPREC; ++q) {
        double by = 0.0;
        work_read(q, nullptr, &by, 0);
        work1 += by;
    }
    int rc = BPP_OK;
    for (int s = 0; s < n; ++s) {
        if (status[s] == BPP_OK && !conv[s]) status[s] = BPP_ERR_NOT_CONVERGED;
        if (status[s] != BPP_OK && rc == BPP_OK) rc = status[s];
        if (stats) {
            stats[s].outer_iters = outer[s];
            stats[s].inner_iters = inner_it[s];
            stats[s].converged = conv[s];
            stats[s].status = status[s];
            stats[s].true_resid = true_res[s];
            stats[s].seconds = secs;
            stats[s].hop_bytes = work1 - work0;
            stats[s].hop_gbs = secs > 0.0 ? (work1 - work0) / secs / 1e9 : 0.0;
        }
    }
    return rc;
}

}  // namespace bpp
