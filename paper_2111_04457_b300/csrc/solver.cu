// Even-odd preconditioned solve of D x = b with a mixed-precision defect
// correction (Sec. 2, Fig. 1: a double-precision outer solver around a
// single-precision inner solver; Sec. 3: single precision "plays a main role
// in multi-precision solver algorithms").
//
//   bhat_e = b_e - D_eo D_oo^-1 b_o = b_e + kappa H_eo A_oo^-1 b_o
//   Mhat   = A_ee - kappa^2 H_eo A_oo^-1 H_oe
//   outer (FP64): r = bhat - Mhat x; stop when ||r|| <= tol ||b||;
//                 e = Mhat^-1 (r/||r||) to inner_tol in the inner precision;
//                 x += ||r|| e
//   x_o = A_oo^-1 (b_o + kappa H_oe x_e)
//   true residual ||b - D x|| / ||b|| recomputed with the full FP64 D.
//
// The inner solver is BiCGStab (van der Vorst 1992) or CGNR (CG on
// Mhat^dag Mhat with Mhat^dag = gamma5 Mhat gamma5) on the Schur system, over a
// batch of systems (right-hand sides and/or lattices) that every launch covers;
// the host only reads the per-system scalars every check_every iterations.
#include <chrono>
#include <cmath>
#include <vector>

#include "blas.h"
#include "kernels.h"
#include "solver.h"

namespace bpp {

void schur(const Batch& b, bool clover, int dag, char* in_e, char* out_e, char* tmp_o, cudaStream_t st) {
    // tmp_o = A_oo^-1 (-kappa H_oe in);  out_e = A_ee in + kappa H_eo tmp_o
    hop(b, 1, dag, clover ? HOP_INV : HOP_PLAIN, -1.0, in_e, tmp_o, nullptr, st);
    hop(b, 0, dag, clover ? HOP_CLOV_XPAY : HOP_XPAY, +1.0, tmp_o, out_e, in_e, st);
}

// Batch vector of `bt` (all systems, one parity).
struct Vec {
    DevBuf buf;
    char* p() const { return buf.as<char>(); }
};

static void make_vec(Vec& v, const Batch& bt, cudaStream_t st) { v.buf.alloc(bt.vec_bytes, st); }

static void read_scalars(const DevBuf& d, std::vector<KScal>& h, cudaStream_t st) {
    BPP_CUDA(cudaMemcpyAsync(h.data(), d.p, h.size() * sizeof(KScal), cudaMemcpyDeviceToHost, st));
    BPP_CUDA(cudaStreamSynchronize(st));
}
static void write_scalars(DevBuf& d, const std::vector<KScal>& h, cudaStream_t st) {
    BPP_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(KScal), cudaMemcpyHostToDevice, st));
}

// Inner Krylov solve Mhat e = rhs on batch bP; returns per-system iterations.
static void inner_solve(const Batch& bP, bool clover, int solver, Vec* w, DevBuf& dsc, std::vector<KScal>& hsc,
                        RedBuf& rb, int check_every, int max_iter, cudaStream_t st) {
    KScal* sc = dsc.as<KScal>();
    // every active system advances one iteration per pass, so this many chunks
    // always suffice; the cap only guards the host loop
    const int max_chunks = max_iter / check_every + 2;
    int chunks = 0;
    BlasVecs v;
    if (solver == BPP_BICGSTAB) {
        v.b = w[0].p(); v.x = w[1].p(); v.r = w[2].p(); v.rhat = w[3].p(); v.p = w[4].p();
        v.v = w[5].p(); v.s = w[6].p(); v.t = w[7].p();
        char* tmp = w[8].p();
        blas(bP, B_INIT_BICG, v, sc, rb, st);
        for (;;) {
            for (int k = 0; k < check_every; ++k) {
                schur(bP, clover, 0, v.p, v.v, tmp, st);
                blas(bP, B_ALPHA, v, sc, rb, st);
                blas(bP, B_S, v, sc, rb, st);
                schur(bP, clover, 0, v.s, v.t, tmp, st);
                blas(bP, B_OMEGA, v, sc, rb, st);
                blas(bP, B_XR, v, sc, rb, st);
                blas(bP, B_P, v, sc, rb, st);
            }
            read_scalars(dsc, hsc, st);
            bool all = true;
            for (auto& k : hsc) all = all && k.done;
            if (all || ++chunks >= max_chunks) break;
        }
    } else {
        v.b = w[0].p(); v.x = w[1].p(); v.r = w[2].p(); v.z = w[3].p(); v.p = w[4].p(); v.w = w[5].p();
        char* tmp = w[8].p();
        blas(bP, B_CG_INIT, v, sc, rb, st);
        schur(bP, clover, 1, v.r, v.z, tmp, st);
        blas(bP, B_CG_PZ, v, sc, rb, st);
        for (;;) {
            for (int k = 0; k < check_every; ++k) {
                schur(bP, clover, 0, v.p, v.w, tmp, st);
                blas(bP, B_CG_ALPHA, v, sc, rb, st);
                blas(bP, B_CG_XR, v, sc, rb, st);
                schur(bP, clover, 1, v.r, v.z, tmp, st);
                blas(bP, B_CG_BETA, v, sc, rb, st);
            }
            read_scalars(dsc, hsc, st);
            bool all = true;
            for (auto& k : hsc) all = all && k.done;
            if (all || ++chunks >= max_chunks) break;
        }
    }
}

int solve_batch(const std::vector<const Gauge*>& G, const std::vector<double>& kappa, bool clover,
                const std::vector<const void*>& b_canon, const std::vector<void*>& x_canon, double tol,
                const bpp_solve_opts& o, bpp_solve_stats* stats, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const int n = (int)G.size();
    BPP_REQUIRE(n >= 1 && n <= MAXSYS, BPP_ERR_INVALID_ARG, "number of systems must be 1..64");
    BPP_REQUIRE(tol > 0.0, BPP_ERR_INVALID_ARG, "tol must be positive");
    BPP_REQUIRE(o.solver == BPP_BICGSTAB || o.solver == BPP_CGNR, BPP_ERR_INVALID_ARG, "unknown solver");
    BPP_REQUIRE(o.inner_prec >= BPP_F64 && o.inner_prec <= BPP_F16, BPP_ERR_INVALID_ARG, "unknown inner precision");
    BPP_REQUIRE(o.max_inner > 0 && o.max_outer > 0 && o.check_every > 0, BPP_ERR_INVALID_ARG, "iteration caps must be positive");

    Batch b64, bP;
    b64.prec = P64;
    bP.prec = o.inner_prec;
    for (int s = 0; s < n; ++s) {
        batch_add(b64, *G[s], kappa[s], clover);
        batch_add(bP, *G[s], kappa[s], clover);
    }
    b64.upload(st);
    bP.upload(st);

    // FP64 vectors: b_e, b_o, bhat, x_e, x_o, r (even), tmp_o, De/Do scratch
    Vec be, bo, bhat, xe, xo, r, tmpo;
    for (Vec* v : {&be, &bo, &bhat, &xe, &xo, &r, &tmpo}) make_vec(*v, b64, st);
    // inner vectors
    Vec w[9];
    for (auto& v : w) make_vec(v, bP, st);
    RedBuf rb;
    DevBuf d64(n * sizeof(KScal), st), dP(n * sizeof(KScal), st);
    std::vector<KScal> h64(n), hP(n);
    BPP_CUDA(cudaMemsetAsync(d64.p, 0, n * sizeof(KScal), st));
    BPP_CUDA(cudaMemsetAsync(dP.p, 0, n * sizeof(KScal), st));

    // b -> even/odd FP64 (gamma5 b for the adjoint solve)
    for (int s = 0; s < n; ++s) full_to_eo(b64, s, 1, b_canon[s], 1, 0, be.p(), bo.p(), o.dagger ? 1 : 0, st);
    const int dag = 0;
    // bhat = b_e + kappa H_eo A_oo^-1 b_o
    if (clover) {
        clover_apply(b64, 1, 1, bo.p(), tmpo.p(), st);
        hop(b64, 0, dag, HOP_XPAY, +1.0, tmpo.p(), bhat.p(), be.p(), st);
    } else {
        hop(b64, 0, dag, HOP_XPAY, +1.0, bo.p(), bhat.p(), be.p(), st);
    }
    // norms: ||b||^2 = ||b_e||^2 + ||b_o||^2, ||bhat||^2
    std::vector<double> bnorm2(n), bhat2(n);
    {
        BlasVecs v;
        v.x = be.p();
        blas(b64, B_NORM2, v, d64.as<KScal>(), rb, st);
        read_scalars(d64, h64, st);
        for (int s = 0; s < n; ++s) bnorm2[s] = h64[s].bb;
        v.x = bo.p();
        blas(b64, B_NORM2, v, d64.as<KScal>(), rb, st);
        read_scalars(d64, h64, st);
        for (int s = 0; s < n; ++s) bnorm2[s] += h64[s].bb;
        v.x = bhat.p();
        blas(b64, B_NORM2, v, d64.as<KScal>(), rb, st);
        read_scalars(d64, h64, st);
        for (int s = 0; s < n; ++s) bhat2[s] = h64[s].bb;
    }
    for (int s = 0; s < n; ++s)
        BPP_REQUIRE(std::isfinite(bnorm2[s]) && std::isfinite(bhat2[s]), BPP_ERR_NONFINITE, "non-finite right-hand side");

    // initial guess
    if (o.use_x0) {
        for (int s = 0; s < n; ++s) full_to_eo(b64, s, 1, x_canon[s], 1, 0, xe.p(), xo.p(), o.dagger ? 1 : 0, st);
    } else {
        BPP_CUDA(cudaMemsetAsync(xe.p(), 0, b64.vec_bytes, st));
    }

    // Schur-residual target per system: ||bhat - Mhat x|| <= target * ||b||
    std::vector<double> target(n, tol);
    std::vector<int> outer(n, 0), inner_it(n, 0), conv(n, 0), status(n, BPP_OK);
    std::vector<double> true_res(n, 0.0);
    const int max_checks = 4;
    for (int check = 0; check < max_checks; ++check) {
        for (int it = 0; it < o.max_outer; ++it) {
            // r = bhat - Mhat x
            schur(b64, clover, dag, xe.p(), r.p(), tmpo.p(), st);
            outer_residual(b64, bhat.p(), r.p(), d64.as<KScal>(), rb, st);
            read_scalars(d64, h64, st);
            bool all = true;
            for (int s = 0; s < n; ++s) {
                if (!std::isfinite(h64[s].rr)) { status[s] = BPP_ERR_NONFINITE; h64[s].scale = 0.0; continue; }
                const double rel = std::sqrt(h64[s].rr / std::max(bnorm2[s], 1e-300));
                if (rel <= target[s] || bnorm2[s] == 0.0 || status[s] != BPP_OK) { h64[s].scale = 0.0; continue; }
                all = false;
            }
            if (all) break;
            write_scalars(d64, h64, st);
            // inner solve of Mhat e = r/||r||
            for (int s = 0; s < n; ++s) {
                KScal k{};
                const double rn = std::sqrt(std::max(h64[s].rr, 0.0));
                double itol = o.inner_tol;
                if (bP.prec == P64 || itol <= 0.0) itol = 0.5 * target[s] * std::sqrt(bnorm2[s]) / std::max(rn, 1e-300);
                itol = std::max(itol, 0.5 * target[s] * std::sqrt(bnorm2[s]) / std::max(rn, 1e-300));
                k.tol2 = itol * itol;
                k.max_iter = o.max_inner;
                hP[s] = k;
                if (h64[s].scale > 0.0) outer[s] += 1;
            }
            write_scalars(dP, hP, st);
            outer_downcast(b64, bP, r.p(), w[0].p(), d64.as<KScal>(), st);
            inner_solve(bP, clover, o.solver, w, dP, hP, rb, o.check_every, o.max_inner, st);
            for (int s = 0; s < n; ++s) inner_it[s] += h64[s].scale > 0.0 ? hP[s].iter : 0;
            outer_accumulate(b64, bP, xe.p(), w[1].p(), d64.as<KScal>(), st);
        }
        // x_o = A_oo^-1 (b_o + kappa H_oe x_e)
        hop(b64, 1, dag, clover ? HOP_INV_XPAY : HOP_XPAY, +1.0, xe.p(), xo.p(), bo.p(), st);
        // true residual with the full FP64 D: De = A_ee x_e - kappa H_eo x_o, Do = A_oo x_o - kappa H_oe x_e
        hop(b64, 0, dag, clover ? HOP_CLOV_XPAY : HOP_XPAY, -1.0, xo.p(), r.p(), xe.p(), st);
        outer_residual(b64, be.p(), r.p(), d64.as<KScal>(), rb, st);
        read_scalars(d64, h64, st);
        std::vector<double> rr(n);
        for (int s = 0; s < n; ++s) rr[s] = h64[s].rr;
        hop(b64, 1, dag, clover ? HOP_CLOV_XPAY : HOP_XPAY, -1.0, xe.p(), tmpo.p(), xo.p(), st);
        outer_residual(b64, bo.p(), tmpo.p(), d64.as<KScal>(), rb, st);
        read_scalars(d64, h64, st);
        bool again = false;
        for (int s = 0; s < n; ++s) {
            rr[s] += h64[s].rr;
            true_res[s] = bnorm2[s] > 0.0 ? std::sqrt(rr[s] / bnorm2[s]) : 0.0;
            if (!std::isfinite(true_res[s])) status[s] = BPP_ERR_NONFINITE;
            conv[s] = status[s] == BPP_OK && true_res[s] <= tol;
            if (!conv[s] && status[s] == BPP_OK) {
                again = true;
                target[s] = target[s] * 0.5 * tol / std::max(true_res[s], 1e-300);
            }
        }
        if (!again) break;
    }
    for (int s = 0; s < n; ++s) eo_to_full(b64, s, 1, xe.p(), xo.p(), x_canon[s], 1, 0, o.dagger ? 1 : 0, st);
    BPP_CUDA(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
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
        }
    }
    return rc;
}

}  // namespace bpp
