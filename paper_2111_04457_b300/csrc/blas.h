// Fused vector updates with reductions for the Krylov solvers (BiCGStab of
// van der Vorst 1992 and CGNR), batched over systems, with all scalars kept on
// the device: every reduction ends in the last block of its system, which
// sums the per-block partials in a fixed order (deterministic) and derives the
// next solver scalars, so the host never waits inside an iteration.
#pragma once

#include "bpp_internal.h"
#include "gauge.h"

namespace bpp {

// Per-system solver scalars (complex numbers as double2).
struct KScal {
    double2 rho;      // <rhat, r>
    double2 alpha, omega, beta;
    double2 rv;       // <rhat, v>
    double2 ts;       // <t, s>
    double tt;        // <t, t>
    double rr;        // ||r||^2 (recursive)
    double bb;        // ||b||^2 of the system being solved
    double tol2;      // stop when rr <= tol2 * bb
    double zz;        // CGNR: ||z||^2
    double scale;     // outer loop: ||r|| of the current defect
    int iter;
    int max_iter;
    int done;         // 1: converged or stopped
    int status;       // 0 ok, 1 breakdown, 2 iteration cap, 3 non-finite
};

// Workspace for the reductions of one batch.
struct RedBuf {
    DevBuf partials;   // nblocks * 4 doubles
    DevBuf tickets;    // MAXSYS unsigned, self-resetting
    int cap_blocks = 0;
    bool persistent = false;
    void ensure(int nblocks, int nsys, cudaStream_t st);
};

enum BlasOp {
    B_INIT_BICG = 0,   // r = b, rhat = b, p = b, x = 0; rho = bb = ||b||^2
    B_ALPHA,           // alpha = rho / <rhat, v>
    B_S,               // s = r - alpha v
    B_OMEGA,           // omega = <t,s>/<t,t>
    B_XR,              // x += alpha p + omega s; r = s - omega t; rho, beta, rr, done
    B_P,               // p = r + beta (p - omega v)
    B_CG_INIT,         // r = b, x = 0; bb = ||b||^2 (CGNR; z = Mdag r follows)
    B_CG_PZ,           // p = z; zz = ||z||^2
    B_CG_ALPHA,        // alpha = zz / ||w||^2
    B_CG_XR,           // x += alpha p; r -= alpha w; rr, done
    B_CG_BETA,         // beta = ||z||^2 / zz; zz = ||z||^2; p = z + beta p
    B_NORM2,           // bb = ||x||^2 (no update)
    B_NORM2X2,         // bb = ||x||^2 + ||r||^2 (no update)
    B_MR               // minimal-residual step after B_OMEGA: x += omega s; s -= omega t (no reduction)
};

struct BlasVecs {
    char *x = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr,
         *b = nullptr, *w = nullptr, *z = nullptr;
};

// With red_out set, the reducing operations write each system's sums
// (4 doubles per system) to red_out instead of deriving the scalars; blas_fin
// then derives them from combined sums (a reduction across the domains of a
// decomposition).  Every operation except B_CG_BETA has this form.
void blas(const Batch& bt, int op, const BlasVecs& vv, KScal* sc, RedBuf& rb, cudaStream_t st,
          double* red_out = nullptr);
void blas_fin(int op, KScal* sc, const double* tot, int n, cudaStream_t st);
// B_ALPHA or B_OMEGA from the per-warp partials of a hop with fused inner
// products (HopRed; part [system][wstride][4]): the (Vh + 31) / 32 partials of
// each active system are summed in fixed chunks (chunk sums in `chunks`,
// [system][hop_red_chunks(wstride)][4] doubles), then in chunk order, and
// alpha or omega is derived; rb's tickets find the last chunk.
int hop_red_chunks(int wstride);
void hop_red_fin(const Batch& bt, int op, const double* part, int wstride, KScal* sc, RedBuf& rb, double* chunks,
                 cudaStream_t st);

// Outer defect-correction steps (FP64 batch b64 and inner-precision batch bP
// over the same systems):
// r64 = bhat - r64 (r64 holds Mhat x on entry); sc.rr = ||r64||^2, sc.scale = ||r64||
// (red_out set: ||r64||^2 is written to red_out[4 s] instead of the scalars)
void outer_residual(const Batch& b64, char* bhat, char* r64, KScal* sc, RedBuf& rb, cudaStream_t st,
                    double* red_out = nullptr);
// lo = r / scale (converted to the inner precision); r is FP64, or split FP64
// when split is set
void outer_downcast(const Batch& b64, const Batch& bP, const char* r64, char* lo, const KScal* sc, cudaStream_t st,
                    bool split = false);
// x64 += scale * e (e in the inner precision); with x_split, also refresh the
// split-FP64 copy of x (hi/lo FP32 pairs) used by the double-float defects;
// x64 may be null when the split copy is the only iterate
void outer_accumulate(const Batch& b64, const Batch& bP, char* x64, const char* e, const KScal* sc, cudaStream_t st,
                      char* x_split = nullptr);
// r_s = bhat_s - m_s in double-float (m_s may be null), split-FP64 output, with
// sc.rr = ||r_s||^2 and sc.scale = ||r_s||
void split_residual(const Batch& b64, char* bhat_s, char* m_s, char* r_s, KScal* sc, RedBuf& rb, cudaStream_t st);
// v *= sc[s].scale (FP64, in place; not stored when keep64 is false) and, when
// out is given, out = its split-FP64 copy
void scale_split(const Batch& b64, char* v, char* out, KScal* sc, cudaStream_t st, bool keep64 = true);
// out (FP32, batch b32) = in (FP16 or FP32, batch bin)
void to_f32(const Batch& bin, const Batch& b32, const char* in, char* out, cudaStream_t st);
// r_s -= scale * m32 (split-FP64 defect, FP32 m = Mhat e), with the new
// ||r_s||^2 and ||r_s|| in the scalars (scale is read before it is replaced)
void defect_update(const Batch& b64, const Batch& b32, char* r_s, const char* m32, KScal* sc, RedBuf& rb,
                   cudaStream_t st);
// Odd half of the final FP64 check: h = kappa H_oe x_e given, x_o = A_oo^-1
// (b_o + h) written, ||b_o - (A_oo x_o - h)||^2 into sc.rr
void odd_reconstruct(const Batch& b64, bool clover, const char* bo, const char* h, char* xo, KScal* sc, RedBuf& rb,
                     cudaStream_t st);

}  // namespace bpp
