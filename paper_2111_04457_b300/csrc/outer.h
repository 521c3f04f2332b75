// Outer-loop (FP64 defect correction) decisions as single-warp device kernels,
// shared by the host-driven solve (which reads the flags back and launches the
// chosen branch) and the whole-solve CUDA graph (which branches with
// conditional nodes on the same flags), so both make identical decisions.
#pragma once

#include "blas.h"
#include "bpp_internal.h"

namespace bpp {

// Per-system outer-loop state.
struct OuterDev {
    double rr_e;       // ||even defect||^2 (relative to ||b|| = 1)
    double rr_o;       // ||odd part of b - D x||^2 after a full residual
    double target;     // Schur-residual target
    double drift;      // accumulated error estimate of reliable updates
    double pred;       // defect predicted by the last inner solve
    double true_res;   // last full true residual
    double bnorm2;     // 1 for a nonzero right-hand side, 0 for b = 0
    int status, conv, active, outer, inner_it, pad;
};

// Batch-wide outer-loop state and settings.
struct OuterCtl {
    double tol, inner_tol, eps32;
    int n, max_outer, max_passes, max_inner, prec, split, reliable;
    int have_full, defect_split, passes, did_work, check, inner, branch, cont;
    int n_full, n_rel, n_schur, n_inner;
};

enum OuterBranch { OB_FULL = 0, OB_RELIABLE = 1, OB_SCHUR = 2 };

// Kernel launchers; a handle of 0 means "no graph: do not set a condition".
void oc_classify(OuterDev* od, OuterCtl* oc, unsigned long long h_check, unsigned long long h_inner, cudaStream_t st);
void oc_full_odd(OuterDev* od, const KScal* s64, int n, cudaStream_t st);
void oc_full_even(OuterDev* od, OuterCtl* oc, KScal* s64, cudaStream_t st, bool split = false);
void oc_inner_setup(OuterDev* od, OuterCtl* oc, KScal* s64, KScal* sP, unsigned long long h_split, cudaStream_t st);
void oc_decide(OuterDev* od, OuterCtl* oc, const KScal* sP, unsigned long long h_branch, cudaStream_t st);
void oc_after_reliable(OuterDev* od, OuterCtl* oc, const KScal* s64, cudaStream_t st);
void oc_after_schur(OuterDev* od, OuterCtl* oc, const KScal* s64, cudaStream_t st);
void oc_loop(OuterCtl* oc, unsigned long long h_outer, cudaStream_t st);

}  // namespace bpp
