// Outer-loop control kernels (see outer.h).  Each runs as one warp; lane 0
// walks the systems (at most 64) in order, so the decisions are the same in the
// host-driven and the graph-driven solve.
#include <cmath>

#include "outer.h"

namespace bpp {

static __device__ __forceinline__ void set_cond(unsigned long long h, unsigned v) {
    if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

// Which systems still need work: converged by a full residual, waiting for a
// confirming full residual, or active for another correction.
__global__ void k_oc_classify(OuterDev* od, OuterCtl* oc, unsigned long long h_check, unsigned long long h_inner) {
    if (threadIdx.x != 0) return;
    bool need_check = false, any_active = false;
    for (int s = 0; s < oc->n; ++s) {
        OuterDev& d = od[s];
        d.active = 0;
        if (d.status != BPP_OK || d.conv) continue;
        const double rr = d.rr_e + (oc->have_full ? d.rr_o : 0.0);
        if (!isfinite(rr)) { d.status = BPP_ERR_NONFINITE; continue; }
        if (d.bnorm2 == 0.0) { d.conv = 1; d.true_res = 0.0; continue; }
        const double rel = sqrt(rr / d.bnorm2);
        if (oc->have_full) {
            d.true_res = rel;
            if (rel <= oc->tol) { d.conv = 1; continue; }
            if (rel <= d.target) d.target *= 0.5 * oc->tol / rel;   // Schur target met but not the true one
        } else if (rel <= d.target) {
            need_check = true;                                   // confirm with the full residual
            continue;
        }
        if (d.outer >= oc->max_outer) continue;
        d.active = 1;
        any_active = true;
    }
    const int check = need_check && !oc->have_full;
    const int inner = !check && any_active;
    oc->check = check;
    oc->inner = inner;
    oc->did_work = check || inner;
    set_cond(h_check, check);
    set_cond(h_inner, inner);
}

// The odd part of the final check came first (its norm is in the scalars)...
__global__ void k_oc_full_odd(OuterDev* od, const KScal* s64, int n) {
    if (threadIdx.x != 0) return;
    for (int s = 0; s < n; ++s) od[s].rr_o = s64[s].rr;
}

// ... then the even part, whose norm stays in the scalars for the downcast of
// a further correction.  split: the double-float check, whose even defect is
// split-FP64 and whose odd half vanishes by construction (x_o is A_oo^-1 of
// b_o + kappa H_oe x_e itself), so it is not recomputed.
__global__ void k_oc_full_even(OuterDev* od, OuterCtl* oc, KScal* s64, int split) {
    if (threadIdx.x != 0) return;
    for (int s = 0; s < oc->n; ++s) {
        od[s].rr_e = s64[s].rr;
        if (split) od[s].rr_o = 0.0;
        s64[s].scale = sqrt(fmax(od[s].rr_e, 0.0));
    }
    oc->have_full = 1;
    oc->defect_split = split;
    oc->n_full += 1;
}

// Scale of each defect and the inner tolerance of each system.
__global__ void k_oc_inner_setup(OuterDev* od, OuterCtl* oc, KScal* s64, KScal* sP, unsigned long long h_split) {
    if (threadIdx.x != 0) return;
    for (int s = 0; s < oc->n; ++s) {
        const OuterDev& d = od[s];
        const double rn = sqrt(fmax(d.rr_e, 0.0));
        s64[s].rr = d.rr_e;
        s64[s].scale = d.active ? rn : 0.0;
        const double need = 0.5 * d.target * sqrt(d.bnorm2) / fmax(rn, 1e-300);
        // inner_tol <= 0: per-precision default (FP32 1e-6, FP16 2e-3)
        const double dflt = oc->prec == P32 ? 1e-6 : 2e-3;
        const double want = oc->inner_tol > 0.0 ? oc->inner_tol : dflt;
        const double itol = oc->prec == P64 ? need : fmax(want, need);
        KScal k = {};
        k.tol2 = itol * itol;
        k.max_iter = oc->max_inner;
        sP[s] = k;
    }
    oc->n_inner += 1;
    set_cond(h_split, oc->defect_split);
}

// After a correction: predicted defects, and the next defect's source: the full
// residual when every active system is predicted to converge, a reliable FP32
// update while its accumulated error stays below 1% of the predicted defect, a
// double-float recomputation otherwise.
__global__ void k_oc_decide(OuterDev* od, OuterCtl* oc, const KScal* sP, unsigned long long h_branch) {
    if (threadIdx.x != 0) return;
    bool all_predicted = true;
    for (int s = 0; s < oc->n; ++s) {
        OuterDev& d = od[s];
        if (!d.active) continue;
        d.outer += 1;
        d.inner_it += sP[s].iter;
        const double inner_rel = sP[s].bb > 0.0 ? sqrt(fmax(sP[s].rr, 0.0) / sP[s].bb) : 0.0;
        d.pred = sqrt(fmax(d.rr_e, 0.0)) * inner_rel;
        if (!(d.pred <= 0.5 * d.target * sqrt(d.bnorm2))) all_predicted = false;
    }
    bool reliable_ok = oc->reliable && oc->defect_split;
    for (int s = 0; s < oc->n; ++s) {
        const OuterDev& d = od[s];
        if (!d.active) continue;
        const double step = oc->eps32 * sqrt(fmax(d.rr_e, 0.0));
        if (!(d.drift + step <= 0.01 * d.pred)) reliable_ok = false;
    }
    const int branch = all_predicted ? OB_FULL : reliable_ok ? OB_RELIABLE : OB_SCHUR;
    oc->branch = branch;
    set_cond(h_branch, (unsigned)branch);
}

__global__ void k_oc_after_reliable(OuterDev* od, OuterCtl* oc, const KScal* s64) {
    if (threadIdx.x != 0) return;
    for (int s = 0; s < oc->n; ++s) {
        if (od[s].active) od[s].drift += oc->eps32 * sqrt(fmax(od[s].rr_e, 0.0));
        od[s].rr_e = s64[s].rr;
    }
    oc->have_full = 0;
    oc->n_rel += 1;
}

__global__ void k_oc_after_schur(OuterDev* od, OuterCtl* oc, const KScal* s64) {
    if (threadIdx.x != 0) return;
    for (int s = 0; s < oc->n; ++s) {
        od[s].drift = 0.0;
        od[s].rr_e = s64[s].rr;
    }
    oc->have_full = 0;
    oc->defect_split = oc->split;
    oc->n_schur += 1;
}

__global__ void k_oc_loop(OuterCtl* oc, unsigned long long h_outer) {
    if (threadIdx.x != 0) return;
    oc->passes += 1;
    oc->cont = oc->did_work && oc->passes < oc->max_passes;
    set_cond(h_outer, oc->cont);
}

#define OC_LAUNCH(...)                           \
    do {                                         \
        ProfScope prof_(PROF_CTL, 0.0, st);      \
        __VA_ARGS__;                             \
        count_launch();                          \
        BPP_CHECK_LAUNCH();                      \
    } while (0)

void oc_classify(OuterDev* od, OuterCtl* oc, unsigned long long hc, unsigned long long hi, cudaStream_t st) {
    OC_LAUNCH(k_oc_classify<<<1, 32, 0, st>>>(od, oc, hc, hi));
}
void oc_full_odd(OuterDev* od, const KScal* s64, int n, cudaStream_t st) {
    OC_LAUNCH(k_oc_full_odd<<<1, 32, 0, st>>>(od, s64, n));
}
void oc_full_even(OuterDev* od, OuterCtl* oc, KScal* s64, cudaStream_t st, bool split) {
    OC_LAUNCH(k_oc_full_even<<<1, 32, 0, st>>>(od, oc, s64, split ? 1 : 0));
}
void oc_inner_setup(OuterDev* od, OuterCtl* oc, KScal* s64, KScal* sP, unsigned long long hs, cudaStream_t st) {
    OC_LAUNCH(k_oc_inner_setup<<<1, 32, 0, st>>>(od, oc, s64, sP, hs));
}
void oc_decide(OuterDev* od, OuterCtl* oc, const KScal* sP, unsigned long long hb, cudaStream_t st) {
    OC_LAUNCH(k_oc_decide<<<1, 32, 0, st>>>(od, oc, sP, hb));
}
void oc_after_reliable(OuterDev* od, OuterCtl* oc, const KScal* s64, cudaStream_t st) {
    OC_LAUNCH(k_oc_after_reliable<<<1, 32, 0, st>>>(od, oc, s64));
}
void oc_after_schur(OuterDev* od, OuterCtl* oc, const KScal* s64, cudaStream_t st) {
    OC_LAUNCH(k_oc_after_schur<<<1, 32, 0, st>>>(od, oc, s64));
}
void oc_loop(OuterCtl* oc, unsigned long long ho, cudaStream_t st) {
    OC_LAUNCH(k_oc_loop<<<1, 32, 0, st>>>(oc, ho));
}

}  // namespace bpp
