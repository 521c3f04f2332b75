// Launchers shared between the library's translation units.
#pragma once

#include "bpp_internal.h"
#include "gauge.h"

namespace bpp {

// ----------------------------------------------------------------------------- gauge
void links_to_internal(Gauge& G, const void* U_dev, cudaStream_t s);

// ----------------------------------------------------------------------------- hopping term
enum HopMode { HOP_PLAIN = 0, HOP_XPAY = 1, HOP_CLOV_XPAY = 2, HOP_INV = 3, HOP_INV_XPAY = 4 };

struct HopParams {
    const SysDesc* sys;
    BlockMap map;
    int parity;        // parity of the output sites
    char* in;          // batch vector on parity 1 - parity
    char* out;         // batch vector on parity
    char* y;           // batch vector on parity (xpay operand) or null
    double a_sign;     // a = a_sign * kappa of the system
    const int* done;   // optional per-system "converged" flags (skip those systems)
    int done_stride;   // ints between consecutive flags
    // domain decomposition in x4 (HopDD launches only): the t-direction hops
    // of the face sites take their neighbour terms from the face buffers of
    // the adjacent domains, [system][6 complex][face site] in the arithmetic
    // type of the precision
    const void* halo_fwd;          // projected half spinors of the upper domain's bottom face
    const void* halo_bwd;          // link-multiplied half spinors of the lower domain's top face
    const float* halo_fwd_scale;   // FP16: the upper domain's per-site spinor scales [system][face site]
    int64_t face;                  // face sites of one parity: L1/2 L2 L3
    int flip_top, flip_bot;        // the boundary sign applies at the top / bottom face
    // BiCGStab inner products fused into an XPAY / CLOV_XPAY epilogue (see
    // HopRed): HRED_NONE, HRED_ALPHA or HRED_OMEGA
    int red_op = 0;
    const char* red_rhat = nullptr;   // HRED_ALPHA: rhat, a batch vector on the output parity
    double* red_part = nullptr;       // per-warp partial sums [system][red_wstride][4]
    int red_wstride = 0;              // warps per system in red_part: (Vh_max + 31) / 32
};

// Inner products of the BiCGStab iteration computed by the second hop of a
// Schur application from the values it stores (FP16: as they will read back):
//   HRED_ALPHA  <rhat, out>               (out = v = Mhat p)
//   HRED_OMEGA  <out, y>, ||out||^2       (out = t = Mhat s, y = s)
// Each warp of 32 consecutive sites of one system sums its sites in the
// arithmetic type of the precision and writes one FP64 partial; hop_red_fin
// then sums a system's partials in warp order.  The order of the sums depends
// only on the lattice, not on the hopping kernel's block size or the number
// of right-hand sides per thread, so batched and single solves stay
// bit-identical.
enum HopRedOp { HRED_NONE = 0, HRED_ALPHA = 1, HRED_OMEGA = 2 };
struct HopRed {
    int op = HRED_NONE;
    const char* rhat = nullptr;
    double* part = nullptr;
    int wstride = 0;
};

// Face buffers and boundary signs of one domain of a decomposition in x4.
struct HopDD {
    const void* fwd = nullptr;
    const void* bwd = nullptr;
    const float* fwd_scale = nullptr;
    int64_t face = 0;
    int flip_top = 0, flip_bot = 0;
};

// out_p = epilogue(a * hop_{p,1-p} in) over every system of the batch.
void hop(const Batch& b, int parity, int dag, int mode, double a_sign, char* in, char* out, char* y,
         cudaStream_t st, const int* done = nullptr, int done_stride = 0, const HopRed* red = nullptr);
double hop_bytes_per_site(int prec, int mode);
// The hopping term on one domain of a decomposition in x4 (FP64 / FP32 /
// FP16): as hop(), with the t-direction neighbour terms of the face sites
// from the face buffers in dd (the batch's geometry is the domain's, with
// bc[3] = +1; dd carries the boundary sign).
void hop_dd(const Batch& b, int parity, int dag, int mode, double a_sign, char* in, char* out, char* y,
            const HopDD& dd, cudaStream_t st, const int* done = nullptr, int done_stride = 0);
// Face buffers of the input field `in` (parity 1 - parity of the hop that
// follows): send_down[s] = the (1 + SF gamma_4) projections of the bottom face
// (x4 = 0), send_up[s] = U_4^dag (1 - SF gamma_4) projections of the top face,
// SF = -1 (D) or +1 (D^dag); FP16 also writes the bottom face's spinor scales.
void dd_pack(const Batch& b, int in_parity, int dag, const char* in, void* send_down, float* send_down_scale,
             void* send_up, int64_t face, cudaStream_t st);

// ----------------------------------------------------------------------------- layout
// Canonical complex (double2 when c64 == 0... see layout.cu) <-> internal.
// Full canonical fields [nsys][V][4][3] -> internal even and odd halves.
void full_to_eo(const Batch& b, int sys0, int nsys, const void* canon, int canon_f64, int64_t canon_sys_stride,
                char* even, char* odd, int gamma5, cudaStream_t st);
void eo_to_full(const Batch& b, int sys0, int nsys, const char* even, const char* odd, void* canon, int canon_f64,
                int64_t canon_sys_stride, int gamma5, cudaStream_t st, double scale = 1.0);
// Half canonical fields [nsys][Vh][4][3] <-> internal half fields.
// cstride: complex elements between the systems' canonical fields (< 0: Vh * 12).
void half_to_int(const Batch& b, const void* canon, int canon_f64, char* out, cudaStream_t st, int64_t cstride = -1);
void int_to_half(const Batch& b, const char* in, void* canon, int canon_f64, cudaStream_t st, int64_t cstride = -1);

// ----------------------------------------------------------------------------- clover
void clover_build(Gauge& G, double kappa, double csw, cudaStream_t st);
// out = A in or A^-1 in on parity p for every system.
void clover_apply(const Batch& b, int parity, int inverse, char* in, char* out, cudaStream_t st);

}  // namespace bpp
