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
};

// out_p = epilogue(a * hop_{p,1-p} in) over every system of the batch.
void hop(const Batch& b, int parity, int dag, int mode, double a_sign, char* in, char* out, char* y,
         cudaStream_t st, const int* done = nullptr, int done_stride = 0);
double hop_bytes_per_site(int prec, int mode);

// ----------------------------------------------------------------------------- layout
// Canonical complex (double2 when c64 == 0... see layout.cu) <-> internal.
// Full canonical fields [nsys][V][4][3] -> internal even and odd halves.
void full_to_eo(const Batch& b, int sys0, int nsys, const void* canon, int canon_f64, int64_t canon_sys_stride,
                char* even, char* odd, int gamma5, cudaStream_t st);
void eo_to_full(const Batch& b, int sys0, int nsys, const char* even, const char* odd, void* canon, int canon_f64,
                int64_t canon_sys_stride, int gamma5, cudaStream_t st, double scale = 1.0);
// Half canonical fields [nsys][Vh][4][3] <-> internal half fields.
void half_to_int(const Batch& b, const void* canon, int canon_f64, char* out, cudaStream_t st);
void int_to_half(const Batch& b, const char* in, void* canon, int canon_f64, cudaStream_t st);

// ----------------------------------------------------------------------------- clover
void clover_build(Gauge& G, double kappa, double csw, cudaStream_t st);
// out = A in or A^-1 in on parity p for every system.
void clover_apply(const Batch& b, int parity, int inverse, char* in, char* out, cudaStream_t st);

}  // namespace bpp
