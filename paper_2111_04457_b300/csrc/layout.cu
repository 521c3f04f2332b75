// Boundary layout conversion (the "interface object" of Sec. 3.3 that
// rearranges fields into a coalesced layout): canonical lexicographic complex
// arrays [nsys][V or Vh][4][3] (complex128 or complex64) <-> the internal
// per-parity structure-of-arrays half fields, with an optional gamma_5
// (= diag(-1,-1,1,1) in the chiral basis) applied on the way.
#include "bpp_internal.h"
#include "gauge.h"
#include "kernels.h"

namespace bpp {

template <class real> struct CanonT;
template <> struct CanonT<double> { using type = double2; };
template <> struct CanonT<float> { using type = float2; };

template <class TC, class real>
__device__ __forceinline__ cx<real> from_canon(TC v) { return mkc<real>((real)v.x, (real)v.y); }
template <class TC, class real>
__device__ __forceinline__ TC to_canon(cx<real> v);
template <> __device__ __forceinline__ double2 to_canon<double2, double>(cx<double> v) { return make_double2(v.r, v.i); }
template <> __device__ __forceinline__ double2 to_canon<double2, float>(cx<float> v) { return make_double2(v.r, v.i); }
template <> __device__ __forceinline__ float2 to_canon<float2, double>(cx<double> v) { return make_float2((float)v.r, (float)v.i); }
template <> __device__ __forceinline__ float2 to_canon<float2, float>(cx<float> v) { return make_float2(v.r, v.i); }
template <> __device__ __forceinline__ double2 to_canon<double2, df64>(cx<df64> v) {
    return make_double2(v.r.to_double(), v.i.to_double());
}
template <> __device__ __forceinline__ float2 to_canon<float2, df64>(cx<df64> v) {
    return make_float2((float)v.r.to_double(), (float)v.i.to_double());
}

// Parity of lexicographic site lex; its half-lattice index is lex / 2.
__device__ __forceinline__ int lex_parity(const Geom& g, int64_t lex) {
    const int x0 = (int)(lex % g.L[0]);
    int r = (int)(lex / g.L[0]);
    const int x1 = r % g.L[1];
    r /= g.L[1];
    return (x0 + x1 + r % g.L[2] + r / g.L[2]) & 1;
}

// Thread per lexicographic site of system sys0 + blockIdx.y: a warp reads 32
// consecutive canonical sites (both parities), so every line of the canonical
// field is read once.
template <int P, class TC>
__global__ void k_full_to_eo(const SysDesc* sys, int sys0, const TC* __restrict__ canon, int64_t cstride,
                             char* even, char* odd, int g5) {
    using real = typename PT<P>::real;
    const SysDesc& d = sys[sys0 + blockIdx.y];
    const Geom g = d.g;
    const int64_t lex = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (lex >= 2 * (int64_t)g.Vh) return;
    const int p = lex_parity(g, lex);
    const int i = (int)(lex >> 1);
    const TC* src = canon + blockIdx.y * cstride + lex * 12;
    cx<real> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        v[k] = from_canon<TC, real>(src[k]);
        if (g5 && k < 6) v[k] = -v[k];
    }
    Access<P>::store_spinor(sys_view<P>(p == 0 ? even : odd, d), i, v);
}

// Threads per block of k_eo_to_full (its shared staging buffer is sized for it).
constexpr int EO_B = 256;

// Thread per lexicographic site, as k_full_to_eo.  The block's 256
// consecutive canonical sites are one contiguous range of the output: each
// thread puts its site in shared memory, then the block writes the range with
// consecutive threads on consecutive 8- or 16-byte elements (whole sectors per
// store instruction instead of 16 bytes every 192).
template <int P, class TC>
__global__ void __launch_bounds__(EO_B) k_eo_to_full(const SysDesc* sys, int sys0, const char* even, const char* odd,
                                                     TC* canon, int64_t cstride, int g5, double scale) {
    using real = typename PT<P>::real;
    __shared__ TC stage[EO_B * 12];
    const SysDesc& d = sys[sys0 + blockIdx.y];
    const Geom g = d.g;
    const int64_t V = 2 * (int64_t)g.Vh;
    const int64_t lex0 = (int64_t)blockIdx.x * EO_B;
    if (lex0 >= V) return;   // whole block
    const int64_t lex = lex0 + threadIdx.x;
    if (lex < V) {
        const int p = lex_parity(g, lex);
        const int i = (int)(lex >> 1);
        cx<real> v[12];
        Access<P>::load_spinor(sys_view<P>(const_cast<char*>(p == 0 ? even : odd), d), i, v);
        TC* dst = stage + threadIdx.x * 12;
        if constexpr (P == P64S) {
            // split values convert to FP64 first and scale there: the scaled
            // solution may lie outside the FP32 exponent range
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cx<double> w = mkc(v[k].r.to_double() * scale, v[k].i.to_double() * scale);
                if (g5 && k < 6) w = -w;
                dst[k] = to_canon<TC, double>(w);
            }
        } else {
            if (scale != 1.0) {
                const real f = (real)scale;
#pragma unroll
                for (int k = 0; k < 12; ++k) v[k] = f * v[k];
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) dst[k] = to_canon<TC, real>((g5 && k < 6) ? -v[k] : v[k]);
        }
    }
    __syncthreads();
    const int n = (int)min((int64_t)EO_B, V - lex0) * 12;
    TC* out = canon + blockIdx.y * cstride + lex0 * 12;
    for (int j = threadIdx.x; j < n; j += EO_B) out[j] = stage[j];
}

// Half fields: canonical [nsys][Vh][4][3] with system s at offset s*Vh*12.
// cstride: elements of TC between systems (< 0: Vh * 12, consecutive fields).
template <int P, class TC>
__global__ void k_half_to_int(const SysDesc* sys, const TC* __restrict__ canon, char* out, int64_t cstride) {
    using real = typename PT<P>::real;
    const SysDesc& d = sys[blockIdx.y];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.g.Vh) return;
    const TC* src = canon + (int64_t)blockIdx.y * (cstride < 0 ? (int64_t)d.g.Vh * 12 : cstride) + i * 12;
    cx<real> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = from_canon<TC, real>(src[k]);
    Access<P>::store_spinor(sys_view<P>(out, d), i, v);
}

template <int P, class TC>
__global__ void k_int_to_half(const SysDesc* sys, const char* in, TC* canon, int64_t cstride) {
    using real = typename PT<P>::real;
    const SysDesc& d = sys[blockIdx.y];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.g.Vh) return;
    cx<real> v[12];
    Access<P>::load_spinor(sys_view<P>(const_cast<char*>(in), d), i, v);
    TC* dst = canon + (int64_t)blockIdx.y * (cstride < 0 ? (int64_t)d.g.Vh * 12 : cstride) + i * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = to_canon<TC, real>(v[k]);
}

#define BPP_PREC_DISPATCH(prec, ...)                                  \
    do {                                                              \
        if ((prec) == P64) { constexpr int PP = P64; __VA_ARGS__; }        \
        else if ((prec) == P32) { constexpr int PP = P32; __VA_ARGS__; }   \
        else if ((prec) == P16) { constexpr int PP = P16; __VA_ARGS__; }   \
        else { constexpr int PP = P64S; __VA_ARGS__; }                     \
    } while (0)

void full_to_eo(const Batch& b, int sys0, int nsys, const void* canon, int canon_f64, int64_t cstride,
                char* even, char* odd, int g5, cudaStream_t st) {
    const int B = 256;
    dim3 grid((unsigned)((2 * (int64_t)b.Vh_max + B - 1) / B), nsys);
    ProfScope prof(PROF_LAYOUT, 2.0 * b.sys[sys0].g.Vh * nsys * (spinor_bytes(b.prec) + (canon_f64 ? 192 : 96)), st);
    BPP_PREC_DISPATCH(b.prec, {
        if (canon_f64)
            k_full_to_eo<PP, double2><<<grid, B, 0, st>>>(b.dev(), sys0, static_cast<const double2*>(canon), cstride, even, odd, g5);
        else
            k_full_to_eo<PP, float2><<<grid, B, 0, st>>>(b.dev(), sys0, static_cast<const float2*>(canon), cstride, even, odd, g5);
    });
    count_launch();
    BPP_CHECK_LAUNCH();
}

void eo_to_full(const Batch& b, int sys0, int nsys, const char* even, const char* odd, void* canon, int canon_f64,
                int64_t cstride, int g5, cudaStream_t st, double scale) {
    const int B = EO_B;
    dim3 grid((unsigned)((2 * (int64_t)b.Vh_max + B - 1) / B), nsys);
    ProfScope prof(PROF_LAYOUT, 2.0 * b.sys[sys0].g.Vh * nsys * (spinor_bytes(b.prec) + (canon_f64 ? 192 : 96)), st);
    BPP_PREC_DISPATCH(b.prec, {
        if (canon_f64)
            k_eo_to_full<PP, double2><<<grid, B, 0, st>>>(b.dev(), sys0, even, odd, static_cast<double2*>(canon), cstride, g5, scale);
        else
            k_eo_to_full<PP, float2><<<grid, B, 0, st>>>(b.dev(), sys0, even, odd, static_cast<float2*>(canon), cstride, g5, scale);
    });
    count_launch();
    BPP_CHECK_LAUNCH();
}

void half_to_int(const Batch& b, const void* canon, int canon_f64, char* out, cudaStream_t st, int64_t cstride) {
    const int B = 256;
    dim3 grid((unsigned)((b.Vh_max + B - 1) / B), b.nsys());
    ProfScope prof(PROF_LAYOUT, b.sites() * (spinor_bytes(b.prec) + (canon_f64 ? 192 : 96)), st);
    BPP_PREC_DISPATCH(b.prec, {
        if (canon_f64) k_half_to_int<PP, double2><<<grid, B, 0, st>>>(b.dev(), static_cast<const double2*>(canon), out, cstride);
        else k_half_to_int<PP, float2><<<grid, B, 0, st>>>(b.dev(), static_cast<const float2*>(canon), out, cstride);
    });
    count_launch();
    BPP_CHECK_LAUNCH();
}

void int_to_half(const Batch& b, const char* in, void* canon, int canon_f64, cudaStream_t st, int64_t cstride) {
    const int B = 256;
    dim3 grid((unsigned)((b.Vh_max + B - 1) / B), b.nsys());
    ProfScope prof(PROF_LAYOUT, b.sites() * (spinor_bytes(b.prec) + (canon_f64 ? 192 : 96)), st);
    BPP_PREC_DISPATCH(b.prec, {
        if (canon_f64) k_int_to_half<PP, double2><<<grid, B, 0, st>>>(b.dev(), in, static_cast<double2*>(canon), cstride);
        else k_int_to_half<PP, float2><<<grid, B, 0, st>>>(b.dev(), in, static_cast<float2*>(canon), cstride);
    });
    count_launch();
    BPP_CHECK_LAUNCH();
}

}  // namespace bpp

namespace bpp {

// Half-field conversions for the non-allocating entry point: the system
// table (nsys systems of one lattice with Vh sites) is already on the device.
void half_to_int_fixed(int prec, const SysDesc* dsys, int nsys, int Vh, const void* canon, int canon_f64, char* out,
                       cudaStream_t st) {
    const int B = 256;
    dim3 grid((unsigned)((Vh + B - 1) / B), nsys);
    BPP_PREC_DISPATCH(prec, {
        if (canon_f64) k_half_to_int<PP, double2><<<grid, B, 0, st>>>(dsys, static_cast<const double2*>(canon), out, -1);
        else k_half_to_int<PP, float2><<<grid, B, 0, st>>>(dsys, static_cast<const float2*>(canon), out, -1);
    });
    count_launch();
}

void int_to_half_fixed(int prec, const SysDesc* dsys, int nsys, int Vh, const char* in, void* canon, int canon_f64,
                       cudaStream_t st) {
    const int B = 256;
    dim3 grid((unsigned)((Vh + B - 1) / B), nsys);
    BPP_PREC_DISPATCH(prec, {
        if (canon_f64) k_int_to_half<PP, double2><<<grid, B, 0, st>>>(dsys, in, static_cast<double2*>(canon), -1);
        else k_int_to_half<PP, float2><<<grid, B, 0, st>>>(dsys, in, static_cast<float2*>(canon), -1);
    });
    count_launch();
}

}  // namespace bpp
