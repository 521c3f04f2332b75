// Deterministic per-system reductions shared by the vector kernels and the
// hopping kernel's fused epilogues: block sums in FP64, per-block partials,
// and the last block of each system (found with a ticket counter) summing the
// partials in block order and deriving the solver scalars.
#pragma once

#include "blas.h"
#include "bpp_internal.h"

namespace bpp {

__host__ __device__ __forceinline__ double2 c2(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) { return c2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cdiv2(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return c2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }


template <class real>
__device__ __forceinline__ void dot12(const cx<real> a[12], const cx<real> b[12], real& re, real& im) {
    re = 0; im = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        re = fma(a[k].r, b[k].r, re); re = fma(a[k].i, b[k].i, re);
        im = fma(a[k].r, b[k].i, im); im = fma(-a[k].i, b[k].r, im);
    }
}
template <class real>
__device__ __forceinline__ real norm12(const cx<real> a[12]) {
    real n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) { n = fma(a[k].r, a[k].r, n); n = fma(a[k].i, a[k].i, n); }
    return n;
}

struct RedCtx {
    BlockMap map;
    double* partials;
    unsigned* tickets;
};

// Block-wide sum of NR doubles, then the last block of system s sums all the
// system's block partials in block order; returns true in every thread of
// that last block, with tot[] valid in thread 0.
// The per-thread values and the warp-level sums use type T (FP32 for the
// FP32 / FP16 vectors: on this GPU every FP64 add runs on the slow FP64
// pipe), the per-warp results and everything after them FP64.
template <int NR, class T>
__device__ bool reduce_sys(const RedCtx& bp, int s, const T v[NR], double tot[NR]) {
    __shared__ double sh[32][NR];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        T a = v[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[warp][k] = (double)a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            double a = 0.0;
            for (int w = 0; w < nw; ++w) a += sh[w][k];
            bp.partials[(size_t)blockIdx.x * NR + k] = a;
        }
        __threadfence();
        const int nb = bp.map.uniform ? bp.map.tiles_per_sys : bp.map.tile_start[s + 1] - bp.map.tile_start[s];
        const unsigned t = atomicAdd(&bp.tickets[s], 1u);
        last = (t == (unsigned)(nb - 1));
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const int nb = bp.map.uniform ? bp.map.tiles_per_sys : bp.map.tile_start[s + 1] - bp.map.tile_start[s];
    double a[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) a[k] = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const int blk = bp.map.uniform ? s + bp.map.nsys * t : bp.map.tile_start[s] + t;
#pragma unroll
        for (int k = 0; k < NR; ++k) a[k] += __ldcg(&bp.partials[(size_t)blk * NR + k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        double b = a[k];
        for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
        if (lane == 0) sh[warp][k] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            double b = 0.0;
            for (int w = 0; w < nw; ++w) b += sh[w][k];
            tot[k] = b;
        }
        bp.tickets[s] = 0u;
    }
    return true;
}


// alpha = rho / <rhat, v> (BiCGStab), from the reduced <rhat, v>.
__device__ __forceinline__ void finalize_alpha(KScal& k, double re, double im) {
    k.rv = c2(re, im);
    if (cabs2(k.rv) == 0.0 || !isfinite(k.rv.x)) { k.status = 1; k.done = 1; k.alpha = c2(0, 0); }
    else k.alpha = cdiv2(k.rho, k.rv);
}

// omega = <t, s> / <t, t> (BiCGStab).
__device__ __forceinline__ void finalize_omega(KScal& k, double re, double im, double tt) {
    k.ts = c2(re, im);
    k.tt = tt;
    k.omega = k.tt > 0.0 ? c2(k.ts.x / k.tt, k.ts.y / k.tt) : c2(0.0, 0.0);
}

}  // namespace bpp
