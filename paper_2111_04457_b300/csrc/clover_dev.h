// Device access to the packed clover blocks: two 6x6 Hermitian chiral blocks
// per site (spins 0,1 and spins 2,3; in-block index spin*3 + colour), each
// stored as 6 real diagonal entries followed by the 15 complex strictly-lower
// entries in row order (1,0),(2,0),(2,1),(3,0),...,(5,4).
#pragma once

#include "bpp_internal.h"

namespace bpp {

template <int P> struct CloverAccess;

template <> struct CloverAccess<P64> {
    static __device__ __forceinline__ void load_block(const CloverView& c, int64_t i, int blk, double r[36]) {
        const double2* p = static_cast<const double2*>(c.data);
#pragma unroll
        for (int j = 0; j < 18; ++j) {
            double2 v = __ldg(p + (blk * 18 + j) * c.stride + i);
            r[2 * j] = v.x;
            r[2 * j + 1] = v.y;
        }
    }
};
template <> struct CloverAccess<P32> {
    static __device__ __forceinline__ void load_block(const CloverView& c, int64_t i, int blk, float r[36]) {
        const float4* p = static_cast<const float4*>(c.data);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            float4 v = __ldg(p + (blk * 9 + j) * c.stride + i);
            r[4 * j] = v.x; r[4 * j + 1] = v.y; r[4 * j + 2] = v.z; r[4 * j + 3] = v.w;
        }
    }
};
template <> struct CloverAccess<P16> {
    static __device__ __forceinline__ void load_block(const CloverView& c, int64_t i, int blk, float r[36]) {
        const uint4* p = static_cast<const uint4*>(c.data);
        float h[40];
        const int first = blk == 0 ? 0 : 4;     // block 1 starts half way into plane 4
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            uint4 v = __ldg(p + (first + j) * c.stride + i);
            float2 a = h2f(v.x), b = h2f(v.y), cc = h2f(v.z), d = h2f(v.w);
            h[8 * j + 0] = a.x; h[8 * j + 1] = a.y; h[8 * j + 2] = b.x; h[8 * j + 3] = b.y;
            h[8 * j + 4] = cc.x; h[8 * j + 5] = cc.y; h[8 * j + 6] = d.x; h[8 * j + 7] = d.y;
        }
        const int off = blk == 0 ? 0 : 4;
#pragma unroll
        for (int k = 0; k < 36; ++k) r[k] = h[off + k];
    }
};

template <> struct CloverAccess<P64S> {
    static __device__ __forceinline__ void load_block(const CloverView& c, int64_t i, int blk, df64 r[36]) {
        const float4* p = static_cast<const float4*>(c.data);
#pragma unroll
        for (int j = 0; j < 18; ++j) {
            float4 v = __ldg(p + (blk * 18 + j) * c.stride + i);
            r[2 * j] = df64(v.x, v.y);
            r[2 * j + 1] = df64(v.z, v.w);
        }
    }
};

// out = A in for one packed 6x6 Hermitian block r[36].
template <class real>
__device__ __forceinline__ void herm6_apply(const real r[36], const cx<real> in[6], cx<real> out[6]) {
#pragma unroll
    for (int row = 0; row < 6; ++row) out[row] = r[row] * in[row];
#pragma unroll
    for (int row = 1; row < 6; ++row)
#pragma unroll
        for (int col = 0; col < row; ++col) {
            const int k = row * (row - 1) / 2 + col;
            const cx<real> o = mkc(r[6 + 2 * k], r[7 + 2 * k]);
            cfma(out[row], o, in[col]);     // A[row][col] = o
            cfmac(out[col], o, in[row]);    // A[col][row] = conj(o)
        }
}

// out = A in on a full spinor (both chiral blocks).
template <int P, class real>
__device__ __forceinline__ void clover_apply_site(const CloverView& c, int64_t i, const cx<real> in[12], cx<real> out[12]) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        real r[36];
        CloverAccess<P>::load_block(c, i, blk, r);
        herm6_apply<real>(r, in + 6 * blk, out + 6 * blk);
    }
}

}  // namespace bpp
