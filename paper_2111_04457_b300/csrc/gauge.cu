// Gauge handle: conversion of canonical links to the internal even-odd
// structure-of-arrays layout in FP64, FP32 and FP16, and batch builders.
#include "gauge.h"
#include "kernels.h"

namespace bpp {

template <int P> struct LinkStore;
template <> struct LinkStore<P64> {
    static __device__ void store(void* base, int64_t stride, int64_t i, const double2 m[9]) {
        double2* p = static_cast<double2*>(base);
        for (int k = 0; k < 9; ++k) p[k * stride + i] = m[k];
    }
};
template <> struct LinkStore<P32> {
    static __device__ void store(void* base, int64_t stride, int64_t i, const double2 m[9]) {
        float4* p = static_cast<float4*>(base);
        for (int k = 0; k < 4; ++k)
            p[k * stride + i] = make_float4((float)m[2 * k].x, (float)m[2 * k].y, (float)m[2 * k + 1].x, (float)m[2 * k + 1].y);
        float2* q = reinterpret_cast<float2*>(p + 4 * stride);
        q[i] = make_float2((float)m[8].x, (float)m[8].y);
    }
};
template <> struct LinkStore<P16> {
    static __device__ void store(void* base, int64_t stride, int64_t i, const double2 m[9]) {
        uint4* p = static_cast<uint4*>(base);
        for (int k = 0; k < 2; ++k) {
            uint4 v;
            v.x = f2h((float)m[4 * k].x, (float)m[4 * k].y);
            v.y = f2h((float)m[4 * k + 1].x, (float)m[4 * k + 1].y);
            v.z = f2h((float)m[4 * k + 2].x, (float)m[4 * k + 2].y);
            v.w = f2h((float)m[4 * k + 3].x, (float)m[4 * k + 3].y);
            p[k * stride + i] = v;
        }
        unsigned int* q = reinterpret_cast<unsigned int*>(p + 2 * stride);
        q[i] = f2h((float)m[8].x, (float)m[8].y);
    }
};

template <> struct LinkStore<P64S> {
    static __device__ void store(void* base, int64_t stride, int64_t i, const double2 m[9]) {
        float4* p = static_cast<float4*>(base);
        for (int k = 0; k < 9; ++k) {
            const df64 re(m[k].x), im(m[k].y);
            p[k * stride + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
};

// One thread per (half-lattice site i, parity p, direction mu).
template <int P>
__global__ void k_links_in(Geom g, const double2* __restrict__ U, void* out, int64_t stride, size_t field_bytes) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)8 * g.Vh) return;
    const int i = (int)(t % g.Vh);
    const int pm = (int)(t / g.Vh);       // parity * 4 + mu
    const int p = pm >> 2, mu = pm & 3;
    int x[4];
    eo_coords(g, i, p, x);
    const int64_t lex = 2 * (int64_t)i + (x[0] & 1);
    const int64_t V = 2 * (int64_t)g.Vh;
    double2 m[9];
    for (int k = 0; k < 9; ++k) m[k] = U[((int64_t)mu * V + lex) * 9 + k];
    LinkStore<P>::store(static_cast<char*>(out) + (size_t)pm * field_bytes, stride, i, m);
}

void links_to_internal(Gauge& G, const void* U_dev, cudaStream_t s) {
    const int64_t n = 8 * G.Vh;
    const int B = 256;
    const int grid = (int)((n + B - 1) / B);
    k_links_in<P64><<<grid, B, 0, s>>>(G.g, static_cast<const double2*>(U_dev), G.links[P64], G.stride, link_alloc_bytes(P64, G.stride));
    k_links_in<P32><<<grid, B, 0, s>>>(G.g, static_cast<const double2*>(U_dev), G.links[P32], G.stride, link_alloc_bytes(P32, G.stride));
    k_links_in<P16><<<grid, B, 0, s>>>(G.g, static_cast<const double2*>(U_dev), G.links[P16], G.stride, link_alloc_bytes(P16, G.stride));
    k_links_in<P64S><<<grid, B, 0, s>>>(G.g, static_cast<const double2*>(U_dev), G.links[P64S], G.stride, link_alloc_bytes(P64S, G.stride));
    count_launch(4);
    BPP_CHECK_LAUNCH();
}

void batch_add(Batch& b, const Gauge& G, double kappa, bool clover) {
    SysDesc d;
    d.g = G.g;
    for (int p = 0; p < 2; ++p)
        for (int mu = 0; mu < 4; ++mu) d.U[p][mu] = link_view(G, b.prec, p, mu);
    for (int p = 0; p < 2; ++p) {
        d.A[p] = clover ? clover_view(G, b.prec, 0, p) : CloverView{nullptr, G.stride};
        d.Ainv[p] = clover ? clover_view(G, b.prec, 1, p) : CloverView{nullptr, G.stride};
    }
    d.kappa = kappa;
    d.stride = G.stride;
    d.vec_off = (int64_t)b.vec_bytes;
    b.vec_bytes += spinor_alloc_bytes(b.prec, G.stride);
    if (!b.sys.empty() && b.sys[0].g.Vh != G.g.Vh) b.uniform = false;
    if (G.g.Vh > b.Vh_max) b.Vh_max = G.g.Vh;
    b.sys.push_back(d);
}

BlockMap block_map(const Batch& b, int spb, int& nblocks) {
    BlockMap m;
    m.nsys = b.nsys();
    BPP_REQUIRE(m.nsys >= 1 && m.nsys <= MAXSYS, BPP_ERR_INVALID_ARG, "batch size must be 1..64");
    m.uniform = b.uniform ? 1 : 0;
    m.tiles_per_sys = (b.Vh_max + spb - 1) / spb;
    int acc = 0;
    for (int s = 0; s < m.nsys; ++s) {
        m.tile_start[s] = acc;
        acc += (b.sys[s].g.Vh + spb - 1) / spb;
    }
    m.tile_start[m.nsys] = acc;
    for (int s = m.nsys + 1; s <= MAXSYS; ++s) m.tile_start[s] = acc;
    nblocks = m.uniform ? m.tiles_per_sys * m.nsys : acc;
    return m;
}

}  // namespace bpp
