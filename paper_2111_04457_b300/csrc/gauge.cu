// Gauge handle: conversion of canonical links to the internal even-odd
// structure-of-arrays layout in FP64, FP32 and FP16, and batch builders.
#include <cstdlib>
#include <cstring>

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

// Largest deviation of any link from SU(3): |U U^dag - 1| and
// |row3 - conj(row1 x row2)| (FP64, as an ordered float bit pattern: the
// values are non-negative).
__global__ void k_links_su3_dev(int64_t n, const double2* __restrict__ U, unsigned* maxdev) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float dev = 0.f;
    if (t < n) {
        cx<double> u[9];
        for (int k = 0; k < 9; ++k) u[k] = mkc(U[t * 9 + k].x, U[t * 9 + k].y);
        double m = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                cx<double> s = mkc(0.0, 0.0);
                for (int k = 0; k < 3; ++k) s = s + cmulc(u[3 * b + k], u[3 * a + k]);   // (U U^dag)_ab
                m = fmax(m, fabs(s.r - (a == b ? 1.0 : 0.0)) + fabs(s.i));
            }
        const cx<double> r0 = u[1] * u[5] - u[2] * u[4], r1 = u[2] * u[3] - u[0] * u[5], r2 = u[0] * u[4] - u[1] * u[3];
        m = fmax(m, fabs(u[6].r - r0.r) + fabs(u[6].i + r0.i));
        m = fmax(m, fabs(u[7].r - r1.r) + fabs(u[7].i + r1.i));
        m = fmax(m, fabs(u[8].r - r2.r) + fabs(u[8].i + r2.i));
        dev = isfinite(m) ? (float)m : 3.0e38f;
    }
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_down_sync(0xffffffffu, dev, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxdev, __float_as_uint(dev));
}

template <int P> struct Link12Store;
template <> struct Link12Store<P32> {
    static __device__ void store(void* base, int64_t stride, int64_t i, const double2 m[9]) {
        float4* p = static_cast<float4*>(base);
        for (int k = 0; k < 3; ++k)
            p[k * stride + i] = make_float4((float)m[2 * k].x, (float)m[2 * k].y, (float)m[2 * k + 1].x, (float)m[2 * k + 1].y);
    }
};
template <int P>
__global__ void k_links_in12(Geom g, const double2* __restrict__ U, void* out, int64_t stride, size_t field_bytes) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)8 * g.Vh) return;
    const int i = (int)(t % g.Vh);
    const int pm = (int)(t / g.Vh);
    const int p = pm >> 2, mu = pm & 3;
    int x[4];
    eo_coords(g, i, p, x);
    const int64_t lex = 2 * (int64_t)i + (x[0] & 1);
    const int64_t V = 2 * (int64_t)g.Vh;
    double2 m[9];
    for (int k = 0; k < 9; ++k) m[k] = U[((int64_t)mu * V + lex) * 9 + k];
    Link12Store<P>::store(static_cast<char*>(out) + (size_t)pm * field_bytes, stride, i, m);
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
    // SU(3) check (to 1e-10): the two-row FP32 links are kept only then
    DevBuf dev(sizeof(unsigned), s);
    BPP_CUDA(cudaMemsetAsync(dev.p, 0, sizeof(unsigned), s));
    const int64_t nl = 4 * G.V;
    k_links_su3_dev<<<(unsigned)((nl + B - 1) / B), B, 0, s>>>(nl, static_cast<const double2*>(U_dev), dev.as<unsigned>());
    count_launch();
    BPP_CHECK_LAUNCH();
    unsigned bits = 0;
    BPP_CUDA(cudaMemcpyAsync(&bits, dev.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    BPP_CUDA(cudaStreamSynchronize(s));
    float maxdev;
    std::memcpy(&maxdev, &bits, sizeof(float));
    G.su3 = maxdev <= 1e-10f;
    if (!G.su3) return;
    BPP_CUDA(cudaMalloc(&G.links12[P32], 8 * link12_alloc_bytes(P32, G.stride)));
    k_links_in12<P32><<<grid, B, 0, s>>>(G.g, static_cast<const double2*>(U_dev), G.links12[P32], G.stride, link12_alloc_bytes(P32, G.stride));
    count_launch();
    BPP_CHECK_LAUNCH();
}

bool link_compression(const Gauge& G, int prec) {
    if (!G.su3 || prec != P32 || !G.links12[prec]) return false;
    const char* e = std::getenv("BPP_LINK_COMPRESSION");
    return !(e && e[0] == '0');
}

void batch_add(Batch& b, const Gauge& G, double kappa, bool clover) {
    BPP_REQUIRE(!b.comp || link_compression(G, b.prec), BPP_ERR_INVALID_ARG,
                "two-row links requested for a gauge field that is not SU(3)");
    SysDesc d;
    d.g = G.g;
    for (int p = 0; p < 2; ++p)
        for (int mu = 0; mu < 4; ++mu) d.U[p][mu] = b.comp ? link12_view(G, b.prec, p, mu) : link_view(G, b.prec, p, mu);
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
