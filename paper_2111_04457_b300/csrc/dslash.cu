// Even-odd hopping term of Eq. (1) (Sec. 3): for every site x of parity p,
//
//   hop(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu^dag(x-mu) psi(x-mu) ]
//
// (projectors swapped for the adjoint), with psi living on parity 1-p, and a
// fused epilogue that forms one of
//   PLAIN     out = a hop                      (a = +-kappa of the system)
//   XPAY      out = y + a hop
//   CLOV_XPAY out = A y + a hop                (A = 1 + F on parity p)
//   INV       out = A^-1 (a hop)
//   INV_XPAY  out = A^-1 (y + a hop)
//
// Each direction uses the chiral-basis structure gamma_mu = [[0, A_mu], [A_mu^dag, 0]]
// with A_k = i sigma_k, A_4 = 1: (1 + s gamma_mu) psi = (h, s A_mu^dag h) where
// h = u + s A_mu l (u, l the upper and lower spin pairs), so only the two-spin
// half spinor h is multiplied by the link and the lower half is rebuilt from
// U h with a few sign and i factors.  One thread per output site; neighbour
// spinors come through L1/L2 (each is read by 8 sites), links stream once.
#include <string>

#include "bpp_internal.h"
#include "clover_dev.h"
#include "gauge.h"
#include "hop_dev.h"
#include "kernels.h"
#include "reduce.h"

namespace bpp {

// Raw (undecoded) loads of one hop: the neighbour spinor and the link.
template <int P> struct Raw;
template <> struct Raw<P64> { double2 s[12]; double2 u[9]; };
template <> struct Raw<P32> { float4 s[6]; float4 u[4]; float2 u8; };
template <> struct Raw<P16> { uint4 s[3]; float sc; uint4 u[2]; unsigned u8; };
template <> struct Raw<P64S> { float4 s[12]; float4 u[9]; };

__device__ __forceinline__ void load_raw(Raw<P64>& r, const SpinorView& in, int64_t j, const LinkView& U, int64_t ju) {
    const double2* p = static_cast<const double2*>(in.data);
#pragma unroll
    for (int k = 0; k < 12; ++k) r.s[k] = __ldg(p + k * in.stride + j);
    const double2* q = static_cast<const double2*>(U.data);
#pragma unroll
    for (int k = 0; k < 9; ++k) r.u[k] = __ldcs(q + k * U.stride + ju);
}
__device__ __forceinline__ void load_raw(Raw<P32>& r, const SpinorView& in, int64_t j, const LinkView& U, int64_t ju) {
    const float4* p = static_cast<const float4*>(in.data);
#pragma unroll
    for (int k = 0; k < 6; ++k) r.s[k] = __ldg(p + k * in.stride + j);
    const float4* q = static_cast<const float4*>(U.data);
#pragma unroll
    for (int k = 0; k < 4; ++k) r.u[k] = __ldcs(q + k * U.stride + ju);
    r.u8 = __ldcs(reinterpret_cast<const float2*>(q + 4 * U.stride) + ju);
}
__device__ __forceinline__ void load_raw(Raw<P16>& r, const SpinorView& in, int64_t j, const LinkView& U, int64_t ju) {
    const uint4* p = static_cast<const uint4*>(in.data);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.s[k] = __ldg(p + k * in.stride + j);
    r.sc = __ldg(in.scale + j);
    const uint4* q = static_cast<const uint4*>(U.data);
#pragma unroll
    for (int k = 0; k < 2; ++k) r.u[k] = __ldcs(q + k * U.stride + ju);
    r.u8 = __ldcs(reinterpret_cast<const unsigned*>(q + 2 * U.stride) + ju);
}

__device__ __forceinline__ void load_raw(Raw<P64S>& r, const SpinorView& in, int64_t j, const LinkView& U, int64_t ju) {
    const float4* p = static_cast<const float4*>(in.data);
#pragma unroll
    for (int k = 0; k < 12; ++k) r.s[k] = __ldg(p + k * in.stride + j);
    const float4* q = static_cast<const float4*>(U.data);
#pragma unroll
    for (int k = 0; k < 9; ++k) r.u[k] = __ldcs(q + k * U.stride + ju);
}
__device__ __forceinline__ void decode(const Raw<P64S>& r, cx<df64> psi[12], cx<df64> u[9]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) psi[k] = mkc(df64(r.s[k].x, r.s[k].y), df64(r.s[k].z, r.s[k].w));
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = mkc(df64(r.u[k].x, r.u[k].y), df64(r.u[k].z, r.u[k].w));
}

__device__ __forceinline__ void decode(const Raw<P64>& r, cx<double> psi[12], cx<double> u[9]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) psi[k] = mkc(r.s[k].x, r.s[k].y);
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = mkc(r.u[k].x, r.u[k].y);
}
__device__ __forceinline__ void decode(const Raw<P32>& r, cx<float> psi[12], cx<float> u[9]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        psi[2 * k] = mkc(r.s[k].x, r.s[k].y);
        psi[2 * k + 1] = mkc(r.s[k].z, r.s[k].w);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        u[2 * k] = mkc(r.u[k].x, r.u[k].y);
        u[2 * k + 1] = mkc(r.u[k].z, r.u[k].w);
    }
    u[8] = mkc(r.u8.x, r.u8.y);
}
// The neighbour's per-site scale multiplies the 18 link reals instead of the
// 24 spinor reals: the hop term is linear in the spinor.
__device__ __forceinline__ void decode(const Raw<P16>& r, cx<float> psi[12], cx<float> u[9]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 a = h2f(r.s[k].x), b = h2f(r.s[k].y), c = h2f(r.s[k].z), d = h2f(r.s[k].w);
        psi[4 * k + 0] = mkc(a.x, a.y);
        psi[4 * k + 1] = mkc(b.x, b.y);
        psi[4 * k + 2] = mkc(c.x, c.y);
        psi[4 * k + 3] = mkc(d.x, d.y);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float2 a = h2f(r.u[k].x), b = h2f(r.u[k].y), c = h2f(r.u[k].z), d = h2f(r.u[k].w);
        u[4 * k + 0] = mkc(a.x * r.sc, a.y * r.sc);
        u[4 * k + 1] = mkc(b.x * r.sc, b.y * r.sc);
        u[4 * k + 2] = mkc(c.x * r.sc, c.y * r.sc);
        u[4 * k + 3] = mkc(d.x * r.sc, d.y * r.sc);
    }
    const float2 a = h2f(r.u8);
    u[8] = mkc(a.x * r.sc, a.y * r.sc);
}

// Two-row FP32 links (the 12 reals of rows 1 and 2 in 3 planes of float4;
// SU(3) gives row 3 as conj(row1 x row2)).
struct Raw32c { float4 s[6]; float4 u[3]; };

__device__ __forceinline__ void load_raw(Raw32c& r, const SpinorView& in, int64_t j, const LinkView& U, int64_t ju) {
    const float4* p = static_cast<const float4*>(in.data);
#pragma unroll
    for (int k = 0; k < 6; ++k) r.s[k] = __ldg(p + k * in.stride + j);
    const float4* q = static_cast<const float4*>(U.data);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.u[k] = __ldcs(q + k * U.stride + ju);
}
// row 3 of an SU(3) matrix from rows 1 and 2
__device__ __forceinline__ void third_row(cx<float> u[9]) {
    const cx<float> a = u[1] * u[5] - u[2] * u[4], b = u[2] * u[3] - u[0] * u[5], c = u[0] * u[4] - u[1] * u[3];
    u[6] = mkc(a.r, -a.i);
    u[7] = mkc(b.r, -b.i);
    u[8] = mkc(c.r, -c.i);
}
__device__ __forceinline__ void decode(const Raw32c& r, cx<float> psi[12], cx<float> u[9]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        psi[2 * k] = mkc(r.s[k].x, r.s[k].y);
        psi[2 * k + 1] = mkc(r.s[k].z, r.s[k].w);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u[2 * k] = mkc(r.u[k].x, r.u[k].y);
        u[2 * k + 1] = mkc(r.u[k].z, r.u[k].w);
    }
    third_row(u);
}
// a two-row FP32 link alone (the multi-RHS kernel loads each link once for
// several right-hand sides; later groups of the batch find it in L2)
__device__ __forceinline__ void load_link12(const LinkView& U, int64_t ju, cx<float> u[9]) {
    const float4* q = static_cast<const float4*>(U.data);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 v = __ldg(q + k * U.stride + ju);
        u[2 * k] = mkc(v.x, v.y);
        u[2 * k + 1] = mkc(v.z, v.w);
    }
    third_row(u);
}
template <int P, bool C> struct RawSel { using type = Raw<P>; };
template <> struct RawSel<P32, true> { using type = Raw32c; };

// One hop term: decode, project with (1 + S gamma_MU), colour-multiply
// (U or U^dag), reconstruct into acc.
template <int MU, int S, bool BACK, class real>
__device__ __forceinline__ void hop_term_dec(cx<real> acc[12], const cx<real> psi[12], const cx<real> u[9], bool flip) {
    cx<real> h[6], g[6];
    project<MU, S>(psi, h);
    if (flip) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = -h[k];
    }
    link_mul<BACK>(u, h, g);
    reconstruct<MU, S>(acc, g);
}

// Double-float g = U h (or U^dag h): each output component is a sum of six
// products, accumulated lazily -- exact products (TwoProd via FMA, cross terms
// of the low parts), one TwoSum chain on the high parts and plain FP32 sums of
// all error terms -- with a single renormalisation at the end.
__device__ __forceinline__ void df_prod(df64 a, df64 b, float& p, float& e) {
    p = a.hi * b.hi;
    e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
}
__device__ __forceinline__ void df_lazy_add(float& S, float& E, float p, float e) {
    const float s = S + p;
    const float bb = s - S;
    E += ((S - (s - bb)) + (p - bb)) + e;
    S = s;
}
// One row of U (u[0..2]) times both colour vectors of h: g0 = u . h[0..2],
// g1 = u . h[3..5].
__device__ __forceinline__ void df_row(const cx<df64> u[3], const cx<df64> h[6], cx<df64>& g0, cx<df64>& g1) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        float Sr = 0.f, Er = 0.f, Si = 0.f, Ei = 0.f, p, e;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const cx<df64> x = h[3 * s + b];
            // re += u.r x.r - u.i x.i
            df_prod(u[b].r, x.r, p, e);
            if (b == 0) { Sr = p; Er = e; } else df_lazy_add(Sr, Er, p, e);
            df_prod(u[b].i, x.i, p, e);
            df_lazy_add(Sr, Er, -p, -e);
            // im += u.r x.i + u.i x.r
            df_prod(u[b].r, x.i, p, e);
            if (b == 0) { Si = p; Ei = e; } else df_lazy_add(Si, Ei, p, e);
            df_prod(u[b].i, x.r, p, e);
            df_lazy_add(Si, Ei, p, e);
        }
        (s == 0 ? g0 : g1) = mkc(quick_two_sum(Sr, Er), quick_two_sum(Si, Ei));
    }
}
// g = U h, or U^dag h (rows of U^dag: conjugated columns of U)
template <bool BACK>
__device__ __forceinline__ void link_mul(const cx<df64> U[9], const cx<df64> h[6], cx<df64> g[6]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<df64> ur[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) ur[b] = BACK ? mkc(U[3 * b + a].r, -U[3 * b + a].i) : U[3 * a + b];
        df_row(ur, h, g[a], g[3 + a]);
    }
}

template <int MU, int S, bool BACK, class RAW, class real>
__device__ __forceinline__ void hop_term(cx<real> acc[12], const RAW& raw, bool flip) {
    cx<real> psi[12], u[9];
    decode(raw, psi, u);
    hop_term_dec<MU, S, BACK>(acc, psi, u, flip);
}

// Element k of an 8-entry register array for a runtime k (a switch keeps the
// array in registers; an indexed access would move it to local memory).
template <class T>
__device__ __forceinline__ T pick8(const T a[8], int k) {
    switch (k) {
        case 0: return a[0];
        case 1: return a[1];
        case 2: return a[2];
        case 3: return a[3];
        case 4: return a[4];
        case 5: return a[5];
        case 6: return a[6];
        default: return a[7];
    }
}

// Projection and reconstruction of direction d = 2 mu + back for a runtime d
// (small code per case; used by the double-float hop, whose colour product is
// too large to inline eight times).
template <int SF, class real>
__device__ __forceinline__ void project_rt(int d, const cx<real> psi[12], cx<real> h[6]) {
    switch (d) {
        case 0: project<0, SF>(psi, h); break;
        case 1: project<0, -SF>(psi, h); break;
        case 2: project<1, SF>(psi, h); break;
        case 3: project<1, -SF>(psi, h); break;
        case 4: project<2, SF>(psi, h); break;
        case 5: project<2, -SF>(psi, h); break;
        case 6: project<3, SF>(psi, h); break;
        default: project<3, -SF>(psi, h); break;
    }
}
template <int SF, class real>
__device__ __forceinline__ void reconstruct_rt(int d, cx<real> acc[12], const cx<real> g[6]) {
    switch (d) {
        case 0: reconstruct<0, SF>(acc, g); break;
        case 1: reconstruct<0, -SF>(acc, g); break;
        case 2: reconstruct<1, SF>(acc, g); break;
        case 3: reconstruct<1, -SF>(acc, g); break;
        case 4: reconstruct<2, SF>(acc, g); break;
        case 5: reconstruct<2, -SF>(acc, g); break;
        case 6: reconstruct<3, SF>(acc, g); break;
        default: reconstruct<3, -SF>(acc, g); break;
    }
}
// Direction d with decoded operands (see hop_term_d).
template <int SF, class real>
__device__ __forceinline__ void hop_term_dec_d(int d, cx<real> acc[12], const cx<real> psi[12], const cx<real> u[9],
                                               bool flip) {
    switch (d) {
        case 0: hop_term_dec<0, SF, false>(acc, psi, u, flip); break;
        case 1: hop_term_dec<0, -SF, true>(acc, psi, u, flip); break;
        case 2: hop_term_dec<1, SF, false>(acc, psi, u, flip); break;
        case 3: hop_term_dec<1, -SF, true>(acc, psi, u, flip); break;
        case 4: hop_term_dec<2, SF, false>(acc, psi, u, flip); break;
        case 5: hop_term_dec<2, -SF, true>(acc, psi, u, flip); break;
        case 6: hop_term_dec<3, SF, false>(acc, psi, u, flip); break;
        default: hop_term_dec<3, -SF, true>(acc, psi, u, flip); break;
    }
}

// Direction d = 2 mu + (0 forward, 1 backward); SF is the forward projector sign.
template <int SF, class RAW, class real>
__device__ __forceinline__ void hop_term_d(int d, cx<real> acc[12], const RAW& raw, bool flip) {
    switch (d) {
        case 0: hop_term<0, SF, false>(acc, raw, flip); break;
        case 1: hop_term<0, -SF, true>(acc, raw, flip); break;
        case 2: hop_term<1, SF, false>(acc, raw, flip); break;
        case 3: hop_term<1, -SF, true>(acc, raw, flip); break;
        case 4: hop_term<2, SF, false>(acc, raw, flip); break;
        case 5: hop_term<2, -SF, true>(acc, raw, flip); break;
        case 6: hop_term<3, SF, false>(acc, raw, flip); break;
        default: hop_term<3, -SF, true>(acc, raw, flip); break;
    }
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only) and their
// group bookkeeping: wait_group N returns once at most N of this thread's
// most recent groups are still pending.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Loads of the next hop are issued before the current one is computed for the
// bandwidth-bound precisions (more bytes in flight per thread); FP64 is bound
// by the FP64 pipe and keeps its registers for arithmetic.
#ifndef BPP_HOP_PREFETCH
#define BPP_HOP_PREFETCH 1
#endif
#ifndef BPP_HOP16_MAXT
#define BPP_HOP16_MAXT 512
#endif
template <int P> struct HopPrefetch { static constexpr bool value = BPP_HOP_PREFETCH != 0; };
template <> struct HopPrefetch<P64> { static constexpr bool value = false; };
template <> struct HopPrefetch<P64S> { static constexpr bool value = false; };

// Neighbour half-lattice indices jn, link indices ju and boundary flips of the
// 8 hops of output site i (coordinates x1..x4, row r = i / Lh).
__device__ __forceinline__ void hop_neighbours(const Geom& g, int i, int x1, int x1h, int r, int x2, int x3, int x4,
                                               int jn[8], int ju[8], bool flip[8]) {
    {
        const bool wf = x1 == g.L[0] - 1, wb = x1 == 0;
        jn[0] = ((wf ? 0 : x1 + 1) >> 1) + g.Lh * r;
        jn[1] = ((wb ? g.L[0] - 1 : x1 - 1) >> 1) + g.Lh * r;
        flip[0] = wf && g.bc[0] < 0;
        flip[1] = wb && g.bc[0] < 0;
    }
    {
        const bool wf = x2 == g.L[1] - 1, wb = x2 == 0;
        jn[2] = x1h + g.Lh * (wf ? r - (g.L[1] - 1) : r + 1);
        jn[3] = x1h + g.Lh * (wb ? r + (g.L[1] - 1) : r - 1);
        flip[2] = wf && g.bc[1] < 0;
        flip[3] = wb && g.bc[1] < 0;
    }
    {
        const int st = g.L[1];
        const bool wf = x3 == g.L[2] - 1, wb = x3 == 0;
        jn[4] = x1h + g.Lh * (wf ? r - (g.L[2] - 1) * st : r + st);
        jn[5] = x1h + g.Lh * (wb ? r + (g.L[2] - 1) * st : r - st);
        flip[4] = wf && g.bc[2] < 0;
        flip[5] = wb && g.bc[2] < 0;
    }
    {
        const int st = g.L[1] * g.L[2];
        const bool wf = x4 == g.L[3] - 1, wb = x4 == 0;
        jn[6] = x1h + g.Lh * (wf ? r - (g.L[3] - 1) * st : r + st);
        jn[7] = x1h + g.Lh * (wb ? r + (g.L[3] - 1) * st : r - st);
        flip[6] = wf && g.bc[3] < 0;
        flip[7] = wb && g.bc[3] < 0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) ju[k] = (k & 1) ? jn[k] : i;   // forward: U_mu(x); backward: U_mu(x - mu)
}

// Launch bounds (compile-time knobs, defaults measured fastest): at most 512
// threads per block for FP32 / FP16 (128 registers; 85-register bounds were
// measured 2-6% slower), 256 for FP64 and double-float, which need more
// registers per thread than a 512-thread block allows.
#ifndef BPP_HOP32_MAXT
#define BPP_HOP32_MAXT 512
#endif
#ifndef BPP_HOP_MINB
#define BPP_HOP_MINB 1
#endif
template <int P> struct HopMaxThreads { static constexpr int value = BPP_HOP32_MAXT; };
template <> struct HopMaxThreads<P64> { static constexpr int value = 256; };
template <> struct HopMaxThreads<P64S> { static constexpr int value = 256; };
template <> struct HopMaxThreads<P16> { static constexpr int value = BPP_HOP16_MAXT; };

// Minimum resident blocks per SM requested from the register allocator.
#ifndef BPP_HOPDF_MINB
#define BPP_HOPDF_MINB 2
#endif
template <int P> struct HopMinBlocks { static constexpr int value = BPP_HOP_MINB; };
template <> struct HopMinBlocks<P64> { static constexpr int value = 1; };
template <> struct HopMinBlocks<P64S> { static constexpr int value = BPP_HOPDF_MINB; };

// Face terms of a domain decomposition in x4 (see HopParams).  Forward hop at
// the top face: the upper domain sent h = (1 + SF gamma_4) psi (and, FP16, the
// site's spinor scale, applied to the link as in decode); backward hop at the
// bottom face: the lower domain sent g = U^dag (1 - SF gamma_4) psi.  The
// arithmetic and its order are those of hop_term, so the result is the same
// to the bit as without the decomposition.
template <int P, int SF>
__device__ __forceinline__ void hop_halo_fwd(cx<typename PT<P>::real> acc[12], const HopParams& hp, int s, int64_t f,
                                             const LinkView& U, int64_t i, bool flip) {
    using real = typename PT<P>::real;
    const cx<real>* hb = static_cast<const cx<real>*>(hp.halo_fwd) + (int64_t)s * 6 * hp.face;
    cx<real> h[6], u[9], g[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = hb[k * hp.face + f];
    Access<P>::load_link(U, i, u);
    if (P == P16) {
        const float sc = hp.halo_fwd_scale[(int64_t)s * hp.face + f];
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k] = mkc<real>(u[k].r * sc, u[k].i * sc);
    }
    if (flip) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = -h[k];
    }
    link_mul<false>(u, h, g);
    reconstruct<3, SF>(acc, g);
}
template <int P, int SB>
__device__ __forceinline__ void hop_halo_bwd(cx<typename PT<P>::real> acc[12], const HopParams& hp, int s, int64_t f,
                                             bool flip) {
    using real = typename PT<P>::real;
    const cx<real>* gb = static_cast<const cx<real>*>(hp.halo_bwd) + (int64_t)s * 6 * hp.face;
    cx<real> g[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) g[k] = flip ? -gb[k * hp.face + f] : gb[k * hp.face + f];
    reconstruct<3, SB>(acc, g);
}

// Stores v as Access<P>::store_spinor does and replaces it by the values a
// later load returns (FP16: the half rounding and the per-site scale, from
// the same packed words; the other formats store exactly).
template <int P>
__device__ __forceinline__ void store_read_back(const SpinorView& f, int64_t i, cx<typename PT<P>::real> v[12]) {
    Access<P>::store_spinor(f, i, v);
}
template <>
__device__ __forceinline__ void store_read_back<P16>(const SpinorView& f, int64_t i, cx<float> v[12]) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].r), fabsf(v[k].i)));
    const float inv = m > 0.f ? 1.f / m : 0.f;
    uint4* p = static_cast<uint4*>(f.data);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint32_t w[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = f2h(v[4 * k + c].r * inv, v[4 * k + c].i * inv);
        p[k * f.stride + i] = make_uint4(w[0], w[1], w[2], w[3]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float2 h = h2f(w[c]);
            v[4 * k + c] = mkc(h.x * m, h.y * m);
        }
    }
    f.scale[i] = m;
}

// Fused BiCGStab inner products of the stored output v (as read back, see
// store_read_back; see HopRed): one FP64 partial per warp of 32 consecutive
// sites of system s; lanes without a valid site add zero.
template <int P>
__device__ __forceinline__ void hop_reduce(const HopParams& hp, const SysDesc& d, int s, int it, bool valid,
                                           const cx<typename PT<P>::real> v[12], const cx<typename PT<P>::real> y[12]) {
    using real = typename PT<P>::real;
    real t[3] = {0, 0, 0};
    if (hp.red_op == HRED_ALPHA) {
        cx<real> rh[12];
        Access<P>::load_spinor(sys_view<P>(const_cast<char*>(hp.red_rhat), d), valid ? it : d.g.Vh - 1, rh);
        dot12(rh, v, t[0], t[1]);
    } else {
        dot12(v, y, t[0], t[1]);
        t[2] = norm12(v);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        real a = valid ? t[k] : (real)0;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        t[k] = a;
    }
    if ((threadIdx.x & 31) == 0) {
        double* o = hp.red_part + ((size_t)s * hp.red_wstride + (it >> 5)) * 4;
#pragma unroll
        for (int k = 0; k < 3; ++k) o[k] = (double)t[k];
    }
}

template <int P, bool DAG, int MODE, bool DD = false, bool C = false>
__global__ void __launch_bounds__(HopMaxThreads<P>::value, HopMinBlocks<P>::value) k_hop(HopParams hp) {
    using real = typename PT<P>::real;
    int s, tile;
    map_block(hp.map, s, tile);
    if (hp.done && hp.done[s * hp.done_stride]) return;
    const SysDesc& d = hp.sys[s];
    const Geom g = d.g;
    const int it = tile * blockDim.x + threadIdx.x;
    // a reducing launch keeps every lane of a warp that holds a valid site
    // (the warp sums need all 32 lanes); the extra lanes redo site Vh - 1 and
    // store nothing
    const bool valid = it < g.Vh;
    if (!valid && (hp.red_op == HRED_NONE || (it & ~31) >= g.Vh)) return;
    const int i = valid ? it : g.Vh - 1;
    const int p = hp.parity, q = 1 - p;

    const int x1h = i % g.Lh;
    const int r = i / g.Lh;
    const int x2 = r % g.L[1];
    const int r2 = r / g.L[1];
    const int x3 = r2 % g.L[2];
    const int x4 = r2 / g.L[2];
    const int x1 = 2 * x1h + ((p + x2 + x3 + x4) & 1);

    const SpinorView in = sys_view<P>(hp.in, d);
    int jn[8], ju[8];
    bool flip[8];
    hop_neighbours(g, i, x1, x1h, r, x2, x3, x4, jn, ju, flip);

    cx<real> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = mkc<real>(0, 0);

    constexpr int SF = DAG ? +1 : -1;   // forward projector 1 + SF gamma (backward: 1 - SF gamma)
    // decomposition in x4: face sites take their t-direction terms from the
    // face buffers (the local neighbour loads there read valid memory of this
    // domain and are not used)
    const bool top = DD && x4 == g.L[3] - 1, bot = DD && x4 == 0;
    const int64_t fidx = DD ? (int64_t)i - (int64_t)g.Lh * g.L[1] * g.L[2] * x4 : 0;
    if constexpr (P == P64S) {
        // one copy of the double-float colour product, the directions in a
        // loop (eight inlined copies overflow the instruction cache).  Each
        // direction's link (9 x 16 B per site) is copied to shared memory with
        // cp.async one direction ahead, so its loads are in flight while the
        // previous direction is computed without holding registers; the
        // product reads it row by row (U) or column by column (U^dag).
        extern __shared__ float4 lsm[];   // [2 buffers][9 entries][blockDim.x]
        const int B = blockDim.x;
        const float4* sp = static_cast<const float4*>(in.data);
        auto stage_link = [&](int k) {
            const LinkView U = d.U[(k & 1) ? q : p][k >> 1];
            const float4* up = static_cast<const float4*>(U.data) + pick8(ju, k);
            float4* dst = lsm + (k & 1) * 9 * B + threadIdx.x;
#pragma unroll
            for (int c = 0; c < 9; ++c) cp_async16(dst + c * B, up + c * U.stride);
            cp_async_commit();
        };
        stage_link(0);
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
            const bool back = k & 1;
            if (k < 7) stage_link(k + 1);
            cx<real> h[6], gk[6];
            {
                cx<real> psi[12];
                const int64_t jk = pick8(jn, k);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const float4 v = __ldg(sp + c * in.stride + jk);
                    psi[c] = mkc(df64(v.x, v.y), df64(v.z, v.w));
                }
                project_rt<SF>(k, psi, h);
            }
            if (pick8(flip, k)) {
#pragma unroll
                for (int c = 0; c < 6; ++c) h[c] = -h[c];
            }
            // this thread's copies of direction k have landed (those of k + 1
            // may still be in flight)
            if (k < 7) cp_async_wait<1>();
            else cp_async_wait<0>();
            const float4* ul = lsm + (k & 1) * 9 * B + threadIdx.x;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                cx<real> ur[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float4 v = ul[(back ? 3 * c + a : 3 * a + c) * B];
                    ur[c] = mkc(df64(v.x, v.y), back ? df64(-v.z, -v.w) : df64(v.z, v.w));
                }
                df_row(ur, h, gk[a], gk[3 + a]);
            }
            reconstruct_rt<SF>(k, acc, gk);
        }
    } else if (HopPrefetch<P>::value) {
        typename RawSel<P, C>::type cur, nxt;
        load_raw(cur, in, jn[0], d.U[p][0], ju[0]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k < 7) load_raw(nxt, in, jn[k + 1], d.U[((k + 1) & 1) ? q : p][(k + 1) >> 1], ju[k + 1]);
            if (DD && k == 6 && top) hop_halo_fwd<P, SF>(acc, hp, s, fidx, d.U[p][3], i, hp.flip_top != 0);
            else if (DD && k == 7 && bot) hop_halo_bwd<P, -SF>(acc, hp, s, fidx, hp.flip_bot != 0);
            else hop_term_d<SF>(k, acc, cur, flip[k]);
            if (k < 7) cur = nxt;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (DD && k == 6 && top) {
                hop_halo_fwd<P, SF>(acc, hp, s, fidx, d.U[p][3], i, hp.flip_top != 0);
            } else if (DD && k == 7 && bot) {
                hop_halo_bwd<P, -SF>(acc, hp, s, fidx, hp.flip_bot != 0);
            } else {
                typename RawSel<P, C>::type cur;
                load_raw(cur, in, jn[k], d.U[(k & 1) ? q : p][k >> 1], ju[k]);
                hop_term_d<SF>(k, acc, cur, flip[k]);
            }
        }
    }

    // v = a hop (+ y, or + A y): the xpay forms as one fused multiply-add
    const real a = (real)(hp.a_sign * d.kappa);
    cx<real> v[12], y[12];
    if (MODE == HOP_XPAY || MODE == HOP_CLOV_XPAY || MODE == HOP_INV_XPAY) {
        Access<P>::load_spinor(sys_view<P>(hp.y, d), i, y);
        if (MODE == HOP_CLOV_XPAY) {
            cx<real> ay[12];
            clover_apply_site<P>(d.A[p], i, y, ay);
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = cxfma(a, acc[k], ay[k]);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = cxfma(a, acc[k], y[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = a * acc[k];
    }
    if (MODE == HOP_INV || MODE == HOP_INV_XPAY) {
        cx<real> w[12];
        clover_apply_site<P>(d.Ainv[p], i, v, w);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = w[k];
    }
    if constexpr ((MODE == HOP_XPAY || MODE == HOP_CLOV_XPAY) && P != P64S) {
        if (hp.red_op != HRED_NONE) {
            if (valid) store_read_back<P>(sys_view<P>(hp.out, d), i, v);
            hop_reduce<P>(hp, d, s, it, valid, v, y);
            return;
        }
    }
    if (valid) Access<P>::store_spinor(sys_view<P>(hp.out, d), i, v);
}

// R right-hand sides of one gauge field per thread: each link is loaded once
// into registers and applied to the R half spinors (systems s0 .. s0+R-1 of a
// uniform batch whose systems share the links).  hp.map counts groups of R.
template <int P, bool DAG, int MODE, int R, bool C = false>
__global__ void __launch_bounds__(256) k_hop_multi(HopParams hp) {
    using real = typename PT<P>::real;
    int grp, tile;
    map_block(hp.map, grp, tile);
    const int s0 = grp * R;
    if (hp.done) {
        bool all = true;
#pragma unroll
        for (int r = 0; r < R; ++r) all = all && hp.done[(s0 + r) * hp.done_stride];
        if (all) return;
    }
    const SysDesc& d0 = hp.sys[s0];
    const Geom g = d0.g;
    const int it = tile * blockDim.x + threadIdx.x;
    const bool valid = it < g.Vh;   // as in k_hop
    if (!valid && (hp.red_op == HRED_NONE || (it & ~31) >= g.Vh)) return;
    const int i = valid ? it : g.Vh - 1;
    const int p = hp.parity, q = 1 - p;
    const int x1h = i % g.Lh;
    const int row = i / g.Lh;
    const int x2 = row % g.L[1];
    const int r2 = row / g.L[1];
    const int x3 = r2 % g.L[2];
    const int x4 = r2 / g.L[2];
    const int x1 = 2 * x1h + ((p + x2 + x3 + x4) & 1);
    int jn[8], ju[8];
    bool flip[8];
    hop_neighbours(g, i, x1, x1h, row, x2, x3, x4, jn, ju, flip);

    cx<real> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = mkc<real>(0, 0);
    constexpr int SF = DAG ? +1 : -1;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if constexpr (P == P16) {
            // the raw FP16 link once; per right-hand side the same decode as
            // the one-RHS kernel (the spinor's scale folded into the link), so
            // the two forms give identical bits
            Raw<P16> raw;
            const uint4* lq = static_cast<const uint4*>(d0.U[(k & 1) ? q : p][k >> 1].data);
            const int64_t ls = d0.U[(k & 1) ? q : p][k >> 1].stride;
#pragma unroll
            for (int c = 0; c < 2; ++c) raw.u[c] = __ldg(lq + c * ls + ju[k]);
            raw.u8 = __ldg(reinterpret_cast<const unsigned*>(lq + 2 * ls) + ju[k]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const SpinorView in = sys_view<P>(hp.in, hp.sys[s0 + r]);
                const uint4* sp = static_cast<const uint4*>(in.data);
#pragma unroll
                for (int c = 0; c < 3; ++c) raw.s[c] = __ldg(sp + c * in.stride + jn[k]);
                raw.sc = __ldg(in.scale + jn[k]);
                cx<real> psi[12], u[9];
                decode(raw, psi, u);
                hop_term_dec_d<SF>(k, acc[r], psi, u, flip[k]);
            }
        } else {
            cx<real> u[9];
            if constexpr (C && P == P32) load_link12(d0.U[(k & 1) ? q : p][k >> 1], ju[k], u);
            else Access<P>::load_link(d0.U[(k & 1) ? q : p][k >> 1], ju[k], u);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                cx<real> psi[12];
                Access<P>::load_spinor(sys_view<P>(hp.in, hp.sys[s0 + r]), jn[k], psi);
                hop_term_dec_d<SF>(k, acc[r], psi, u, flip[k]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const SysDesc& d = hp.sys[s0 + r];
        const real a = (real)(hp.a_sign * d.kappa);
        cx<real> v[12], y[12];
        if (MODE == HOP_XPAY || MODE == HOP_CLOV_XPAY || MODE == HOP_INV_XPAY) {
            Access<P>::load_spinor(sys_view<P>(hp.y, d), i, y);
            if (MODE == HOP_CLOV_XPAY) {
                cx<real> ay[12];
                clover_apply_site<P>(d.A[p], i, y, ay);
#pragma unroll
                for (int k = 0; k < 12; ++k) v[k] = cxfma(a, acc[r][k], ay[k]);
            } else {
#pragma unroll
                for (int k = 0; k < 12; ++k) v[k] = cxfma(a, acc[r][k], y[k]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = a * acc[r][k];
        }
        if (MODE == HOP_INV || MODE == HOP_INV_XPAY) {
            cx<real> w[12];
            clover_apply_site<P>(d.Ainv[p], i, v, w);
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = w[k];
        }
        bool reduced = false;
        if constexpr ((MODE == HOP_XPAY || MODE == HOP_CLOV_XPAY) && P != P64S) {
            if (hp.red_op != HRED_NONE) {
                if (valid) store_read_back<P>(sys_view<P>(hp.out, d), i, v);
                hop_reduce<P>(hp, d, s0 + r, it, valid, v, y);
                reduced = true;
            }
        }
        if (!reduced && valid) Access<P>::store_spinor(sys_view<P>(hp.out, d), i, v);
    }
}

double hop_bytes_per_site(int prec, int mode) {
    const double S = spinor_bytes(prec), L = link_bytes(prec);
    const double C = (prec == P64 || prec == P64S) ? 576 : prec == P32 ? 288 : 144;
    double b = 8 * L + 2 * S;
    if (mode == HOP_XPAY) b += S;
    if (mode == HOP_CLOV_XPAY) b += S + C;
    if (mode == HOP_INV) b += C;
    if (mode == HOP_INV_XPAY) b += S + C;
    return b;
}

template <int P, bool DAG, int MODE>
static void launch_t(const Batch& b, int parity, double a_sign, char* in, char* out, char* y, cudaStream_t st,
                     const int* done, int done_stride, const HopDD* dd = nullptr, const HopRed* red = nullptr) {
    HopParams hp;
    if (red && red->op != HRED_NONE) {
        if constexpr ((MODE == HOP_XPAY || MODE == HOP_CLOV_XPAY) && P != P64S) {
            BPP_REQUIRE(!dd && red->part && red->wstride >= (b.Vh_max + 31) / 32 &&
                            (red->op != HRED_ALPHA || red->rhat),
                        BPP_ERR_INVALID_ARG, "fused inner products: bad arguments");
            hp.red_op = red->op;
            hp.red_rhat = red->rhat;
            hp.red_part = red->part;
            hp.red_wstride = red->wstride;
        } else {
            throw Error(BPP_ERR_INVALID_ARG, "fused inner products need an FP64 / FP32 / FP16 XPAY or CLOV_XPAY hop");
        }
    }
    hp.halo_fwd = dd ? dd->fwd : nullptr;
    hp.halo_bwd = dd ? dd->bwd : nullptr;
    hp.halo_fwd_scale = dd ? dd->fwd_scale : nullptr;
    hp.face = dd ? dd->face : 0;
    hp.flip_top = dd ? dd->flip_top : 0;
    hp.flip_bot = dd ? dd->flip_bot : 0;
    hp.done = done;
    hp.done_stride = done_stride;
    hp.sys = b.dev();
    hp.parity = parity;
    hp.in = in;
    hp.out = out;
    hp.y = y;
    hp.a_sign = a_sign;
    const std::string key = "hop" + std::to_string(P) + (DAG ? "d" : "n") + std::to_string(MODE) + (dd ? "dd" : "") +
                            (hp.red_op ? "r" + std::to_string(hp.red_op) : "") +
                            (b.comp ? "c" : "") +
                            "_" + std::to_string(b.Vh_max) + "x" + std::to_string(b.nsys()) + (b.uniform ? "u" : "r");
    const bool may_tune = out != y && out != in;
    auto run = [&](int B) {
        int nb = 0;
        hp.map = block_map(b, B, nb);
        if constexpr (P == P64S) {
            // the double-float kernel stages two directions' links in shared
            // memory (the attribute is per device, so it is set at every launch)
            const int smem = 2 * 9 * B * (int)sizeof(float4);
            BPP_CUDA(cudaFuncSetAttribute(k_hop<P, DAG, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          2 * 9 * HopMaxThreads<P>::value * (int)sizeof(float4)));
            k_hop<P, DAG, MODE><<<nb, B, smem, st>>>(hp);
            return;
        } else {
            if (dd) {
                k_hop<P, DAG, MODE, true><<<nb, B, 0, st>>>(hp);
                return;
            }
        }
        if constexpr (P == P32) {
            if (b.comp) {
                k_hop<P, DAG, MODE, false, true><<<nb, B, 0, st>>>(hp);
                return;
            }
        }
        k_hop<P, DAG, MODE><<<nb, B, 0, st>>>(hp);
    };
    // right-hand sides of one gauge field can share each link load in registers
    bool shared = !dd && b.uniform && b.nsys() >= 2 && (P == P32 || P == P16);
    for (int s = 1; shared && s < b.nsys(); ++s) shared = b.sys[s].U[0][0].data == b.sys[0].U[0][0].data;
    auto run_multi = [&](int R, int B) {
        BlockMap m;
        m.nsys = b.nsys() / R;
        m.uniform = 1;
        m.tiles_per_sys = (b.Vh_max + B - 1) / B;
        for (int t = 0; t <= MAXSYS; ++t) m.tile_start[t] = 0;
        hp.map = m;
        const int nb = m.tiles_per_sys * m.nsys;
        if constexpr (P == P32) {
            if (b.comp) {
                if (R == 2) k_hop_multi<P, DAG, MODE, 2, true><<<nb, B, 0, st>>>(hp);
                else k_hop_multi<P, DAG, MODE, 4, true><<<nb, B, 0, st>>>(hp);
                return;
            }
        }
        if constexpr (P == P32 || P == P16) {
            if (R == 2) k_hop_multi<P, DAG, MODE, 2><<<nb, B, 0, st>>>(hp);
            else k_hop_multi<P, DAG, MODE, 4><<<nb, B, 0, st>>>(hp);
        }
    };
    int R = 1;   // right-hand sides per thread: 1 (k_hop), 2 or 4 (k_hop_multi)
    if (shared) {
        const int stored = tune_lookup(key + "R");
        if (stored > 0) {
            R = stored;
        } else if (may_tune && !capturing(st)) {
            // time the R = 1, 2, 4 variants (each with its own block size) and keep the fastest
            cudaEvent_t e0, e1;
            BPP_CUDA(cudaEventCreate(&e0));
            BPP_CUDA(cudaEventCreate(&e1));
            float best = 1e30f;
            R = 1;
            for (int cand : {1, 2, 4}) {
                if (b.nsys() % cand) continue;
                int Bc;
                if (cand == 1) Bc = tuned_block(key, st, run, true, HopMaxThreads<P>::value);
                else Bc = tuned_block(key + "R" + std::to_string(cand), st, [&](int B) { run_multi(cand, B); }, true, 256);
                auto go = [&]() { if (cand == 1) run(Bc); else run_multi(cand, Bc); };
                go();
                BPP_CUDA(cudaEventRecord(e0, st));
                for (int rep = 0; rep < 3; ++rep) go();
                BPP_CUDA(cudaEventRecord(e1, st));
                BPP_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                BPP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; R = cand; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            tune_store(key + "R", R);
        }
    }
    const int B = R == 1 ? tuned_block(key, st, run, may_tune, HopMaxThreads<P>::value)
                         : tuned_block(key + "R" + std::to_string(R), st, [&](int Bx) { run_multi(R, Bx); }, may_tune, 256);
    // algorithmic bytes: systems that share a gauge field (the right-hand sides
    // of one lattice) read its links once per launch
    double sites = 0, bytes = 0;
    const double lb = b.comp ? 48.0 : (double)link_bytes(P);
    const double bps = hop_bytes_per_site(P, MODE) - 8.0 * (link_bytes(P) - lb), lbytes = 8.0 * lb;
    std::vector<double> per_sys(b.nsys());
    for (int s = 0; s < b.nsys(); ++s) {
        bool first = true;
        for (int r = 0; r < s; ++r)
            if (b.sys[r].U[0][0].data == b.sys[s].U[0][0].data) first = false;
        per_sys[s] = b.sys[s].g.Vh * ((first ? bps : bps - lbytes) + (hp.red_op == HRED_ALPHA ? spinor_bytes(P) : 0));
        sites += b.sys[s].g.Vh;
        bytes += per_sys[s];
    }
    ProfScope prof(P, bytes, st);
    if (R == 1) run(B);
    else run_multi(R, B);
    count_launch();
    BPP_CHECK_LAUNCH();
    if (thread_capturing()) {
        for (int s = 0; s < b.nsys(); ++s) capture_hop_work(P, s, per_sys[s]);
        capture_hop_launch(P);
    } else {
        add_hop_work(P, 1, bytes);
    }
}

template <int P, bool DAG>
static void launch_mode(const Batch& b, int parity, int mode, double a_sign, char* in, char* out, char* y,
                        cudaStream_t st, const int* dn, int ds, const HopDD* dd, const HopRed* red = nullptr) {
    switch (mode) {
        case HOP_PLAIN: launch_t<P, DAG, HOP_PLAIN>(b, parity, a_sign, in, out, y, st, dn, ds, dd, red); break;
        case HOP_XPAY: launch_t<P, DAG, HOP_XPAY>(b, parity, a_sign, in, out, y, st, dn, ds, dd, red); break;
        case HOP_CLOV_XPAY: launch_t<P, DAG, HOP_CLOV_XPAY>(b, parity, a_sign, in, out, y, st, dn, ds, dd, red); break;
        case HOP_INV: launch_t<P, DAG, HOP_INV>(b, parity, a_sign, in, out, y, st, dn, ds, dd, red); break;
        case HOP_INV_XPAY: launch_t<P, DAG, HOP_INV_XPAY>(b, parity, a_sign, in, out, y, st, dn, ds, dd, red); break;
        default: throw Error(BPP_ERR_INVALID_ARG, "bad hopping mode");
    }
}

static void hop_any(const Batch& b, int parity, int dag, int mode, double a_sign, char* in, char* out, char* y,
                    cudaStream_t st, const int* dn, int ds, const HopDD* dd, const HopRed* red = nullptr) {
    BPP_REQUIRE(in != out, BPP_ERR_INVALID_ARG, "hopping term: output aliases input");
    if (b.prec == P64) {
        dag ? launch_mode<P64, true>(b, parity, mode, a_sign, in, out, y, st, dn, ds, dd, red)
            : launch_mode<P64, false>(b, parity, mode, a_sign, in, out, y, st, dn, ds, dd, red);
    } else if (b.prec == P32) {
        dag ? launch_mode<P32, true>(b, parity, mode, a_sign, in, out, y, st, dn, ds, dd, red)
            : launch_mode<P32, false>(b, parity, mode, a_sign, in, out, y, st, dn, ds, dd, red);
    } else if (b.prec == P64S) {
        BPP_REQUIRE(!dd, BPP_ERR_UNSUPPORTED, "the decomposed hopping term takes FP64, FP32 or FP16");
        dag ? launch_mode<P64S, true>(b, parity, mode, a_sign, in, out, y, st, dn, ds, dd, red)
            : launch_mode<P64S, false>(b, parity, mode, a_sign, in, out, y, st, dn, ds, dd, red);
    } else {
        dag ? launch_mode<P16, true>(b, parity, mode, a_sign, in, out, y, st, dn, ds, dd, red)
            : launch_mode<P16, false>(b, parity, mode, a_sign, in, out, y, st, dn, ds, dd, red);
    }
}

void hop(const Batch& b, int parity, int dag, int mode, double a_sign, char* in, char* out, char* y,
         cudaStream_t st, const int* dn, int ds, const HopRed* red) {
    hop_any(b, parity, dag, mode, a_sign, in, out, y, st, dn, ds, nullptr, red);
}

void hop_dd(const Batch& b, int parity, int dag, int mode, double a_sign, char* in, char* out, char* y,
            const HopDD& dd, cudaStream_t st, const int* dn, int ds) {
    hop_any(b, parity, dag, mode, a_sign, in, out, y, st, dn, ds, &dd);
}

// One thread per face site of both faces of the input field's parity q:
// the bottom face (x4 = 0) sends (1 + SF gamma_4) psi down, the top face
// (x4 = L4 - 1) sends U_4(x)^dag (1 - SF gamma_4) psi up (the arithmetic of
// hop_term for the corresponding hops of the neighbouring domains).
template <int P, bool DAG>
__global__ void k_dd_pack(const SysDesc* sys, BlockMap map, int q, const char* in, void* send_down,
                          float* send_down_scale, void* send_up, int64_t face) {
    using real = typename PT<P>::real;
    int s, tile;
    map_block(map, s, tile);
    const SysDesc& d = sys[s];
    const int64_t t = (int64_t)tile * blockDim.x + threadIdx.x;
    if (t >= 2 * face) return;
    const bool up = t >= face;
    const int64_t f = up ? t - face : t;
    const int64_t i = up ? face * (d.g.L[3] - 1) + f : f;
    constexpr int SF = DAG ? +1 : -1;
    Raw<P> raw;
    load_raw(raw, sys_view<P>(const_cast<char*>(in), d), i, d.U[q][3], i);
    cx<real> psi[12], u[9], h[6];
    decode(raw, psi, u);
    if (!up) {
        project<3, SF>(psi, h);
        cx<real>* o = static_cast<cx<real>*>(send_down) + (int64_t)s * 6 * face;
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k * face + f] = h[k];
        if (P == P16) send_down_scale[(int64_t)s * face + f] = __ldg(sys_view<P>(const_cast<char*>(in), d).scale + i);
    } else {
        cx<real> gg[6];
        project<3, -SF>(psi, h);
        link_mul<true>(u, h, gg);
        cx<real>* o = static_cast<cx<real>*>(send_up) + (int64_t)s * 6 * face;
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k * face + f] = gg[k];
    }
}

void dd_pack(const Batch& b, int in_parity, int dag, const char* in, void* send_down, float* send_down_scale,
             void* send_up, int64_t face, cudaStream_t st) {
    const int B = 128;
    BlockMap m;
    m.nsys = b.nsys();
    m.uniform = 1;
    m.tiles_per_sys = (int)((2 * face + B - 1) / B);
    for (int t = 0; t <= MAXSYS; ++t) m.tile_start[t] = 0;
    const int nb = m.tiles_per_sys * m.nsys;
    // per face site: the spinor read, the link read on the top face, 6
    // complex of face buffer written
    const double csize = b.prec == P64 ? 16.0 : 8.0;
    const double bytes = (double)b.nsys() * face * (2.0 * spinor_bytes(b.prec) + link_bytes(b.prec) + 2 * 6 * csize);
    ProfScope prof(PROF_OUTER, bytes, st);
    if (b.prec == P64) dag ? k_dd_pack<P64, true><<<nb, B, 0, st>>>(b.dev(), m, in_parity, in, send_down, send_down_scale, send_up, face)
                           : k_dd_pack<P64, false><<<nb, B, 0, st>>>(b.dev(), m, in_parity, in, send_down, send_down_scale, send_up, face);
    else if (b.prec == P32) dag ? k_dd_pack<P32, true><<<nb, B, 0, st>>>(b.dev(), m, in_parity, in, send_down, send_down_scale, send_up, face)
                                : k_dd_pack<P32, false><<<nb, B, 0, st>>>(b.dev(), m, in_parity, in, send_down, send_down_scale, send_up, face);
    else if (b.prec == P16) dag ? k_dd_pack<P16, true><<<nb, B, 0, st>>>(b.dev(), m, in_parity, in, send_down, send_down_scale, send_up, face)
                                : k_dd_pack<P16, false><<<nb, B, 0, st>>>(b.dev(), m, in_parity, in, send_down, send_down_scale, send_up, face);
    else throw Error(BPP_ERR_UNSUPPORTED, "the decomposed hopping term takes FP64, FP32 or FP16");
    count_launch();
    BPP_CHECK_LAUNCH();
}

}  // namespace bpp

namespace bpp {

// Hopping-kernel launch for the non-allocating entry point: fixed block size,
// no autotuner lookup, no timing events, the system table already resident
// on the device (dsys); all systems share one lattice (uniform map).
void hop_fixed(int prec, const SysDesc* dsys, int nsys, int Vh, int parity, int mode, double a_sign, char* in,
               char* out, char* y, cudaStream_t st) {
    constexpr int B = 128;
    HopParams hp;
    hp.sys = dsys;
    hp.parity = parity;
    hp.in = in;
    hp.out = out;
    hp.y = y;
    hp.a_sign = a_sign;
    hp.done = nullptr;
    hp.done_stride = 0;
    hp.halo_fwd = hp.halo_bwd = nullptr;
    hp.halo_fwd_scale = nullptr;
    hp.face = 0;
    hp.flip_top = hp.flip_bot = 0;
    hp.map.nsys = nsys;
    hp.map.uniform = 1;
    hp.map.tiles_per_sys = (Vh + B - 1) / B;
    for (int s = 0; s <= MAXSYS; ++s) hp.map.tile_start[s] = 0;
    const int nb = hp.map.tiles_per_sys * nsys;
    if (prec == P64) {
        if (mode == HOP_XPAY) k_hop<P64, false, HOP_XPAY><<<nb, B, 0, st>>>(hp);
        else k_hop<P64, false, HOP_PLAIN><<<nb, B, 0, st>>>(hp);
    } else if (prec == P32) {
        if (mode == HOP_XPAY) k_hop<P32, false, HOP_XPAY><<<nb, B, 0, st>>>(hp);
        else k_hop<P32, false, HOP_PLAIN><<<nb, B, 0, st>>>(hp);
    } else {
        if (mode == HOP_XPAY) k_hop<P16, false, HOP_XPAY><<<nb, B, 0, st>>>(hp);
        else k_hop<P16, false, HOP_PLAIN><<<nb, B, 0, st>>>(hp);
    }
    count_launch();
}

}  // namespace bpp
