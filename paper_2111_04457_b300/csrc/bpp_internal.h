// Internal definitions of the B300 Wilson / Wilson-clover library: precision
// traits, device field views, complex helpers, lattice geometry, errors.
//
// Field layout in HBM (one parity, "half field", Vh = V/2 sites):
//   spinors  structure of arrays, site index fastest, one plane per 16 bytes
//            of a site's 12 complex components (spin-major, colour fastest):
//              F64: 12 planes of double2        (192 B / site)
//              F32:  6 planes of float4         ( 96 B / site)
//              F16:  3 planes of 8 x half + 1 plane of float scale (52 B / site)
//            a plane holds `stride` entries (Vh rounded up to a multiple of 64).
//   links    per (parity of the site x, direction mu) the 3x3 matrix U_mu(x),
//            row-major entries, same plane scheme:
//              F64: 9 planes double2; F32: 4 planes float4 + 1 plane float2;
//              F16: 2 planes of 8 x half + 1 plane of half2.
//   clover   per parity, two 6x6 Hermitian chiral blocks per site (spins 0,1
//            and spins 2,3), each packed as 6 real diagonal entries followed by
//            the 15 complex strictly-lower entries (1,0),(2,0),(2,1),(3,0),...
//            (36 reals per block, 72 per site): F64 36 planes double2,
//            F32 18 planes float4, F16 9 planes of 8 x half.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/bpp.h"
#include "df64.h"

namespace bpp {

// ----------------------------------------------------------------------------- errors
struct Error : public std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define BPP_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw ::bpp::Error(e_ == cudaErrorMemoryAllocation ? BPP_ERR_OOM : BPP_ERR_CUDA,   \
                               std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

#define BPP_REQUIRE(cond, code, msg)                                                           \
    do {                                                                                       \
        if (!(cond)) throw ::bpp::Error((code), (msg));                                        \
    } while (0)

#define BPP_CHECK_LAUNCH() BPP_CUDA(cudaGetLastError())

// ----------------------------------------------------------------------------- precision
// P64S is internal only: FP64 values stored as (hi, lo) FP32 pairs and used
// with double-float arithmetic (df64.h); same bytes as FP64.
enum Prec { P64 = BPP_F64, P32 = BPP_F32, P16 = BPP_F16, P64S = 3 };
constexpr int NPREC = 4;

// Kernel classes of the launch timing (bpp_prof_read): the hopping kernels
// per precision (0..3 = Prec), then the other kernel families.
enum ProfClass { PROF_BLAS = 4, PROF_OUTER = 5, PROF_LAYOUT = 6, PROF_CTL = 7, PROF_CLOVER = 8, PROF_FORCE = 9 };
constexpr int NPROF = 10;

template <int P> struct PT;
template <> struct PT<P64> {
    using real = double;
    static constexpr int spinor_bytes = 192;
    static constexpr int link_bytes = 144;
    static constexpr int clover_bytes = 576;   // 2 blocks x 36 reals x 8 B
};
template <> struct PT<P32> {
    using real = float;
    static constexpr int spinor_bytes = 96;
    static constexpr int link_bytes = 72;
    static constexpr int clover_bytes = 288;
};
template <> struct PT<P16> {
    using real = float;
    static constexpr int spinor_bytes = 52;    // 48 B of halves + 4 B scale
    static constexpr int link_bytes = 36;
    static constexpr int clover_bytes = 144;
};
template <> struct PT<P64S> {
    using real = df64;
    static constexpr int spinor_bytes = 192;
    static constexpr int link_bytes = 144;
    static constexpr int clover_bytes = 576;
};

inline int spinor_bytes(int prec) {
    return (prec == P64 || prec == P64S) ? 192 : prec == P32 ? 96 : 52;
}
inline int link_bytes(int prec) {
    return (prec == P64 || prec == P64S) ? 144 : prec == P32 ? 72 : 36;
}

// ----------------------------------------------------------------------------- complex
template <class T> struct cx {
    T r, i;
};
template <class T> __host__ __device__ __forceinline__ cx<T> mkc(T r, T i) { cx<T> c; c.r = r; c.i = i; return c; }
template <class T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mkc(a.r + b.r, a.i + b.i); }
template <class T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mkc(a.r - b.r, a.i - b.i); }
template <class T> __device__ __forceinline__ cx<T> operator-(cx<T> a) { return mkc(-a.r, -a.i); }
template <class T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mkc(s * a.r, s * a.i); }
template <class T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mkc(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
// conj(a) * b
template <class T> __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
    return mkc(a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r);
}
// i * a
template <class T> __device__ __forceinline__ cx<T> ix(cx<T> a) { return mkc(-a.i, a.r); }
// a += b * c
template <class T> __device__ __forceinline__ void cfma(cx<T>& a, cx<T> b, cx<T> c) {
    a.r = fma(b.r, c.r, a.r); a.r = fma(-b.i, c.i, a.r);
    a.i = fma(b.r, c.i, a.i); a.i = fma(b.i, c.r, a.i);
}
// a * x + y for a real a (one rounding per component)
template <class T> __device__ __forceinline__ cx<T> cxfma(T a, cx<T> x, cx<T> y) {
    return mkc(fma(a, x.r, y.r), fma(a, x.i, y.i));
}
// a += conj(b) * c
template <class T> __device__ __forceinline__ void cfmac(cx<T>& a, cx<T> b, cx<T> c) {
    a.r = fma(b.r, c.r, a.r); a.r = fma(b.i, c.i, a.r);
    a.i = fma(b.r, c.i, a.i); a.i = fma(-b.i, c.r, a.i);
}

// ----------------------------------------------------------------------------- field views
// A half-lattice spinor field in one of the three storage formats.
struct SpinorView {
    void* data;      // plane 0 base
    float* scale;    // F16 only: one float per site
    int64_t stride;  // entries per plane
};
// One link field (one parity, one direction).
struct LinkView {
    const void* data;
    int64_t stride;
};
// One parity of a clover field (A or A^-1).
struct CloverView {
    const void* data;
    int64_t stride;
};

inline int64_t pad_stride(int64_t n) { return (n + 63) / 64 * 64; }

inline size_t spinor_alloc_bytes(int prec, int64_t stride) {
    if (prec == P64 || prec == P64S) return (size_t)stride * 192;
    if (prec == P32) return (size_t)stride * 96;
    return (size_t)stride * 52;
}
inline size_t link_alloc_bytes(int prec, int64_t stride) { return (size_t)stride * link_bytes(prec); }

__host__ __device__ inline SpinorView make_spinor_view(int prec, void* base, int64_t stride) {
    SpinorView v;
    v.data = base;
    v.stride = stride;
    v.scale = prec == P16 ? reinterpret_cast<float*>(static_cast<char*>(base) + (size_t)stride * 48) : nullptr;
    return v;
}

// ----------------------------------------------------------------------------- loads/stores
template <int P> struct Access;

template <> struct Access<P64> {
    using real = double;
    static __device__ __forceinline__ void load_spinor(const SpinorView& f, int64_t i, cx<double> s[12]) {
        const double2* p = static_cast<const double2*>(f.data);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = __ldg(p + k * f.stride + i);
            s[k] = mkc(v.x, v.y);
        }
    }
    static __device__ __forceinline__ void store_spinor(const SpinorView& f, int64_t i, const cx<double> s[12]) {
        double2* p = static_cast<double2*>(f.data);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k * f.stride + i] = make_double2(s[k].r, s[k].i);
    }
    static __device__ __forceinline__ void load_link(const LinkView& u, int64_t i, cx<double> m[9]) {
        const double2* p = static_cast<const double2*>(u.data);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 v = __ldcs(p + k * u.stride + i);
            m[k] = mkc(v.x, v.y);
        }
    }
};

template <> struct Access<P32> {
    using real = float;
    static __device__ __forceinline__ void load_spinor(const SpinorView& f, int64_t i, cx<float> s[12]) {
        const float4* p = static_cast<const float4*>(f.data);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 v = __ldg(p + k * f.stride + i);
            s[2 * k] = mkc(v.x, v.y);
            s[2 * k + 1] = mkc(v.z, v.w);
        }
    }
    static __device__ __forceinline__ void store_spinor(const SpinorView& f, int64_t i, const cx<float> s[12]) {
        float4* p = static_cast<float4*>(f.data);
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k * f.stride + i] = make_float4(s[2 * k].r, s[2 * k].i, s[2 * k + 1].r, s[2 * k + 1].i);
    }
    static __device__ __forceinline__ void load_link(const LinkView& u, int64_t i, cx<float> m[9]) {
        const float4* p = static_cast<const float4*>(u.data);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 v = __ldcs(p + k * u.stride + i);
            m[2 * k] = mkc(v.x, v.y);
            m[2 * k + 1] = mkc(v.z, v.w);
        }
        const float2* q = reinterpret_cast<const float2*>(p + 4 * u.stride);
        float2 v = __ldcs(q + i);
        m[8] = mkc(v.x, v.y);
    }
};

// Split FP64: each complex component is one float4 (re.hi, re.lo, im.hi, im.lo).
template <> struct Access<P64S> {
    using real = df64;
    static __device__ __forceinline__ void load_spinor(const SpinorView& f, int64_t i, cx<df64> s[12]) {
        const float4* p = static_cast<const float4*>(f.data);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float4 v = __ldg(p + k * f.stride + i);
            s[k] = mkc(df64(v.x, v.y), df64(v.z, v.w));
        }
    }
    static __device__ __forceinline__ void store_spinor(const SpinorView& f, int64_t i, const cx<df64> s[12]) {
        float4* p = static_cast<float4*>(f.data);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const df64 r = normalized(s[k].r), m = normalized(s[k].i);
            p[k * f.stride + i] = make_float4(r.hi, r.lo, m.hi, m.lo);
        }
    }
    static __device__ __forceinline__ void load_link(const LinkView& u, int64_t i, cx<df64> m[9]) {
        const float4* p = static_cast<const float4*>(u.data);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float4 v = __ldcs(p + k * u.stride + i);
            m[k] = mkc(df64(v.x, v.y), df64(v.z, v.w));
        }
    }
};

__device__ __forceinline__ float2 h2f(uint32_t w) {
    __half2 h = *reinterpret_cast<__half2*>(&w);
    return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <> struct Access<P16> {
    using real = float;
    static __device__ __forceinline__ void load_spinor(const SpinorView& f, int64_t i, cx<float> s[12]) {
        const uint4* p = static_cast<const uint4*>(f.data);
        const float sc = __ldg(f.scale + i);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = __ldg(p + k * f.stride + i);
            float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
            s[4 * k + 0] = mkc(a.x * sc, a.y * sc);
            s[4 * k + 1] = mkc(b.x * sc, b.y * sc);
            s[4 * k + 2] = mkc(c.x * sc, c.y * sc);
            s[4 * k + 3] = mkc(d.x * sc, d.y * sc);
        }
    }
    static __device__ __forceinline__ void store_spinor(const SpinorView& f, int64_t i, const cx<float> s[12]) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(s[k].r), fabsf(s[k].i)));
        const float inv = m > 0.f ? 1.f / m : 0.f;
        uint4* p = static_cast<uint4*>(f.data);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v;
            v.x = f2h(s[4 * k + 0].r * inv, s[4 * k + 0].i * inv);
            v.y = f2h(s[4 * k + 1].r * inv, s[4 * k + 1].i * inv);
            v.z = f2h(s[4 * k + 2].r * inv, s[4 * k + 2].i * inv);
            v.w = f2h(s[4 * k + 3].r * inv, s[4 * k + 3].i * inv);
            p[k * f.stride + i] = v;
        }
        f.scale[i] = m;
    }
    static __device__ __forceinline__ void load_link(const LinkView& u, int64_t i, cx<float> m[9]) {
        const uint4* p = static_cast<const uint4*>(u.data);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint4 v = __ldcs(p + k * u.stride + i);
            float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
            m[4 * k + 0] = mkc(a.x, a.y);
            m[4 * k + 1] = mkc(b.x, b.y);
            m[4 * k + 2] = mkc(c.x, c.y);
            m[4 * k + 3] = mkc(d.x, d.y);
        }
        const unsigned int* q = reinterpret_cast<const unsigned int*>(p + 2 * u.stride);
        float2 a = h2f(__ldcs(q + i));
        m[8] = mkc(a.x, a.y);
    }
};

// ----------------------------------------------------------------------------- geometry
// Lattice extents and boundary signs as the kernels see them.  L[0] is even;
// a half-lattice index i (sites of one parity in lexicographic order) is the
// lexicographic index divided by two.
struct Geom {
    int L[4];
    int bc[4];
    int Lh;          // L[0] / 2
    int Vh;          // V / 2
};

// Coordinates of half-lattice site i of parity p.
__host__ __device__ __forceinline__ void eo_coords(const Geom& g, int i, int p, int x[4]) {
    const int x1h = i % g.Lh;
    int r = i / g.Lh;
    x[1] = r % g.L[1];
    r /= g.L[1];
    x[2] = r % g.L[2];
    x[3] = r / g.L[2];
    x[0] = 2 * x1h + ((p + x[1] + x[2] + x[3]) & 1);
}

// ----------------------------------------------------------------------------- systems
// A "system" is one linear system of a batch: one lattice (gauge field, kappa)
// and one right-hand side.  Every kernel launch covers all systems of a batch.
// Vectors of a batch live in one allocation per vector name; system s owns the
// bytes [vec_off, vec_off + spinor_alloc_bytes(prec, stride)) of each.
constexpr int MAXSYS = 64;

struct SysDesc {
    Geom g;
    LinkView U[2][4];      // [parity of x][mu] -> U_mu(x), at the launch precision
    CloverView A[2];       // 1 + F per parity (data == nullptr: Wilson)
    CloverView Ainv[2];    // (1 + F)^-1 per parity
    double kappa;
    int64_t vec_off;       // byte offset of this system in every batch vector
    int64_t stride;        // plane stride of this system's vectors
};

// How the blocks of one launch map to (system, tile).  Uniform batches (all
// systems the same size) interleave systems fastest, so the CTAs that work on
// one site tile for different right-hand sides run together and share the
// link loads through L2; ragged batches go system by system.
struct BlockMap {
    int nsys;
    int uniform;
    int tiles_per_sys;               // uniform: tiles of each system
    int tile_start[MAXSYS + 1];      // ragged: first block of each system
};

__device__ __forceinline__ void map_block(const BlockMap& m, int& s, int& tile) {
    const int b = blockIdx.x;
    if (m.uniform) {
        s = b % m.nsys;
        tile = b / m.nsys;
    } else {
        int lo = 0, hi = m.nsys;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (m.tile_start[mid] <= b) lo = mid; else hi = mid;
        }
        s = lo;
        tile = b - m.tile_start[lo];
    }
}

template <int P>
__host__ __device__ __forceinline__ SpinorView sys_view(char* base, const SysDesc& d) {
    SpinorView v;
    v.data = base + d.vec_off;
    v.stride = d.stride;
    v.scale = P == P16 ? reinterpret_cast<float*>(base + d.vec_off + d.stride * 48) : nullptr;
    return v;
}

// ----------------------------------------------------------------------------- runtime
// Counts every kernel launch of the library (bpp_launch_count); launches made
// while the calling thread captures a CUDA graph are not counted (the graph's
// executions are counted instead).
void count_launch(int64_t n = 1);
void set_capturing(bool on);
bool thread_capturing();
// Algorithmic work of the hopping kernels (bpp_work_read): added per launch,
// or, for launches recorded into a graph, accumulated per system into the
// calling thread's capture record so the graph's executions can be credited.
void add_hop_work(int prec, int64_t launches, double bytes);
void capture_hop_work(int prec, int sys, double bytes);
void capture_work_reset(int nsys);
void capture_hop_launch(int prec);
int64_t capture_hop_launches(int prec);
const std::vector<double>& capture_work_bytes(int prec);
int64_t capture_launches();
// True while `s` is being captured into a CUDA graph.
bool capturing(cudaStream_t s);

// Chooses the block size for a launch identified by `key` (kernel + shape).
// On the first call outside graph capture it times each candidate with CUDA
// events through `run(block)` and keeps the fastest; `run` must be a pure
// function of its inputs (it is launched several times).
int tune_lookup(const std::string& key);
void tune_store(const std::string& key, int block);
// Launch timing (bpp_prof_enable / bpp_prof_read): while enabled, a
// ProfScope brackets the launches made in its lifetime with CUDA events on
// its stream and credits them to kernel class `prec` (a Prec for the hopping
// kernels, else a ProfClass) with `bytes` of algorithmic traffic.
struct ProfScope {
    int prec;
    double bytes;
    cudaStream_t s;
    cudaEvent_t e0, e1;
    bool on;
    ProfScope(int prec, double bytes, cudaStream_t s);
    ~ProfScope();
};

// Stream-ordered device scratch from the CUDA memory pool (cached by the pool).
// With persistent = true the block comes from cudaMalloc (for long-lived
// solver plans that outlive the caller's stream).
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    bool persistent = false;
    DevBuf() = default;
    DevBuf(size_t bytes, cudaStream_t st) { alloc(bytes, st); }
    void alloc(size_t bytes, cudaStream_t st);
    void alloc_persistent(size_t bytes);
    void release();
    ~DevBuf() { release(); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    template <class T> T* as() const { return static_cast<T*>(p); }
};

template <class Run>
int tuned_block(const std::string& key, cudaStream_t s, Run run, bool may_tune = true, int max_block = 512,
                int min_block = 32) {
    int b = tune_lookup(key);
    if (b > 0) return b;
    if (!may_tune || capturing(s)) return max_block < 256 ? max_block : 256;
    static const int cand_all[] = {32, 64, 128, 256, 512};
    std::vector<int> cand;
    for (int c : cand_all)
        if (c <= max_block && c >= min_block) cand.push_back(c);
    cudaEvent_t e0, e1;
    BPP_CUDA(cudaEventCreate(&e0));
    BPP_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_b = 256;
    for (int c : cand) {
        run(c);                         // warm-up
        BPP_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < 3; ++r) run(c);
        BPP_CUDA(cudaEventRecord(e1, s));
        BPP_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        BPP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; best_b = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_store(key, best_b);
    return best_b;
}

// Measured FMA-pipe throughput (TFLOP/s, an FMA counted as 2 flop) of
// prec = P64 or P32 (peak.cu).
double fma_peak(int prec, cudaStream_t st);

}  // namespace bpp
