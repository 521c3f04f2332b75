// Batched BLAS-1 with fused reductions for the solvers; see blas.h.
#include <string>

#include "blas.h"
#include "clover_dev.h"
#include "kernels.h"
#include "reduce.h"

namespace bpp {

constexpr int BLAS_B = 256;
#ifndef BPP_BLAS_SPT
#define BPP_BLAS_SPT 8
#endif
constexpr int BLAS_SPT = BPP_BLAS_SPT;   // sites per thread

// Threads per block of the vector kernels: 256, or fewer on small lattices so
// that the grid still spans about two blocks per SM (on few SMs the FP64 work
// of a small lattice is bound by the FP64 pipe, 1/64 of the FP32 rate).
static int vec_block(const Batch& b) {
    const int64_t S = b.sites();
    int B = BLAS_B;
    while (B > 32 && S < (int64_t)B * 2 * 148) B >>= 1;
    return B;
}

void RedBuf::ensure(int nblocks, int nsys, cudaStream_t st) {
    if (nblocks > cap_blocks) {
        BPP_REQUIRE(!capturing(st), BPP_ERR_CUDA, "reduction buffer must be sized before graph capture");
        if (persistent) partials.alloc_persistent((size_t)nblocks * 4 * sizeof(double));
        else partials.alloc((size_t)nblocks * 4 * sizeof(double), st);
        cap_blocks = nblocks;
    }
    if (tickets.n < (size_t)MAXSYS * sizeof(unsigned)) {
        if (persistent) tickets.alloc_persistent((size_t)MAXSYS * sizeof(unsigned));
        else tickets.alloc((size_t)MAXSYS * sizeof(unsigned), st);
        BPP_CUDA(cudaMemsetAsync(tickets.p, 0, (size_t)MAXSYS * sizeof(unsigned), st));
    }
}

struct BlasParams {
    const SysDesc* sys;
    BlockMap map;
    BlasVecs v;
    KScal* sc;
    double* partials;
    unsigned* tickets;
    double* red_out = nullptr;   // set: write the system's sums here [s][4], do not finalize
};

__device__ __forceinline__ void check_done(KScal& k) {
    if (!isfinite(k.rr)) { k.done = 1; k.status = 3; return; }
    if (k.rr <= k.tol2 * k.bb) { k.done = 1; return; }
    if (k.iter >= k.max_iter) { k.done = 1; k.status = 2; }
}

// The update and reduction terms of one site i of system d.
template <int P, int OP>
__device__ __forceinline__ void blas_site(const BlasParams& bp, const SysDesc& d, int i, double2 al, double2 om,
                                          double2 be, typename PT<P>::real red[4]) {
    using real = typename PT<P>::real;
    using A = Access<P>;
    cx<real> a[12], b[12], c[12];
    if (OP == B_INIT_BICG) {
        A::load_spinor(sys_view<P>(bp.v.b, d), i, a);
        A::store_spinor(sys_view<P>(bp.v.r, d), i, a);
        A::store_spinor(sys_view<P>(bp.v.rhat, d), i, a);
        A::store_spinor(sys_view<P>(bp.v.p, d), i, a);
#pragma unroll
        for (int k = 0; k < 12; ++k) b[k] = mkc<real>(0, 0);
        A::store_spinor(sys_view<P>(bp.v.x, d), i, b);
        red[0] += norm12(a);
    } else if (OP == B_ALPHA) {
        real re, im;
        A::load_spinor(sys_view<P>(bp.v.rhat, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.v, d), i, b);
        dot12(a, b, re, im);
        red[0] += re; red[1] += im;
    } else if (OP == B_S) {
        const cx<real> alr = mkc<real>((real)al.x, (real)al.y);
        A::load_spinor(sys_view<P>(bp.v.r, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.v, d), i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) { c[k] = a[k]; cfma(c[k], -alr, b[k]); }
        A::store_spinor(sys_view<P>(bp.v.s, d), i, c);
    } else if (OP == B_OMEGA) {
        real re, im;
        A::load_spinor(sys_view<P>(bp.v.t, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.s, d), i, b);
        dot12(a, b, re, im);
        red[0] += re; red[1] += im; red[2] += norm12(a);
    } else if (OP == B_XR) {
        const cx<real> alr = mkc<real>((real)al.x, (real)al.y), omr = mkc<real>((real)om.x, (real)om.y);
        // x += alpha p + omega s
        A::load_spinor(sys_view<P>(bp.v.x, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.p, d), i, b);
        A::load_spinor(sys_view<P>(bp.v.s, d), i, c);
#pragma unroll
        for (int k = 0; k < 12; ++k) { cfma(a[k], alr, b[k]); cfma(a[k], omr, c[k]); }
        A::store_spinor(sys_view<P>(bp.v.x, d), i, a);
        // r = s - omega t
        A::load_spinor(sys_view<P>(bp.v.t, d), i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) cfma(c[k], -omr, b[k]);
        A::store_spinor(sys_view<P>(bp.v.r, d), i, c);
        A::load_spinor(sys_view<P>(bp.v.rhat, d), i, a);
        real re, im;
        dot12(a, c, re, im);
        red[0] += norm12(c); red[1] += re; red[2] += im;
    } else if (OP == B_P) {
        const cx<real> ber = mkc<real>((real)be.x, (real)be.y), omr = mkc<real>((real)om.x, (real)om.y);
        A::load_spinor(sys_view<P>(bp.v.r, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.p, d), i, b);
        A::load_spinor(sys_view<P>(bp.v.v, d), i, c);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            cfma(b[k], -omr, c[k]);     // p - omega v
            cfma(a[k], ber, b[k]);      // r + beta (...)
        }
        A::store_spinor(sys_view<P>(bp.v.p, d), i, a);
    } else if (OP == B_CG_INIT) {
        A::load_spinor(sys_view<P>(bp.v.b, d), i, a);
        A::store_spinor(sys_view<P>(bp.v.r, d), i, a);
#pragma unroll
        for (int k = 0; k < 12; ++k) b[k] = mkc<real>(0, 0);
        A::store_spinor(sys_view<P>(bp.v.x, d), i, b);
        red[0] += norm12(a);
    } else if (OP == B_CG_PZ) {
        A::load_spinor(sys_view<P>(bp.v.z, d), i, a);
        A::store_spinor(sys_view<P>(bp.v.p, d), i, a);
        red[0] += norm12(a);
    } else if (OP == B_CG_ALPHA) {
        A::load_spinor(sys_view<P>(bp.v.w, d), i, a);
        red[0] += norm12(a);
    } else if (OP == B_CG_XR) {
        const real alr = (real)al.x;
        A::load_spinor(sys_view<P>(bp.v.x, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.p, d), i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) a[k] = a[k] + alr * b[k];
        A::store_spinor(sys_view<P>(bp.v.x, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.r, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.w, d), i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) a[k] = a[k] - alr * b[k];
        A::store_spinor(sys_view<P>(bp.v.r, d), i, a);
        red[0] += norm12(a);
    } else if (OP == B_CG_BETA) {
        A::load_spinor(sys_view<P>(bp.v.z, d), i, a);
        red[0] += norm12(a);
    } else if (OP == B_NORM2) {
        A::load_spinor(sys_view<P>(bp.v.x, d), i, a);
        red[0] += norm12(a);
    } else if (OP == B_NORM2X2) {
        A::load_spinor(sys_view<P>(bp.v.x, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.r, d), i, b);
        red[0] += norm12(a) + norm12(b);
    } else if (OP == B_MR) {
        const cx<real> omr = mkc<real>((real)om.x, (real)om.y);
        A::load_spinor(sys_view<P>(bp.v.x, d), i, a);
        A::load_spinor(sys_view<P>(bp.v.s, d), i, b);
        A::load_spinor(sys_view<P>(bp.v.t, d), i, c);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            cfma(a[k], omr, b[k]);
            cfma(b[k], -omr, c[k]);
        }
        A::store_spinor(sys_view<P>(bp.v.x, d), i, a);
        A::store_spinor(sys_view<P>(bp.v.s, d), i, b);
    }
}

// Solver scalars from the reduced sums tot[] of one system (the end of a
// fused vector kernel, or of a decomposed reduction).
template <int OP>
__device__ void blas_finalize(KScal& k, const double tot[4]) {
    if (OP == B_INIT_BICG) {
        k.bb = tot[0];
        k.rr = tot[0];
        k.rho = c2(tot[0], 0.0);
        k.alpha = c2(1.0, 0.0);
        k.omega = c2(1.0, 0.0);
        k.beta = c2(0.0, 0.0);
        k.iter = 0;
        k.status = 0;
        k.done = 0;
        check_done(k);
        if (k.bb == 0.0) { k.done = 1; k.status = 0; }
    } else if (OP == B_ALPHA) {
        finalize_alpha(k, tot[0], tot[1]);
    } else if (OP == B_OMEGA) {
        finalize_omega(k, tot[0], tot[1], tot[2]);
    } else if (OP == B_XR) {
        k.rr = tot[0];
        const double2 rho_new = c2(tot[1], tot[2]);
        k.iter += 1;
        if (cabs2(k.omega) == 0.0) { k.status = 1; k.done = 1; }
        else k.beta = cmul2(cdiv2(rho_new, k.rho), cdiv2(k.alpha, k.omega));
        k.rho = rho_new;
        if (cabs2(rho_new) < 1e-60 * k.rr * k.bb && !(k.rr <= k.tol2 * k.bb)) { k.status = 1; k.done = 1; }
        check_done(k);
    } else if (OP == B_CG_INIT) {
        k.bb = tot[0];
        k.rr = tot[0];
        k.iter = 0;
        k.status = 0;
        k.done = 0;
        check_done(k);
        if (k.bb == 0.0) { k.done = 1; k.status = 0; }
    } else if (OP == B_CG_PZ) {
        k.zz = tot[0];
    } else if (OP == B_CG_ALPHA) {
        if (tot[0] > 0.0) k.alpha = c2(k.zz / tot[0], 0.0);
        else { k.alpha = c2(0.0, 0.0); k.status = 1; k.done = 1; }
    } else if (OP == B_CG_XR) {
        k.rr = tot[0];
        k.iter += 1;
        check_done(k);
    } else if (OP == B_CG_BETA) {
        k.beta = c2(k.zz > 0.0 ? tot[0] / k.zz : 0.0, 0.0);
        k.zz = tot[0];
    } else if (OP == B_NORM2 || OP == B_NORM2X2) {
        k.bb = tot[0];
    }
}

// Finalize of a reduction whose sums were combined elsewhere (one thread per
// system).
template <int OP>
__global__ void k_blas_fin(KScal* sc, const double* tot, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    if (!(OP == B_INIT_BICG || OP == B_CG_INIT || OP == B_NORM2 || OP == B_NORM2X2) && sc[s].done) return;
    blas_finalize<OP>(sc[s], tot + 4 * s);
}

// Each block covers BLAS_SPT * BLAS_B sites of one system, so the last block
// of a reduction sums few per-block partials.
template <int P, int OP, int SPT>
__global__ void __launch_bounds__(BLAS_B) k_blas(BlasParams bp) {
    int s, tile;
    map_block(bp.map, s, tile);
    const SysDesc& d = bp.sys[s];
    KScal* K = bp.sc + s;
    const bool active = (OP == B_INIT_BICG || OP == B_CG_INIT || OP == B_NORM2 || OP == B_NORM2X2) || !K->done;
    // scalars used by the update (read before any finalize of this launch)
    const double2 al = K->alpha, om = K->omega, be = K->beta;
    using real = typename PT<P>::real;
    real red[4] = {0, 0, 0, 0};
    if (active) {
        const int base = tile * (SPT * blockDim.x) + threadIdx.x;
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int i = base + k * blockDim.x;
            if (i < d.g.Vh) blas_site<P, OP>(bp, d, i, al, om, be, red);
        }
    }
    constexpr bool HAS_RED = OP != B_S && OP != B_P && OP != B_MR;
    if (!HAS_RED) return;
    if (!active) return;   // whole system inactive: every block of it returns here
    double tot[4];
    if (!reduce_sys<4, real>(RedCtx{bp.map, bp.partials, bp.tickets}, s, red, tot)) return;
    if (threadIdx.x != 0) return;
    if (bp.red_out) {
#pragma unroll
        for (int k = 0; k < 4; ++k) bp.red_out[4 * s + k] = tot[k];
        return;
    }
    blas_finalize<OP>(*K, tot);
}

// p = z + beta p for CGNR (separate: needs the finalised beta)
template <int P, int SPT>
__global__ void __launch_bounds__(BLAS_B) k_cg_p(BlasParams bp) {
    using real = typename PT<P>::real;
    int s, tile;
    map_block(bp.map, s, tile);
    const SysDesc& d = bp.sys[s];
    if (bp.sc[s].done) return;
    const real be = (real)bp.sc[s].beta.x;
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
        const int i = tile * (SPT * blockDim.x) + k * blockDim.x + threadIdx.x;
        if (i >= d.g.Vh) break;
        cx<real> a[12], b[12];
        Access<P>::load_spinor(sys_view<P>(bp.v.z, d), i, a);
        Access<P>::load_spinor(sys_view<P>(bp.v.p, d), i, b);
#pragma unroll
        for (int c = 0; c < 12; ++c) a[c] = a[c] + be * b[c];
        Access<P>::store_spinor(sys_view<P>(bp.v.p, d), i, a);
    }
}

template <int P>
static void blas_t(const Batch& bt, int op, const BlasVecs& vv, KScal* sc, RedBuf& rb, cudaStream_t st,
                   double* red_out) {
    BPP_REQUIRE(!red_out || op != B_CG_BETA, BPP_ERR_UNSUPPORTED, "CG beta update has no deferred form");
    BlasParams bp;
    bp.red_out = red_out;
    bp.sys = bt.dev();
    int nb = 0;
    // BLAS_SPT sites per thread on large batches (few partials per reduction),
    // one per thread and smaller blocks on small ones
    const bool big = bt.sites() >= (int64_t)2 * 148 * BLAS_B * BLAS_SPT;
    const int vb = big ? BLAS_B : vec_block(bt);
    bp.map = block_map(bt, vb * (big ? BLAS_SPT : 1), nb);
    rb.ensure(nb, bt.nsys(), st);
    bp.v = vv;
    bp.sc = sc;
    bp.partials = rb.partials.as<double>();
    bp.tickets = rb.tickets.as<unsigned>();
    // vectors each op reads plus writes (its algorithmic traffic per site)
    static const int passes[] = {5, 2, 3, 2, 7, 4, 3, 2, 1, 6, 4, 1, 2, 5};
    ProfScope prof(PROF_BLAS, bt.sites() * spinor_bytes(P) * passes[op], st);
#define K_BLAS(OPC)                                                      \
    do {                                                                  \
        if (big) k_blas<P, OPC, BLAS_SPT><<<nb, vb, 0, st>>>(bp);         \
        else k_blas<P, OPC, 1><<<nb, vb, 0, st>>>(bp);                    \
    } while (0)
    switch (op) {
        case B_INIT_BICG: K_BLAS(B_INIT_BICG); break;
        case B_ALPHA: K_BLAS(B_ALPHA); break;
        case B_S: K_BLAS(B_S); break;
        case B_OMEGA: K_BLAS(B_OMEGA); break;
        case B_XR: K_BLAS(B_XR); break;
        case B_P: K_BLAS(B_P); break;
        case B_CG_INIT: K_BLAS(B_CG_INIT); break;
        case B_CG_PZ: K_BLAS(B_CG_PZ); break;
        case B_CG_ALPHA: K_BLAS(B_CG_ALPHA); break;
        case B_CG_XR: K_BLAS(B_CG_XR); break;
        case B_CG_BETA:
            K_BLAS(B_CG_BETA);
            count_launch();
            if (big) k_cg_p<P, BLAS_SPT><<<nb, vb, 0, st>>>(bp);
            else k_cg_p<P, 1><<<nb, vb, 0, st>>>(bp);
            break;
        case B_NORM2: K_BLAS(B_NORM2); break;
        case B_NORM2X2: K_BLAS(B_NORM2X2); break;
        case B_MR: K_BLAS(B_MR); break;
        default: throw Error(BPP_ERR_INVALID_ARG, "bad blas op");
    }
#undef K_BLAS
    count_launch();
    BPP_CHECK_LAUNCH();
}

void blas(const Batch& bt, int op, const BlasVecs& vv, KScal* sc, RedBuf& rb, cudaStream_t st, double* red_out) {
    BPP_REQUIRE(bt.prec != P64S, BPP_ERR_UNSUPPORTED, "Krylov vector kernels do not run on split-FP64 vectors");
    if (bt.prec == P64) blas_t<P64>(bt, op, vv, sc, rb, st, red_out);
    else if (bt.prec == P32) blas_t<P32>(bt, op, vv, sc, rb, st, red_out);
    else blas_t<P16>(bt, op, vv, sc, rb, st, red_out);
}

void blas_fin(int op, KScal* sc, const double* tot, int n, cudaStream_t st) {
    ProfScope prof(PROF_CTL, 0.0, st);
    switch (op) {
        case B_INIT_BICG: k_blas_fin<B_INIT_BICG><<<1, 64, 0, st>>>(sc, tot, n); break;
        case B_ALPHA: k_blas_fin<B_ALPHA><<<1, 64, 0, st>>>(sc, tot, n); break;
        case B_OMEGA: k_blas_fin<B_OMEGA><<<1, 64, 0, st>>>(sc, tot, n); break;
        case B_XR: k_blas_fin<B_XR><<<1, 64, 0, st>>>(sc, tot, n); break;
        case B_NORM2: k_blas_fin<B_NORM2><<<1, 64, 0, st>>>(sc, tot, n); break;
        case B_NORM2X2: k_blas_fin<B_NORM2X2><<<1, 64, 0, st>>>(sc, tot, n); break;
        default: throw Error(BPP_ERR_UNSUPPORTED, "no deferred finalize for this vector operation");
    }
    count_launch();
    BPP_CHECK_LAUNCH();
}

// Sum of one system's per-warp partials of a fused hop (see hop_red_fin) in
// two fixed levels: block c of system s sums partials [c RF_CH, (c+1) RF_CH)
// (thread t adds t, t + RF_B, ... in order, its loads issued together, then
// the warps' and the block's sums in order) into a chunk sum; the last block
// of the system, found with a ticket, sums the chunk sums the same way (thread
// t adds chunks t, t + RF_B, ...) and derives alpha or omega.  The grouping
// depends only on the lattice.
constexpr int RF_B = 256;
constexpr int RF_CH = 8 * RF_B;

// Block sum of three values per thread in a fixed order (warp shuffles, then
// the warps in order); valid in thread 0.
__device__ __forceinline__ void rf_block_sum(double a[3], double (*sh)[3]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double b = a[k];
        for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
        if (lane == 0) sh[warp][k] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double b = 0.0;
            for (int w = 0; w < RF_B / 32; ++w) b += sh[w][k];
            a[k] = b;
        }
    }
}

template <int OP>
__global__ void __launch_bounds__(RF_B) k_hop_red_fin(const SysDesc* sys, KScal* sc, const double* part, int wstride,
                                                      double* chunks, int chunk_stride, unsigned* tickets) {
    const int s = blockIdx.y, c = blockIdx.x;
    KScal& K = sc[s];
    if (K.done) return;
    const int nw = (sys[s].g.Vh + 31) >> 5;
    const int nch = (nw + RF_CH - 1) / RF_CH;
    if (c >= nch) return;
    const double* p = part + (size_t)s * wstride * 4;
    double a[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < RF_CH / RF_B; ++j) {
        const int w = c * RF_CH + j * RF_B + threadIdx.x;
        if (w < nw) {
#pragma unroll
            for (int k = 0; k < 3; ++k) a[k] += p[4 * w + k];
        }
    }
    __shared__ double sh[RF_B / 32][3];
    __shared__ int last;
    rf_block_sum(a, sh);
    double* c0 = chunks + (size_t)s * chunk_stride * 4;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) c0[4 * c + k] = a[k];
        __threadfence();
        last = atomicAdd(&tickets[s], 1u) == (unsigned)(nch - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = 0.0;
    for (int j = threadIdx.x; j < nch; j += RF_B)
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] += __ldcg(&c0[4 * j + k]);
    rf_block_sum(a, sh);
    if (threadIdx.x != 0) return;
    tickets[s] = 0u;
    double tot[4] = {a[0], a[1], a[2], 0.0};
    blas_finalize<OP>(K, tot);
}

int hop_red_chunks(int wstride) { return (wstride + RF_CH - 1) / RF_CH; }

void hop_red_fin(const Batch& bt, int op, const double* part, int wstride, KScal* sc, RedBuf& rb, double* chunks,
                 cudaStream_t st) {
    rb.ensure(0, bt.nsys(), st);
    const int nch = hop_red_chunks(wstride);
    const dim3 grid(nch, bt.nsys());
    unsigned* tk = rb.tickets.as<unsigned>();
    ProfScope prof(PROF_BLAS, (double)bt.nsys() * wstride * 3 * sizeof(double), st);
    if (op == B_ALPHA) k_hop_red_fin<B_ALPHA><<<grid, RF_B, 0, st>>>(bt.dev(), sc, part, wstride, chunks, nch, tk);
    else if (op == B_OMEGA) k_hop_red_fin<B_OMEGA><<<grid, RF_B, 0, st>>>(bt.dev(), sc, part, wstride, chunks, nch, tk);
    else throw Error(BPP_ERR_INVALID_ARG, "fused hop reductions finalize alpha or omega");
    count_launch();
    BPP_CHECK_LAUNCH();
}

// ----------------------------------------------------------------------------- outer loop
// Compiler barrier: the loads issued before it stay ahead of the stores that
// follow, so a thread has all of them in flight at once.
__device__ __forceinline__ void loads_issued() { asm volatile("" ::: "memory"); }

struct OuterParams {
    const SysDesc* s64;
    const SysDesc* sP;
    BlockMap map;
    char* a;
    char* b;
    char* c;           // optional third vector (split-FP64 outputs / inputs)
    KScal* sc;
    double* partials;
    unsigned* tickets;
    double* red_out = nullptr;   // set (residual kernels): write the sums here [s][4] instead of sc
};

__global__ void __launch_bounds__(BLAS_B) k_outer_residual(OuterParams op) {
    int s, tile;
    map_block(op.map, s, tile);
    const SysDesc& d = op.s64[s];
    const int i = tile * blockDim.x + threadIdx.x;
    double red[4] = {0, 0, 0, 0};
    if (i < d.g.Vh) {
        cx<double> bh[12], r[12];
        Access<P64>::load_spinor(sys_view<P64>(op.a, d), i, bh);
        Access<P64>::load_spinor(sys_view<P64>(op.b, d), i, r);
#pragma unroll
        for (int k = 0; k < 12; ++k) r[k] = bh[k] - r[k];
        Access<P64>::store_spinor(sys_view<P64>(op.b, d), i, r);
        red[0] = norm12(r);
    }
    double tot[4];
    if (!reduce_sys<4, double>(RedCtx{op.map, op.partials, op.tickets}, s, red, tot)) return;
    if (threadIdx.x == 0) {
        if (op.red_out) {
            for (int k = 0; k < 4; ++k) op.red_out[4 * s + k] = tot[k];
            return;
        }
        op.sc[s].rr = tot[0];
        op.sc[s].scale = sqrt(tot[0]);
    }
}

template <int P, bool SPLIT>
__global__ void __launch_bounds__(BLAS_B) k_outer_down(OuterParams op) {
    using real = typename PT<P>::real;
    int s, tile;
    map_block(op.map, s, tile);
    const SysDesc& d = op.s64[s];
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= d.g.Vh) return;
    const double sc = op.sc[s].scale;
    const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
    cx<real> lo[12];
    if (SPLIT) {
        // the defect's high parts carry all the accuracy the inner precision can hold
        const float invf = (float)inv;
        cx<df64> r[12];
        Access<P64S>::load_spinor(sys_view<P64S>(op.a, d), i, r);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            if (P == P64) lo[k] = mkc<real>((real)(r[k].r.to_double() * inv), (real)(r[k].i.to_double() * inv));
            else lo[k] = mkc<real>((real)(r[k].r.hi * invf), (real)(r[k].i.hi * invf));
        }
    } else {
        cx<double> r[12];
        Access<P64>::load_spinor(sys_view<P64>(op.a, d), i, r);
#pragma unroll
        for (int k = 0; k < 12; ++k) lo[k] = mkc<real>((real)(r[k].r * inv), (real)(r[k].i * inv));
    }
    Access<P>::store_spinor(sys_view<P>(op.b, op.sP[s]), i, lo);
}

__device__ __forceinline__ df64 to_df(float v) { return df64(v, 0.f); }
__device__ __forceinline__ df64 to_df(double v) { return df64(v); }


template <int P>
__global__ void __launch_bounds__(BLAS_B, 2) k_outer_acc(OuterParams op) {
    using real = typename PT<P>::real;
    int s, tile;
    map_block(op.map, s, tile);
    const SysDesc& d = op.s64[s];
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= d.g.Vh) return;
    const double sc = op.sc[s].scale;
    cx<real> e[12];
    Access<P>::load_spinor(sys_view<P>(op.b, op.sP[s]), i, e);
    double2* xp = op.a ? reinterpret_cast<double2*>(op.a + d.vec_off) : nullptr;
    float4* xsp = op.c ? reinterpret_cast<float4*>(op.c + d.vec_off) : nullptr;
    const df64 scd(sc);
    // half a spinor of x at a time: its loads are issued together (the
    // compiler barrier keeps them ahead of the stores, which it cannot prove
    // independent of them), without holding a whole FP64 or split spinor
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double2 xv[6];
        float4 xs[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int64_t j = (6 * h + k) * d.stride + i;
            if (xp) xv[k] = xp[j];
            if (xsp) xs[k] = xsp[j];
        }
        loads_issued();
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int64_t j = (6 * h + k) * d.stride + i;
            const cx<real> ek = e[6 * h + k];
            if (xp) {
                double2 xk = xv[k];
                xk.x = fma(sc, (double)ek.r, xk.x);
                xk.y = fma(sc, (double)ek.i, xk.y);
                xp[j] = xk;
            }
            if (xsp) {
                // the split copy takes the same update in double-float arithmetic
                // (no FP64 conversions); beside an FP64 x it tracks x to ~1e-14 and
                // only feeds the defects, without one (x64 null) it is the iterate
                const float4 v = xs[k];
                const df64 r = normalized(fma(scd, to_df(ek.r), df64(v.x, v.y)));
                const df64 m = normalized(fma(scd, to_df(ek.i), df64(v.z, v.w)));
                xsp[j] = make_float4(r.hi, r.lo, m.hi, m.lo);
            }
        }
    }
}

// r = bhat - m in double-float from split-FP64 bhat (op.a) and m (op.b, may
// be null), written split to op.c, with ||r||^2 per system from the high parts
// (FP32 per site, FP64 across sites: relative accuracy ~1e-7, ample for the
// convergence test and the defect scale).  Split vectors share the FP64
// vectors' offsets and strides (both 192 B per site).
__global__ void __launch_bounds__(BLAS_B) k_split_residual(OuterParams op) {
    int s, tile;
    map_block(op.map, s, tile);
    const SysDesc& d = op.s64[s];
    const int i = tile * blockDim.x + threadIdx.x;
    float red[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < d.g.Vh) {
        // half a spinor at a time, its loads issued together (no whole split
        // spinor held in registers)
        const float4* pa = reinterpret_cast<const float4*>(op.a + d.vec_off);
        const float4* pb = op.b ? reinterpret_cast<const float4*>(op.b + d.vec_off) : nullptr;
        float4* pc = reinterpret_cast<float4*>(op.c + d.vec_off);
        float n = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4 va[6], vb[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int64_t j = (6 * h + k) * d.stride + i;
                va[k] = pa[j];
                if (pb) vb[k] = pb[j];
            }
            loads_issued();
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                df64 r(va[k].x, va[k].y), m(va[k].z, va[k].w);
                if (pb) {
                    r = r - df64(vb[k].x, vb[k].y);
                    m = m - df64(vb[k].z, vb[k].w);
                }
                r = normalized(r);
                m = normalized(m);
                pc[(6 * h + k) * d.stride + i] = make_float4(r.hi, r.lo, m.hi, m.lo);
                n = fmaf(r.hi, r.hi, n);
                n = fmaf(m.hi, m.hi, n);
            }
        }
        red[0] = n;
    }
    double tot[4];
    if (!reduce_sys<4, float>(RedCtx{op.map, op.partials, op.tickets}, s, red, tot)) return;
    if (threadIdx.x == 0) {
        op.sc[s].rr = tot[0];
        op.sc[s].scale = sqrt(tot[0]);
    }
}

// Copy of an inner-precision vector (op.a, batch sP) as FP32 (op.b, batch s64
// holds the FP32 batch here).
template <int PIN>
__global__ void __launch_bounds__(BLAS_B) k_to_f32(OuterParams op) {
    using real = typename PT<PIN>::real;
    int s, tile;
    map_block(op.map, s, tile);
    const SysDesc& d = op.s64[s];
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= d.g.Vh) return;
    cx<real> v[12];
    cx<float> w[12];
    Access<PIN>::load_spinor(sys_view<PIN>(op.a, op.sP[s]), i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = mkc((float)v[k].r, (float)v[k].i);
    Access<P32>::store_spinor(sys_view<P32>(op.b, d), i, w);
}

void to_f32(const Batch& bin, const Batch& b32, const char* in, char* out, cudaStream_t st) {
    OuterParams op;
    op.s64 = b32.dev();
    op.sP = bin.dev();
    int nb = 0;
    const int vb = vec_block(b32);
    op.map = block_map(b32, vb, nb);
    op.a = const_cast<char*>(in);
    op.b = out;
    op.c = nullptr;
    op.sc = nullptr;
    ProfScope prof(PROF_OUTER, b32.sites() * (96.0 + spinor_bytes(bin.prec)), st);
    if (bin.prec == P16) k_to_f32<P16><<<nb, vb, 0, st>>>(op);
    else if (bin.prec == P32) k_to_f32<P32><<<nb, vb, 0, st>>>(op);
    else throw Error(BPP_ERR_UNSUPPORTED, "to_f32 takes FP16 or FP32 vectors");
    count_launch();
    BPP_CHECK_LAUNCH();
}

// Recursive defect update r_s -= scale * m (m = Mhat e in FP32, op.b with the
// FP32 batch in sP), double-float, with ||r_s||^2 from the high parts.
__global__ void __launch_bounds__(BLAS_B) k_defect_update(OuterParams op) {
    int s, tile;
    map_block(op.map, s, tile);
    const SysDesc& d = op.s64[s];
    const int i = tile * blockDim.x + threadIdx.x;
    const df64 sc = df64(-op.sc[s].scale);
    float red[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < d.g.Vh) {
        cx<float> m[12];
        Access<P32>::load_spinor(sys_view<P32>(op.b, op.sP[s]), i, m);
        float4* pr = reinterpret_cast<float4*>(op.a + d.vec_off);
        float n = 0.f;
        // half a spinor of r at a time, its loads issued together with m's
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4 rv[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) rv[k] = pr[(6 * h + k) * d.stride + i];
            loads_issued();
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const cx<float> mk = m[6 * h + k];
                const df64 r = normalized(fma(sc, df64(mk.r, 0.f), df64(rv[k].x, rv[k].y)));
                const df64 q = normalized(fma(sc, df64(mk.i, 0.f), df64(rv[k].z, rv[k].w)));
                pr[(6 * h + k) * d.stride + i] = make_float4(r.hi, r.lo, q.hi, q.lo);
                n = fmaf(r.hi, r.hi, n);
                n = fmaf(q.hi, q.hi, n);
            }
        }
        red[0] = n;
    }
    double tot[4];
    if (!reduce_sys<4, float>(RedCtx{op.map, op.partials, op.tickets}, s, red, tot)) return;
    if (threadIdx.x == 0) {
        op.sc[s].rr = tot[0];
        op.sc[s].scale = sqrt(tot[0]);
    }
}

void defect_update(const Batch& b64, const Batch& b32, char* r_s, const char* m32, KScal* sc, RedBuf& rb,
                   cudaStream_t st) {
    OuterParams op;
    op.s64 = b64.dev();
    op.sP = b32.dev();
    int nb = 0;
    const int vb = vec_block(b64);
    op.map = block_map(b64, vb, nb);
    rb.ensure(nb, b64.nsys(), st);
    op.a = r_s;
    op.b = const_cast<char*>(m32);
    op.c = nullptr;
    op.sc = sc;
    op.partials = rb.partials.as<double>();
    op.tickets = rb.tickets.as<unsigned>();
    ProfScope prof(PROF_OUTER, b64.sites() * (2 * 192.0 + 96.0), st);
    k_defect_update<<<nb, vb, 0, st>>>(op);
    count_launch();
    BPP_CHECK_LAUNCH();
}


// v (op.a) *= scale in place (FP64) and op.b = its split-FP64 copy (op.b may be null).
__global__ void __launch_bounds__(BLAS_B) k_scale_split(OuterParams op) {
    int s, tile;
    map_block(op.map, s, tile);
    const SysDesc& d = op.s64[s];
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= d.g.Vh) return;
    const double f = op.sc[s].scale;
    cx<double> v[12];
    Access<P64>::load_spinor(sys_view<P64>(op.a, d), i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = f * v[k];
    if (op.c) Access<P64>::store_spinor(sys_view<P64>(op.a, d), i, v);
    if (op.b) {
        cx<df64> w[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = mkc(df64(v[k].r), df64(v[k].i));
        Access<P64S>::store_spinor(sys_view<P64S>(op.b, d), i, w);
    }
}


static void launch_outer(void (*kern)(OuterParams), const Batch& b64, char* a, char* b, KScal* sc, double bytes,
                         cudaStream_t st, char* c = nullptr) {
    OuterParams op;
    op.s64 = b64.dev();
    op.sP = b64.dev();
    int nb = 0;
    const int vb = vec_block(b64);
    op.map = block_map(b64, vb, nb);
    op.a = a;
    op.b = b;
    op.c = c;
    op.sc = sc;
    ProfScope prof(PROF_OUTER, bytes, st);
    kern<<<nb, vb, 0, st>>>(op);
    count_launch();
    BPP_CHECK_LAUNCH();
}

void scale_split(const Batch& b64, char* v, char* out, KScal* sc, cudaStream_t st, bool keep64) {
    BPP_REQUIRE(keep64 || out, BPP_ERR_INVALID_ARG, "scale_split: nothing to write");
    launch_outer(k_scale_split, b64, v, out, sc, b64.sites() * (192.0 + (keep64 ? 192.0 : 0.0) + (out ? 192.0 : 0.0)),
                 st, keep64 ? v : nullptr);
}

// Odd half of the final check, all FP64: with h = kappa H_oe x_e (op.b) and
// y = b_o + h, x_o = A_oo^-1 y (Wilson: y) is written to op.c and the odd
// residual b_o - (A_oo x_o - h) of the full D is reduced into sc.rr.
template <bool CLOVER>
__global__ void __launch_bounds__(BLAS_B) k_odd_reconstruct(OuterParams op) {
    int s, tile;
    map_block(op.map, s, tile);
    const SysDesc& d = op.s64[s];
    const int i = tile * blockDim.x + threadIdx.x;
    double red[4] = {0, 0, 0, 0};
    if (i < d.g.Vh) {
        cx<double> b[12], h[12], y[12], x[12], ax[12];
        Access<P64>::load_spinor(sys_view<P64>(op.a, d), i, b);
        Access<P64>::load_spinor(sys_view<P64>(op.b, d), i, h);
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = b[k] + h[k];
        if (CLOVER) {
            clover_apply_site<P64>(d.Ainv[1], i, y, x);
            clover_apply_site<P64>(d.A[1], i, x, ax);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) x[k] = ax[k] = y[k];
        }
        Access<P64>::store_spinor(sys_view<P64>(op.c, d), i, x);
        cx<double> r[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) r[k] = b[k] - (ax[k] - h[k]);
        red[0] = norm12(r);
    }
    double tot[4];
    if (!reduce_sys<4, double>(RedCtx{op.map, op.partials, op.tickets}, s, red, tot)) return;
    if (threadIdx.x == 0) op.sc[s].rr = tot[0];
}

void odd_reconstruct(const Batch& b64, bool clover, const char* bo, const char* h, char* xo, KScal* sc, RedBuf& rb,
                     cudaStream_t st) {
    OuterParams op;
    op.s64 = b64.dev();
    op.sP = b64.dev();
    int nb = 0;
    const int vb = vec_block(b64);
    op.map = block_map(b64, vb, nb);
    rb.ensure(nb, b64.nsys(), st);
    op.a = const_cast<char*>(bo);
    op.b = const_cast<char*>(h);
    op.c = xo;
    op.sc = sc;
    op.partials = rb.partials.as<double>();
    op.tickets = rb.tickets.as<unsigned>();
    ProfScope prof(PROF_OUTER, b64.sites() * (3 * 192.0 + (clover ? 2 * 576.0 : 0.0)), st);
    if (clover) k_odd_reconstruct<true><<<nb, vb, 0, st>>>(op);
    else k_odd_reconstruct<false><<<nb, vb, 0, st>>>(op);
    count_launch();
    BPP_CHECK_LAUNCH();
}

void split_residual(const Batch& b64, char* bhat_s, char* m_s, char* r64, KScal* sc, RedBuf& rb, cudaStream_t st) {
    OuterParams op;
    op.s64 = b64.dev();
    op.sP = b64.dev();
    int nb = 0;
    const int vb = vec_block(b64);
    op.map = block_map(b64, vb, nb);
    rb.ensure(nb, b64.nsys(), st);
    op.a = bhat_s;
    op.b = m_s;
    op.c = r64;
    op.sc = sc;
    op.partials = rb.partials.as<double>();
    op.tickets = rb.tickets.as<unsigned>();
    ProfScope prof(PROF_OUTER, b64.sites() * (m_s ? 3 : 2) * 192.0, st);
    k_split_residual<<<nb, vb, 0, st>>>(op);
    count_launch();
    BPP_CHECK_LAUNCH();
}

void outer_residual(const Batch& b64, char* bhat, char* r64, KScal* sc, RedBuf& rb, cudaStream_t st,
                    double* red_out) {
    OuterParams op;
    op.red_out = red_out;
    op.s64 = b64.dev();
    op.sP = b64.dev();
    int nb = 0;
    const int vb = vec_block(b64);
    op.map = block_map(b64, vb, nb);
    rb.ensure(nb, b64.nsys(), st);
    op.a = bhat;
    op.b = r64;
    op.c = nullptr;
    op.sc = sc;
    op.partials = rb.partials.as<double>();
    op.tickets = rb.tickets.as<unsigned>();
    ProfScope prof(PROF_OUTER, b64.sites() * 3 * 192.0, st);
    k_outer_residual<<<nb, vb, 0, st>>>(op);
    count_launch();
    BPP_CHECK_LAUNCH();
}

void outer_downcast(const Batch& b64, const Batch& bP, const char* r64, char* lo, const KScal* sc, cudaStream_t st,
                    bool split) {
    OuterParams op;
    op.s64 = b64.dev();
    op.sP = bP.dev();
    int nb = 0;
    const int vb = vec_block(b64);
    op.map = block_map(b64, vb, nb);
    op.a = const_cast<char*>(r64);
    op.b = lo;
    op.c = nullptr;
    op.sc = const_cast<KScal*>(sc);
    ProfScope prof(PROF_OUTER, b64.sites() * (192.0 + spinor_bytes(bP.prec)), st);
    if (split) {
        if (bP.prec == P64) k_outer_down<P64, true><<<nb, vb, 0, st>>>(op);
        else if (bP.prec == P32) k_outer_down<P32, true><<<nb, vb, 0, st>>>(op);
        else k_outer_down<P16, true><<<nb, vb, 0, st>>>(op);
    } else {
        if (bP.prec == P64) k_outer_down<P64, false><<<nb, vb, 0, st>>>(op);
        else if (bP.prec == P32) k_outer_down<P32, false><<<nb, vb, 0, st>>>(op);
        else k_outer_down<P16, false><<<nb, vb, 0, st>>>(op);
    }
    count_launch();
    BPP_CHECK_LAUNCH();
}

void outer_accumulate(const Batch& b64, const Batch& bP, char* x64, const char* e, const KScal* sc, cudaStream_t st,
                      char* x_split) {
    OuterParams op;
    op.s64 = b64.dev();
    op.sP = bP.dev();
    int nb = 0;
    const int vb = vec_block(b64);
    op.map = block_map(b64, vb, nb);
    op.a = x64;
    op.b = const_cast<char*>(e);
    op.c = x_split;
    op.sc = const_cast<KScal*>(sc);
    ProfScope prof(PROF_OUTER, b64.sites() * ((x64 ? 2 * 192.0 : 0.0) + spinor_bytes(bP.prec) + (x_split ? 2 * 192.0 : 0.0)), st);
    if (bP.prec == P64) k_outer_acc<P64><<<nb, vb, 0, st>>>(op);
    else if (bP.prec == P32) k_outer_acc<P32><<<nb, vb, 0, st>>>(op);
    else k_outer_acc<P16><<<nb, vb, 0, st>>>(op);
    count_launch();
    BPP_CHECK_LAUNCH();
}

}  // namespace bpp
