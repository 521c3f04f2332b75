// Two-level aggregation multigrid preconditioner for the full-lattice Wilson /
// Wilson-clover matrix D of Eq. (1) (the multi-grid solver the paper names
// among the algorithms of the code set, Sec. 1 and Sec. 4), inside the
// mixed-precision defect correction of the solve (Sec. 2):
//
//   setup    six near-null vectors v_k (the caller's vectors, optionally
//            improved by approximate solves D v = v); the lattice is cut into
//            blocks of bs[0] x .. x bs[3] sites; on every block and chirality
//            (spins 0,1 / spins 2,3) the vectors restricted there are
//            orthonormalised (Gram-Schmidt), giving the prolongator P whose
//            columns are those restricted vectors: 12 coarse degrees of freedom
//            per block;
//   coarse   D_c = P^dag D P, a nearest-neighbour stencil on the block lattice
//            (a 12x12 self term and one 12x12 term per direction and sense);
//   V-cycle  z = M r: minimal-residual smoothing steps on D, restriction
//            r_c = P^dag s, an approximate coarse solve D_c e_c = r_c
//            (BiCGStab), prolongation z += P e_c, the residual recomputed,
//            further smoothing steps;
//   solve    flexible GCR on D preconditioned by M in FP32, restarted, under
//            the FP64 defect correction (r = b - D x in FP64, x += |r| e).
//
// Fields are in the full-lattice layout of lex.h (FP32 for the whole
// preconditioner).  Coarse vectors have exactly 12 complex numbers per block,
// the shape of a spinor, so the solver's vector kernels run on them
// unchanged (one "site" per block).  Every reduction is done in a fixed order:
// the results do not depend on scheduling.
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "blas.h"
#include "clover_dev.h"
#include "hop_dev.h"
#include "lex.h"
#include "mg.h"
#include "solver.h"

namespace bpp {

int work_read(int prec, int64_t* n, double* bytes, int reset);

// Index of the prolongator plane of (chirality, spin within it, colour, vector).
__host__ __device__ __forceinline__ int pidx(int chi, int s2, int col, int k) { return ((chi * 2 + s2) * 3 + col) * 6 + k; }

struct MGGeom {
    Geom g;           // fine lattice
    int64_t S;        // fine half-field plane stride; full fields use 2 S
    int bs[4], Lc[4];
    int bv;           // sites per block
    int64_t Vc, Sc;   // blocks, coarse plane stride
};

// fine position (lexical layout) of coordinates x
__device__ __forceinline__ int64_t fine_pos(const MGGeom& m, const int x[4]) {
    const int64_t lex = x[0] + (int64_t)m.g.L[0] * (x[1] + (int64_t)m.g.L[1] * (x[2] + (int64_t)m.g.L[2] * x[3]));
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    return (int64_t)p * m.S + (lex >> 1);
}
__device__ __forceinline__ int64_t block_of(const MGGeom& m, const int x[4]) {
    return x[0] / m.bs[0] + (int64_t)m.Lc[0] * (x[1] / m.bs[1] + (int64_t)m.Lc[1] * (x[2] / m.bs[2] + (int64_t)m.Lc[2] * (x[3] / m.bs[3])));
}
// coordinates of local site t of block B
__device__ __forceinline__ void block_site(const MGGeom& m, int64_t B, int t, int x[4]) {
    int64_t b = B;
    int bc[4];
    bc[0] = (int)(b % m.Lc[0]); b /= m.Lc[0];
    bc[1] = (int)(b % m.Lc[1]); b /= m.Lc[1];
    bc[2] = (int)(b % m.Lc[2]); bc[3] = (int)(b / m.Lc[2]);
    int l = t;
    for (int mu = 0; mu < 4; ++mu) {
        x[mu] = bc[mu] * m.bs[mu] + l % m.bs[mu];
        l /= m.bs[mu];
    }
}

// Deterministic block-wide sum of N doubles (all threads get the result).
template <int N>
__device__ void block_sum(double v[N], double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double a = v[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[warp * N + k] = a;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += sh[w * N + threadIdx.x];
        sh[32 * N + threadIdx.x] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = sh[32 * N + k];
    __syncthreads();
}

// ----------------------------------------------------------------------------- setup
// One block per (coarse site, chirality): Gram-Schmidt of the six vectors
// restricted to the block and chirality (inner products summed in FP64 in a
// fixed order), written as prolongator columns.
__global__ void __launch_bounds__(256) k_mg_orth(MGGeom m, const char* vecs, int64_t fbytes, float2* P) {
    __shared__ double sh[33 * 2];
    const int64_t B = blockIdx.x;
    const int chi = blockIdx.y;
    const int64_t S2 = 2 * m.S;
    int x[4];
    block_site(m, B, threadIdx.x, x);
    const int64_t j = fine_pos(m, x);
    cx<float> v[6][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        cx<float> s[12];
        Access<P32>::load_spinor(make_spinor_view(P32, const_cast<char*>(vecs) + k * fbytes, S2), j, s);
#pragma unroll
        for (int e = 0; e < 6; ++e) v[k][e] = s[chi * 6 + e];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int q = 0; q < k; ++q) {
            float dr = 0.f, di = 0.f;   // <v_q, v_k> at this site
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                dr = fmaf(v[q][e].r, v[k][e].r, fmaf(v[q][e].i, v[k][e].i, dr));
                di = fmaf(v[q][e].r, v[k][e].i, fmaf(-v[q][e].i, v[k][e].r, di));
            }
            double d[2] = {dr, di};
            block_sum<2>(d, sh);
            const cx<float> c = mkc((float)d[0], (float)d[1]);
#pragma unroll
            for (int e = 0; e < 6; ++e) v[k][e] = v[k][e] - c * v[q][e];
        }
        float nn = 0.f;
#pragma unroll
        for (int e = 0; e < 6; ++e) nn = fmaf(v[k][e].r, v[k][e].r, fmaf(v[k][e].i, v[k][e].i, nn));
        double n[1] = {nn};
        block_sum<1>(n, sh);
        const float inv = n[0] > 0.0 ? (float)(1.0 / sqrt(n[0])) : 0.f;
#pragma unroll
        for (int e = 0; e < 6; ++e) v[k][e] = inv * v[k][e];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int e = 0; e < 6; ++e) P[(int64_t)pidx(chi, e / 3, e % 3, k) * S2 + j] = make_float2(v[k][e].r, v[k][e].i);
}

// Column c = (chi', k') of the prolongator at fine position j, as a spinor.
__device__ __forceinline__ void pcol(const float2* P, int64_t S2, int64_t j, int c, cx<float> s[12]) {
    const int chi = c / 6, k = c % 6;
#pragma unroll
    for (int e = 0; e < 12; ++e) {
        const int sp = e / 3;
        if ((sp >> 1) == chi) {
            const float2 t = P[(int64_t)pidx(chi, sp & 1, e % 3, k) * S2 + j];
            s[e] = mkc(t.x, t.y);
        } else {
            s[e] = mkc(0.f, 0.f);
        }
    }
}

// rows[chi * 6 + k] = sum_e conj(P_(chi,k)(x))_e w_e at one fine site
__device__ __forceinline__ void prow(const float2* P, int64_t S2, int64_t j, const cx<float> w[12], double r[24]) {
#pragma unroll
    for (int chi = 0; chi < 2; ++chi)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            // per site in FP32 (six terms), across the block in FP64
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                const float2 p = P[(int64_t)pidx(chi, e / 3, e % 3, k) * S2 + j];
                const cx<float> q = w[chi * 6 + e];
                re = fmaf(p.x, q.r, fmaf(p.y, q.i, re));
                im = fmaf(p.x, q.i, fmaf(-p.y, q.r, im));
            }
            r[2 * (chi * 6 + k)] = re;
            r[2 * (chi * 6 + k) + 1] = im;
        }
}

template <int MU, bool BACK>
__device__ __forceinline__ void hop_dir(const SysDesc& d, const MGGeom& m, const int x[4], const int y[4], int px,
                                        int py, const cx<float> psi[12], bool flip, cx<float> acc[12]) {
    // forward: (1 - gamma_mu) U_mu(x) psi(x + mu); backward: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
    constexpr int S = BACK ? +1 : -1;
    cx<float> h[6], u[9], g[6];
    project<MU, S>(psi, h);
    if (flip) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = -h[k];
    }
    const int* c = BACK ? y : x;
    const int pc = BACK ? py : px;
    const int64_t lex = c[0] + (int64_t)m.g.L[0] * (c[1] + (int64_t)m.g.L[1] * (c[2] + (int64_t)m.g.L[2] * c[3]));
    Access<P32>::load_link(d.U[pc][MU], lex >> 1, u);
    link_mul<BACK>(u, h, g);
    reconstruct<MU, S>(acc, g);
}

// Coarse operator D_c = P^dag D P, one block per (coarse site B, stencil term
// t, column c): term 0 = everything that stays inside the block (the site
// term 1 + F and the hops that do not cross a block face), term 1 + 2 mu + s =
// the hops across the block face in direction mu forward (s = 0) or backward.
__global__ void __launch_bounds__(256) k_mg_coarse_build(MGGeom m, const float2* P, const SysDesc* sys, float2* Dc) {
    __shared__ double sh[33 * 24];
    const SysDesc& d = sys[0];
    const int64_t B = blockIdx.x;
    const int term = blockIdx.y, c = blockIdx.z;
    const int64_t S2 = 2 * m.S;
    int x[4];
    block_site(m, B, threadIdx.x, x);
    const int px = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int64_t jx = fine_pos(m, x);
    cx<float> w[12], acc[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) w[e] = acc[e] = mkc(0.f, 0.f);
    if (term == 0) {
        cx<float> s[12];
        pcol(P, S2, jx, c, s);
        if (d.A[0].data) clover_apply_site<P32>(d.A[px], (((int64_t)x[0] + (int64_t)m.g.L[0] * (x[1] + (int64_t)m.g.L[1] * (x[2] + (int64_t)m.g.L[2] * x[3]))) >> 1), s, w);
        else
#pragma unroll
            for (int e = 0; e < 12; ++e) w[e] = s[e];
    }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int back = 0; back < 2; ++back) {
            const int l = x[mu] % m.bs[mu];
            const bool cross = back ? l == 0 : l == m.bs[mu] - 1;
            // term 0 takes the hops inside the block, term 1 + 2 mu + back the
            // hop across that face
            if (term == 0 ? cross : (term != 1 + 2 * mu + back || !cross)) continue;
            int y[4] = {x[0], x[1], x[2], x[3]};
            const bool wrap = back ? x[mu] == 0 : x[mu] == m.g.L[mu] - 1;
            y[mu] = back ? (wrap ? m.g.L[mu] - 1 : x[mu] - 1) : (wrap ? 0 : x[mu] + 1);
            const bool flip = wrap && m.g.bc[mu] < 0;
            cx<float> s[12];
            pcol(P, S2, fine_pos(m, y), c, s);
            const int py = 1 - px;
            switch (2 * mu + back) {
                case 0: hop_dir<0, false>(d, m, x, y, px, py, s, flip, acc); break;
                case 1: hop_dir<0, true>(d, m, x, y, px, py, s, flip, acc); break;
                case 2: hop_dir<1, false>(d, m, x, y, px, py, s, flip, acc); break;
                case 3: hop_dir<1, true>(d, m, x, y, px, py, s, flip, acc); break;
                case 4: hop_dir<2, false>(d, m, x, y, px, py, s, flip, acc); break;
                case 5: hop_dir<2, true>(d, m, x, y, px, py, s, flip, acc); break;
                case 6: hop_dir<3, false>(d, m, x, y, px, py, s, flip, acc); break;
                default: hop_dir<3, true>(d, m, x, y, px, py, s, flip, acc); break;
            }
        }
    const float mk = (float)(-d.kappa);
#pragma unroll
    for (int e = 0; e < 12; ++e) w[e] = cxfma(mk, acc[e], w[e]);
    double r[24];
    prow(P, S2, jx, w, r);
    block_sum<24>(r, sh);
    if (threadIdx.x < 12) {
        const int row = threadIdx.x;
        Dc[((int64_t)(term * 144 + row * 12 + c)) * m.Sc + B] = make_float2((float)r[2 * row], (float)r[2 * row + 1]);
    }
}

// ----------------------------------------------------------------------------- transfer
// fine (+)= P coarse, one thread per fine position
__global__ void k_mg_prolong(MGGeom m, const float2* P, const char* coarse, const SysDesc* csys, char* fine,
                             const SysDesc* fsys, int add) {
    const int s = blockIdx.y;
    const int64_t S2 = 2 * m.S;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S2) return;
    const int p = j >= m.S;
    const int i = (int)(j - p * m.S);
    if (i >= m.g.Vh) return;
    int x[4];
    eo_coords(m.g, i, p, x);
    const int64_t B = block_of(m, x);
    cx<float> cv[12], e[12];
    Access<P32>::load_spinor(sys_view<P32>(const_cast<char*>(coarse), csys[s]), B, cv);
    if (add) Access<P32>::load_spinor(sys_view<P32>(fine, fsys[s]), j, e);
    else
#pragma unroll
        for (int q = 0; q < 12; ++q) e[q] = mkc(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const int sp = q / 3, col = q % 3, chi = sp >> 1;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 t = P[(int64_t)pidx(chi, sp & 1, col, k) * S2 + j];
            cfma(e[q], mkc(t.x, t.y), cv[chi * 6 + k]);
        }
    }
    Access<P32>::store_spinor(sys_view<P32>(fine, fsys[s]), j, e);
}

// coarse = P^dag fine, one block per (coarse site, system)
__global__ void __launch_bounds__(256) k_mg_restrict(MGGeom m, const float2* P, const char* fine, const SysDesc* fsys, char* coarse,
                              const SysDesc* csys) {
    __shared__ double sh[33 * 24];
    const int64_t B = blockIdx.x;
    const int s = blockIdx.y;
    int x[4];
    block_site(m, B, threadIdx.x, x);
    const int64_t j = fine_pos(m, x);
    cx<float> w[12];
    Access<P32>::load_spinor(sys_view<P32>(const_cast<char*>(fine), fsys[s]), j, w);
    double r[24];
    prow(P, 2 * m.S, j, w, r);
    block_sum<24>(r, sh);
    if (threadIdx.x == 0) {
        cx<float> out[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) out[q] = mkc((float)r[2 * q], (float)r[2 * q + 1]);
        Access<P32>::store_spinor(sys_view<P32>(coarse, csys[s]), B, out);
    }
}

// out = D_c in, one thread per (coarse site, output component, system)
__global__ void __launch_bounds__(384) k_mg_coarse_apply(MGGeom m, const float2* Dc, const char* in, char* out,
                                                          const SysDesc* csys, const int* done, int ds) {
    // one thread per (coarse site, output component r): the coarse lattice
    // is small (Vc = V / block volume), so a thread per site would leave most
    // SMs idle; the warps run over 32 consecutive coarse sites, so the D_c
    // planes (site fastest) stay coalesced, and the 12 component warps of a
    // block share the neighbour loads through L1
    const int s = blockIdx.y;
    if (done && done[s * ds]) return;
    const int r = threadIdx.y;
    const int64_t B = (int64_t)blockIdx.x * 32 + threadIdx.x;
    if (B >= m.Vc) return;
    int b[4];
    {
        int64_t t = B;
        b[0] = (int)(t % m.Lc[0]); t /= m.Lc[0];
        b[1] = (int)(t % m.Lc[1]); t /= m.Lc[1];
        b[2] = (int)(t % m.Lc[2]); b[3] = (int)(t / m.Lc[2]);
    }
    const SpinorView vin = sys_view<P32>(const_cast<char*>(in), csys[s]);
    const float4* vp = static_cast<const float4*>(vin.data);
    cx<float> acc = mkc(0.f, 0.f);
    for (int term = 0; term < 9; ++term) {
        int nb[4] = {b[0], b[1], b[2], b[3]};
        if (term > 0) {
            const int mu = (term - 1) >> 1;
            nb[mu] = ((term - 1) & 1) ? (b[mu] - 1 + m.Lc[mu]) % m.Lc[mu] : (b[mu] + 1) % m.Lc[mu];
        }
        const int64_t Bn = nb[0] + (int64_t)m.Lc[0] * (nb[1] + (int64_t)m.Lc[1] * (nb[2] + (int64_t)m.Lc[2] * nb[3]));
        const float2* row = Dc + (int64_t)(term * 144 + r * 12) * m.Sc + B;
#pragma unroll
        for (int c2 = 0; c2 < 6; ++c2) {
            const float4 w = __ldg(vp + c2 * vin.stride + Bn);
            const float2 a0 = __ldg(row + (int64_t)(2 * c2) * m.Sc);
            const float2 a1 = __ldg(row + (int64_t)(2 * c2 + 1) * m.Sc);
            cfma(acc, mkc(a0.x, a0.y), mkc(w.x, w.y));
            cfma(acc, mkc(a1.x, a1.y), mkc(w.z, w.w));
        }
    }
    float2* op = reinterpret_cast<float2*>(static_cast<float4*>(sys_view<P32>(out, csys[s]).data) +
                                           (int64_t)(r >> 1) * csys[s].stride + B) + (r & 1);
    *op = make_float2(acc.r, acc.i);
}

// y = coef_s x (mode 0) or y += coef_s x (mode 1), per system coefficients
struct Coefs {
    double2 c[MAXSYS];
};
__global__ void k_mg_axpy(const SysDesc* sys, BlockMap map, char* y, const char* x, Coefs cf, int accumulate) {
    int s, tile;
    map_block(map, s, tile);
    const SysDesc& d = sys[s];
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= d.g.Vh) return;
    const cx<float> c = mkc((float)cf.c[s].x, (float)cf.c[s].y);
    cx<float> a[12], b[12];
    Access<P32>::load_spinor(sys_view<P32>(const_cast<char*>(x), d), i, a);
    if (accumulate) Access<P32>::load_spinor(sys_view<P32>(y, d), i, b);
    else
#pragma unroll
        for (int q = 0; q < 12; ++q) b[q] = mkc(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 12; ++q) cfma(b[q], c, a[q]);
    Access<P32>::store_spinor(sys_view<P32>(y, d), i, b);
}

}  // namespace bpp

// ----------------------------------------------------------------------------- handle
struct bpp_mg_s {
    bpp_gauge G = nullptr;
    double kappa = 0.0, csw = 0.0;
    bpp::MGGeom geom{};
    bpp::DevBuf P, Dc;
    bpp_mg_params prm{};
};

namespace bpp {

namespace {

void coarse_batch(Batch& cb, const MGGeom& m, int nrhs, cudaStream_t st) {
    cb.prec = P32;
    const size_t vb = spinor_alloc_bytes(P32, m.Sc);
    for (int r = 0; r < nrhs; ++r) {
        SysDesc d{};
        d.g.Vh = (int)m.Vc;
        d.stride = m.Sc;
        d.vec_off = (int64_t)(r * vb);
        cb.sys.push_back(d);
    }
    cb.vec_bytes = vb * nrhs;
    cb.Vh_max = (int)m.Vc;
    cb.uniform = true;
    cb.upload(st);
}

struct Buf {
    DevBuf b;
    char* p() const { return b.as<char>(); }
    void zero(size_t n, cudaStream_t st) {
        b.alloc(n, st);
        BPP_CUDA(cudaMemsetAsync(b.p, 0, n, st));
    }
};

// Workspace and steps of the preconditioned inner solve for nrhs systems.
struct MGRun {
    const bpp_mg_s& mg;
    int n;
    bool clover;
    LexBatches L;     // FP32 fine fields
    Batch cb;         // coarse fields
    RedBuf rb, rbc;
    DevBuf red, ks, kc;   // reduction sums, smoother and coarse solver scalars
    std::vector<double> hred;
    Buf s, t, z0;                                           // V-cycle fine work
    Buf cr, cx_, cr2, crh, cp, cv, cs, ct;                  // coarse BiCGStab
    MGRun(const bpp_mg_s& m, int nrhs, cudaStream_t st) : mg(m), n(nrhs), clover(m.csw != 0.0) {
        lex_batches(L, *m.G, P32, m.kappa, clover, n, st);
        coarse_batch(cb, m.geom, n, st);
        for (Buf* b : {&s, &t, &z0}) b->zero(L.vec.vec_bytes, st);
        for (Buf* b : {&cr, &cx_, &cr2, &crh, &cp, &cv, &cs, &ct}) b->zero(cb.vec_bytes, st);
        red.alloc((size_t)n * 4 * sizeof(double), st);
        ks.alloc(n * sizeof(KScal), st);
        kc.alloc(n * sizeof(KScal), st);
        BPP_CUDA(cudaMemsetAsync(ks.p, 0, n * sizeof(KScal), st));
        hred.resize((size_t)n * 4);
    }
    void axpy(const Batch& b, char* y, const char* x, const std::vector<double2>& c, bool acc, cudaStream_t st) {
        Coefs cf;
        for (int q = 0; q < n; ++q) cf.c[q] = c[q];
        for (int q = n; q < MAXSYS; ++q) cf.c[q] = make_double2(0.0, 0.0);
        int nb = 0;
        BlockMap map = block_map(b, 256, nb);
        ProfScope prof(PROF_OUTER, b.sites() * 96.0 * (acc ? 3 : 2), st);
        k_mg_axpy<<<nb, 256, 0, st>>>(b.dev(), map, y, x, cf, acc ? 1 : 0);
        count_launch();
        BPP_CHECK_LAUNCH();
    }
    // raw per-system sums of a reducing vector operation (no scalar update)
    const std::vector<double>& sums(const Batch& b, int op, const BlasVecs& v, KScal* sc, RedBuf& r, cudaStream_t st) {
        blas(b, op, v, sc, r, st, red.as<double>());
        BPP_CUDA(cudaMemcpyAsync(hred.data(), red.p, hred.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        BPP_CUDA(cudaStreamSynchronize(st));
        return hred;
    }
    void prolong(const char* c, char* f, bool add, cudaStream_t st) {
        const MGGeom& m = mg.geom;
        dim3 grid((unsigned)((2 * m.S + 127) / 128), n);
        ProfScope prof(PROF_OUTER, (double)n * (2 * m.S) * (96.0 * (add ? 2 : 1) + 72 * 8), st);
        k_mg_prolong<<<grid, 128, 0, st>>>(m, mg.P.as<float2>(), c, cb.dev(), f, L.vec.dev(), add ? 1 : 0);
        count_launch();
        BPP_CHECK_LAUNCH();
    }
    void restrict_(const char* f, char* c, cudaStream_t st) {
        const MGGeom& m = mg.geom;
        dim3 grid((unsigned)m.Vc, n);
        ProfScope prof(PROF_OUTER, (double)n * (2 * m.S) * (96.0 + 72 * 8), st);
        k_mg_restrict<<<grid, m.bv, 0, st>>>(m, mg.P.as<float2>(), f, L.vec.dev(), c, cb.dev());
        count_launch();
        BPP_CHECK_LAUNCH();
    }
    void coarse_apply(const char* in, char* out, cudaStream_t st) {
        const MGGeom& m = mg.geom;
        dim3 grid((unsigned)((m.Vc + 31) / 32), n);
        const KScal* k = kc.as<KScal>();
        ProfScope prof(PROF_OUTER, (double)n * m.Vc * (9 * 96.0 + 9 * 144 * 8 + 96), st);
        k_mg_coarse_apply<<<grid, dim3(32, 12), 0, st>>>(m, mg.Dc.as<float2>(), in, out, cb.dev(), &k[0].done,
                                                         (int)(sizeof(KScal) / sizeof(int)));
        count_launch();
        BPP_CHECK_LAUNCH();
    }
    // approximate coarse solve D_c e = r (BiCGStab, relative tolerance coarse_tol)
    void coarse_solve(char* r, char* e, cudaStream_t st) {
        std::vector<KScal> h(n);
        for (auto& k : h) {
            k = KScal{};
            k.tol2 = mg.prm.coarse_tol * mg.prm.coarse_tol;
            k.max_iter = mg.prm.coarse_maxiter;
        }
        BPP_CUDA(cudaMemcpyAsync(kc.p, h.data(), n * sizeof(KScal), cudaMemcpyHostToDevice, st));
        BlasVecs v;
        v.b = r; v.x = e; v.r = cr2.p(); v.rhat = crh.p(); v.p = cp.p(); v.v = cv.p(); v.s = cs.p(); v.t = ct.p();
        KScal* k = kc.as<KScal>();
        blas(cb, B_INIT_BICG, v, k, rbc, st);
        for (int chunk = 0; chunk * 4 < mg.prm.coarse_maxiter + 4; ++chunk) {
            for (int it = 0; it < 4; ++it) {
                coarse_apply(v.p, v.v, st);
                blas(cb, B_ALPHA, v, k, rbc, st);
                blas(cb, B_S, v, k, rbc, st);
                coarse_apply(v.s, v.t, st);
                blas(cb, B_OMEGA, v, k, rbc, st);
                blas(cb, B_XR, v, k, rbc, st);
                blas(cb, B_P, v, k, rbc, st);
            }
            BPP_CUDA(cudaMemcpyAsync(h.data(), kc.p, n * sizeof(KScal), cudaMemcpyDeviceToHost, st));
            BPP_CUDA(cudaStreamSynchronize(st));
            bool all = true;
            for (auto& q : h) all = all && q.done;
            if (all) break;
        }
    }
    // minimal-residual smoothing: nu steps on (z, s) with s the residual
    void smooth(char* z, int nu, cudaStream_t st) {
        BlasVecs v;
        v.x = z; v.s = s.p(); v.t = t.p();
        for (int q = 0; q < nu; ++q) {
            lex_apply(L, clover, 0, s.p(), t.p(), st);
            blas(L.vec, B_OMEGA, v, ks.as<KScal>(), rb, st);
            blas(L.vec, B_MR, v, ks.as<KScal>(), rb, st);
        }
    }
    // z = M r (V-cycle)
    void vcycle(const char* r, char* z, cudaStream_t st) {
        const std::vector<double2> one(n, make_double2(1.0, 0.0)), mone(n, make_double2(-1.0, 0.0)),
            zero(n, make_double2(0.0, 0.0));
        axpy(L.vec, z, r, zero, false, st);       // z = 0
        axpy(L.vec, s.p(), r, one, false, st);    // s = r
        smooth(z, mg.prm.nu_pre, st);
        restrict_(s.p(), cr.p(), st);
        coarse_solve(cr.p(), cx_.p(), st);
        prolong(cx_.p(), z, true, st);
        lex_apply(L, clover, 0, z, t.p(), st);    // s = r - D z
        axpy(L.vec, s.p(), r, one, false, st);
        axpy(L.vec, s.p(), t.p(), mone, true, st);
        smooth(z, mg.prm.nu_post, st);
    }
};

}  // namespace

// ----------------------------------------------------------------------------- entry points
void mg_create(bpp_gauge G, double kappa, double csw, const int bs[4], const void* vecs, int refine,
               const bpp_mg_params* prm, cudaStream_t st, bpp_mg_s** out) {
    BPP_REQUIRE(G && vecs && out && bs, BPP_ERR_INVALID_ARG, "NULL argument");
    const bool clover = csw != 0.0;
    if (clover)
        BPP_REQUIRE(G->has_clover && std::fabs(G->clov_kappa - kappa) <= 1e-14 * std::fabs(kappa) &&
                        std::fabs(G->clov_csw - csw) <= 1e-14 * std::fabs(csw),
                    BPP_ERR_UNSUPPORTED, "the clover term must be built with the same kappa and csw");
    std::unique_ptr<bpp_mg_s> mg(new bpp_mg_s());
    mg->G = G;
    mg->kappa = kappa;
    mg->csw = csw;
    bpp_mg_params_default(&mg->prm);
    if (prm) mg->prm = *prm;
    BPP_REQUIRE(mg->prm.nu_pre >= 0 && mg->prm.nu_post >= 0 && mg->prm.coarse_maxiter > 0 && mg->prm.gcr_restart > 0 &&
                    mg->prm.gcr_restart <= 64 && mg->prm.coarse_tol > 0.0,
                BPP_ERR_INVALID_ARG, "bad multigrid parameters");
    MGGeom& m = mg->geom;
    m.g = G->g;
    m.S = G->stride;
    m.bv = 1;
    for (int mu = 0; mu < 4; ++mu) {
        BPP_REQUIRE(bs[mu] >= 1 && G->g.L[mu] % bs[mu] == 0, BPP_ERR_INVALID_ARG,
                    "block extents must divide the lattice extents");
        m.bs[mu] = bs[mu];
        m.Lc[mu] = G->g.L[mu] / bs[mu];
        m.bv *= bs[mu];
    }
    BPP_REQUIRE(m.bv >= 32 && m.bv <= 256 && m.bv % 32 == 0, BPP_ERR_INVALID_ARG,
                "a block must hold 32..256 sites, a multiple of 32");
    m.Vc = G->V / m.bv;
    m.Sc = pad_stride(m.Vc);
    // near-null vectors: the caller's, optionally improved by approximate
    // solves v <- D^-1 v (one inverse-iteration step each)
    const size_t field = (size_t)G->V * 12 * 16;
    DevBuf v64(6 * field, st);
    BPP_CUDA(cudaMemcpyAsync(v64.p, vecs, 6 * field, cudaMemcpyDefault, st));
    for (int it = 0; it < refine; ++it) {
        DevBuf w(6 * field, st);
        std::vector<const Gauge*> Gs(6, G);
        std::vector<double> ks(6, kappa);
        std::vector<const void*> bv(6);
        std::vector<void*> xv(6);
        for (int k = 0; k < 6; ++k) {
            bv[k] = v64.as<char>() + k * field;
            xv[k] = w.as<char>() + k * field;
        }
        bpp_solve_opts o;
        bpp_solve_opts_default(&o);
        o.inner_prec = BPP_F32;
        o.use_graph = 0;
        std::vector<bpp_solve_stats> stt(6);
        const int rc = solve_batch(Gs, ks, clover, bv, xv, mg->prm.setup_tol, o, stt.data(), st);
        BPP_REQUIRE(rc == BPP_OK || rc == BPP_ERR_NOT_CONVERGED, rc, "near-null vector solve failed");
        BPP_CUDA(cudaMemcpyAsync(v64.p, w.p, 6 * field, cudaMemcpyDeviceToDevice, st));
    }
    LexBatches L;
    lex_batches(L, *G, P32, kappa, clover, 6, st);
    DevBuf v32(L.vec.vec_bytes, st);
    BPP_CUDA(cudaMemsetAsync(v32.p, 0, L.vec.vec_bytes, st));
    for (int k = 0; k < 6; ++k)
        full_to_eo(L.hop, k, 1, v64.as<char>() + k * field, 1, 0, v32.as<char>(), v32.as<char>() + L.half_off, 0, st);
    mg->P.alloc_persistent((size_t)72 * 2 * m.S * sizeof(float2));
    BPP_CUDA(cudaMemsetAsync(mg->P.p, 0, (size_t)72 * 2 * m.S * sizeof(float2), st));
    {
        ProfScope prof(PROF_OUTER, 0.0, st);
        k_mg_orth<<<dim3((unsigned)m.Vc, 2), m.bv, 0, st>>>(m, v32.as<char>(), (int64_t)(L.vec.vec_bytes / 6),
                                                             mg->P.as<float2>());
        count_launch();
        BPP_CHECK_LAUNCH();
    }
    mg->Dc.alloc_persistent((size_t)9 * 144 * m.Sc * sizeof(float2));
    BPP_CUDA(cudaMemsetAsync(mg->Dc.p, 0, (size_t)9 * 144 * m.Sc * sizeof(float2), st));
    {
        ProfScope prof(PROF_OUTER, 0.0, st);
        k_mg_coarse_build<<<dim3((unsigned)m.Vc, 9, 12), m.bv, 0, st>>>(m, mg->P.as<float2>(), L.hop.dev(),
                                                                        mg->Dc.as<float2>());
        count_launch();
        BPP_CHECK_LAUNCH();
    }
    BPP_CUDA(cudaStreamSynchronize(st));
    *out = mg.release();
}

void mg_destroy(bpp_mg_s* mg) {
    if (!mg) return;
    cudaDeviceSynchronize();
    delete mg;
}

// Transfer and coarse-operator access for tests and users (canonical-free:
// fields in the full-lattice layout are not exposed, so these take and
// return canonical complex64 full fields and coarse fields [nrhs][Vc][12]).
void mg_apply_op(const bpp_mg_s* mg, int op, const void* in, void* out, int nrhs, cudaStream_t st) {
    BPP_REQUIRE(mg && in && out, BPP_ERR_INVALID_ARG, "NULL argument");
    BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
    MGRun run(*mg, nrhs, st);
    const MGGeom& m = mg->geom;
    const size_t ffield = (size_t)mg->G->V * 12 * 8;   // canonical complex64 full field
    Buf f;
    f.zero(run.L.vec.vec_bytes, st);
    // canonical coarse fields: complex64 [nrhs][Vc][12]
    auto coarse_in = [&](char* dst) { half_to_int(run.cb, in, 0, dst, st, m.Vc * 12); };
    auto coarse_out = [&](const char* src) { int_to_half(run.cb, src, out, 0, st, m.Vc * 12); };
    if (op == BPP_MG_PROLONG) {
        coarse_in(run.cr.p());
        run.prolong(run.cr.p(), f.p(), false, st);
        for (int r = 0; r < nrhs; ++r)
            eo_to_full(run.L.hop, r, 1, f.p(), f.p() + run.L.half_off, static_cast<char*>(out) + r * ffield, 0, 0, 0, st);
    } else if (op == BPP_MG_RESTRICT) {
        for (int r = 0; r < nrhs; ++r)
            full_to_eo(run.L.hop, r, 1, static_cast<const char*>(in) + r * ffield, 0, 0, f.p(), f.p() + run.L.half_off, 0, st);
        run.restrict_(f.p(), run.cr.p(), st);
        coarse_out(run.cr.p());
    } else if (op == BPP_MG_COARSE) {
        coarse_in(run.cr.p());
        BPP_CUDA(cudaMemsetAsync(run.kc.p, 0, nrhs * sizeof(KScal), st));
        run.coarse_apply(run.cr.p(), run.cp.p(), st);
        coarse_out(run.cp.p());
    } else if (op == BPP_MG_VCYCLE) {
        Buf z;
        z.zero(run.L.vec.vec_bytes, st);
        for (int r = 0; r < nrhs; ++r)
            full_to_eo(run.L.hop, r, 1, static_cast<const char*>(in) + r * ffield, 0, 0, f.p(), f.p() + run.L.half_off, 0, st);
        run.vcycle(f.p(), z.p(), st);
        for (int r = 0; r < nrhs; ++r)
            eo_to_full(run.L.hop, r, 1, z.p(), z.p() + run.L.half_off, static_cast<char*>(out) + r * ffield, 0, 0, 0, st);
    } else {
        throw Error(BPP_ERR_INVALID_ARG, "unknown multigrid operation");
    }
    BPP_CUDA(cudaStreamSynchronize(st));
}

// D x = b through FP64 defect correction around flexible GCR(m) in FP32
// preconditioned by the V-cycle.
int mg_solve(const bpp_mg_s* mg, const void* b_canon, void* x_canon, double tol, int nrhs, const bpp_solve_opts& o,
             bpp_solve_stats* stats, cudaStream_t st) {
    BPP_REQUIRE(mg && b_canon && x_canon, BPP_ERR_INVALID_ARG, "NULL argument");
    BPP_REQUIRE(nrhs >= 1 && nrhs <= MAXSYS, BPP_ERR_INVALID_ARG, "nrhs must be 1..64");
    BPP_REQUIRE(tol > 0.0, BPP_ERR_INVALID_ARG, "tol must be positive");
    BPP_REQUIRE(o.max_inner > 0 && o.max_outer > 0, BPP_ERR_INVALID_ARG, "iteration caps must be positive");
    const auto t0 = std::chrono::steady_clock::now();
    double work0 = 0.0;
    for (int q = 0; q < NPREC; ++q) {
        double by = 0.0;
        work_read(q, nullptr, &by, 0);
        work0 += by;
    }
    const int n = nrhs;
    const bool clover = mg->csw != 0.0;
    const Gauge& G = *mg->G;
    LexBatches L64;
    lex_batches(L64, G, P64, mg->kappa, clover, n, st);
    MGRun run(*mg, n, st);
    const LexBatches& LP = run.L;
    Buf B, X, R;
    for (Buf* v : {&B, &X, &R}) v->zero(L64.vec.vec_bytes, st);
    const int m = mg->prm.gcr_restart;
    std::vector<Buf> Z(m), W(m);
    for (int q = 0; q < m; ++q) {
        Z[q].zero(LP.vec.vec_bytes, st);
        W[q].zero(LP.vec.vec_bytes, st);
    }
    Buf e, r, rhs;
    for (Buf* v : {&e, &r, &rhs}) v->zero(LP.vec.vec_bytes, st);
    RedBuf rb;
    DevBuf d64(n * sizeof(KScal), st), dgcr(n * sizeof(KScal), st);
    BPP_CUDA(cudaMemsetAsync(d64.p, 0, n * sizeof(KScal), st));
    BPP_CUDA(cudaMemsetAsync(dgcr.p, 0, n * sizeof(KScal), st));
    KScal* sc64 = d64.as<KScal>();
    KScal* scg = dgcr.as<KScal>();
    std::vector<KScal> h64(n);
    const size_t field = (size_t)G.V * 12 * 16;
    for (int q = 0; q < n; ++q)
        full_to_eo(L64.hop, q, 1, static_cast<const char*>(b_canon) + q * field, 1, 0, B.p(), B.p() + L64.half_off,
                   o.dagger ? 1 : 0, st);
    std::vector<double> bnorm2(n);
    {
        BlasVecs v;
        v.x = B.p();
        blas(L64.vec, B_NORM2, v, sc64, rb, st);
        BPP_CUDA(cudaMemcpyAsync(h64.data(), d64.p, n * sizeof(KScal), cudaMemcpyDeviceToHost, st));
        BPP_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < n; ++q) bnorm2[q] = h64[q].bb;
    }
    for (int q = 0; q < n; ++q) BPP_REQUIRE(std::isfinite(bnorm2[q]), BPP_ERR_NONFINITE, "non-finite right-hand side");
    auto defect = [&]() {
        lex_apply(L64, clover, 0, X.p(), R.p(), st);
        outer_residual(L64.vec, B.p(), R.p(), sc64, rb, st);
        BPP_CUDA(cudaMemcpyAsync(h64.data(), d64.p, n * sizeof(KScal), cudaMemcpyDeviceToHost, st));
        BPP_CUDA(cudaStreamSynchronize(st));
    };
    std::vector<int> outer(n, 0), inner_it(n, 0), conv(n, 0), status(n, BPP_OK);
    std::vector<double> true_res(n, 0.0);
    const std::vector<double2> zero(n, make_double2(0.0, 0.0)), one(n, make_double2(1.0, 0.0));
    auto dot = [&](const char* a, const char* bb) {   // <a, b> per system
        BlasVecs v;
        v.rhat = const_cast<char*>(a);
        v.v = const_cast<char*>(bb);
        const auto& t = run.sums(LP.vec, B_ALPHA, v, scg, rb, st);
        std::vector<double2> out(n);
        for (int q = 0; q < n; ++q) out[q] = make_double2(t[4 * q], t[4 * q + 1]);
        return out;
    };
    auto norm2 = [&](const char* a) {
        BlasVecs v;
        v.x = const_cast<char*>(a);
        const auto& t = run.sums(LP.vec, B_NORM2, v, scg, rb, st);
        std::vector<double> out(n);
        for (int q = 0; q < n; ++q) out[q] = t[4 * q];
        return out;
    };
    defect();
    for (;;) {
        bool any = false;
        std::vector<double> itol(n, 0.0);
        for (int q = 0; q < n; ++q) {
            if (status[q] != BPP_OK || conv[q]) { h64[q].scale = 0.0; continue; }
            const double rr = h64[q].rr;
            if (!std::isfinite(rr)) { status[q] = BPP_ERR_NONFINITE; h64[q].scale = 0.0; continue; }
            true_res[q] = bnorm2[q] > 0.0 ? std::sqrt(rr / bnorm2[q]) : 0.0;
            if (true_res[q] <= tol) { conv[q] = 1; h64[q].scale = 0.0; continue; }
            if (outer[q] >= o.max_outer) { h64[q].scale = 0.0; continue; }
            any = true;
            itol[q] = std::max(o.inner_tol > 0.0 ? o.inner_tol : 1e-6, 0.5 * tol * std::sqrt(bnorm2[q] / rr));
        }
        if (!any) break;
        BPP_CUDA(cudaMemcpyAsync(d64.p, h64.data(), n * sizeof(KScal), cudaMemcpyHostToDevice, st));
        outer_downcast(L64.vec, LP.vec, R.p(), rhs.p(), sc64, st);
        // flexible GCR on D e = rhs (|rhs| = 1 for active systems, 0 otherwise)
        run.axpy(LP.vec, e.p(), rhs.p(), zero, false, st);
        run.axpy(LP.vec, r.p(), rhs.p(), one, false, st);
        std::vector<double> rr0 = norm2(r.p());
        std::vector<int> its(n, 0);
        bool done_all = false;
        for (int it = 0; it < o.max_inner && !done_all;) {
            for (int j = 0; j < m && it < o.max_inner; ++j, ++it) {
                run.vcycle(r.p(), Z[j].p(), st);
                lex_apply(LP, clover, 0, Z[j].p(), W[j].p(), st);
                for (int i = 0; i < j; ++i) {
                    std::vector<double2> beta = dot(W[i].p(), W[j].p()), mb(n);
                    for (int q = 0; q < n; ++q) mb[q] = make_double2(-beta[q].x, -beta[q].y);
                    run.axpy(LP.vec, W[j].p(), W[i].p(), mb, true, st);
                    run.axpy(LP.vec, Z[j].p(), Z[i].p(), mb, true, st);
                }
                std::vector<double> nw = norm2(W[j].p());
                std::vector<double2> sc(n);
                for (int q = 0; q < n; ++q) sc[q] = make_double2(nw[q] > 0.0 ? 1.0 / std::sqrt(nw[q]) : 0.0, 0.0);
                run.axpy(LP.vec, W[j].p(), W[j].p(), sc, false, st);
                run.axpy(LP.vec, Z[j].p(), Z[j].p(), sc, false, st);
                std::vector<double2> al = dot(W[j].p(), r.p()), mal(n);
                for (int q = 0; q < n; ++q) mal[q] = make_double2(-al[q].x, -al[q].y);
                run.axpy(LP.vec, e.p(), Z[j].p(), al, true, st);
                run.axpy(LP.vec, r.p(), W[j].p(), mal, true, st);
                const std::vector<double> rn = norm2(r.p());
                done_all = true;
                for (int q = 0; q < n; ++q) {
                    const bool ok = !(rn[q] > itol[q] * itol[q] * rr0[q]);
                    if (!ok) its[q] += 1;
                    done_all = done_all && ok;
                }
                if (done_all) break;
            }
        }
        outer_accumulate(L64.vec, LP.vec, X.p(), e.p(), sc64, st);
        for (int q = 0; q < n; ++q)
            if (h64[q].scale != 0.0) {
                outer[q] += 1;
                inner_it[q] += its[q] + 1;
            }
        defect();
    }
    for (int q = 0; q < n; ++q) {
        if (status[q] == BPP_OK) {
            true_res[q] = bnorm2[q] > 0.0 ? std::sqrt(h64[q].rr / bnorm2[q]) : 0.0;
            if (!std::isfinite(true_res[q])) status[q] = BPP_ERR_NONFINITE;
            conv[q] = true_res[q] <= tol;
        }
    }
    for (int q = 0; q < n; ++q)
        eo_to_full(L64.hop, q, 1, X.p(), X.p() + L64.half_off, static_cast<char*>(x_canon) + q * field, 1, 0,
                   o.dagger ? 1 : 0, st);
    BPP_CUDA(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    double work1 = 0.0;
    for (int q = 0; q < NPREC; ++q) {
        double by = 0.0;
        work_read(q, nullptr, &by, 0);
        work1 += by;
    }
    int rc = BPP_OK;
    for (int q = 0; q < n; ++q) {
        if (status[q] == BPP_OK && !conv[q]) status[q] = BPP_ERR_NOT_CONVERGED;
        if (status[q] != BPP_OK && rc == BPP_OK) rc = status[q];
        if (stats) {
            stats[q].outer_iters = outer[q];
            stats[q].inner_iters = inner_it[q];
            stats[q].converged = conv[q];
            stats[q].status = status[q];
            stats[q].true_resid = true_res[q];
            stats[q].seconds = secs;
            stats[q].hop_bytes = work1 - work0;
            stats[q].hop_gbs = secs > 0.0 ? (work1 - work0) / secs / 1e9 : 0.0;
        }
    }
    return rc;
}

}  // namespace bpp
