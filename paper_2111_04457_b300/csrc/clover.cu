// Clover term of Eq. (1): "F(x) is a 12x12 Hermitian matrix made of the link
// variables" (Sec. 3).  Built once per gauge field:
//
//   F = i kappa c_SW sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu},  Fhat = (Q - Q^dag)/8,
//
// Q_{mu nu}(x) the sum of the four plaquettes around x in the mu-nu plane, all
// with the same orientation.  In the chiral basis sigma_{mu nu} is block
// diagonal, and with X1 = -(F23 +- F14), X2 = F13 -+ F24, X3 = -(F12 +- F34)
// (upper sign: spins 0,1; lower sign: spins 2,3; Fmn = Fhat for directions
// m,n = 1..4) each 6x6 block is
//
//   kappa c_SW [[ i X3,  i X1 + X2 ], [ i X1 - X2, -i X3 ]]   (2x2 in spin, 3x3 in colour).
//
// A = 1 + F and A^-1 (Gauss-Jordan with partial pivoting, FP64, per block) are
// stored packed in all three precisions.
#include "bpp_internal.h"
#include "clover_dev.h"
#include "gauge.h"
#include "kernels.h"

namespace bpp {

typedef cx<double> zd;

__device__ __forceinline__ void load_u(const Gauge* G, LinkView v[2][4], const Geom& g, int y0, int y1, int y2, int y3,
                                       int mu, zd u[9]) {
    // wrap coordinates
    y0 = (y0 + g.L[0]) % g.L[0];
    y1 = (y1 + g.L[1]) % g.L[1];
    y2 = (y2 + g.L[2]) % g.L[2];
    y3 = (y3 + g.L[3]) % g.L[3];
    const int par = (y0 + y1 + y2 + y3) & 1;
    const int64_t lex = y0 + (int64_t)g.L[0] * (y1 + (int64_t)g.L[1] * (y2 + (int64_t)g.L[2] * y3));
    const double2* p = static_cast<const double2*>(v[par][mu].data);
    const int64_t i = lex >> 1;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 t = p[k * v[par][mu].stride + i];
        u[k] = mkc(t.x, t.y);
    }
}

// c = a' * b' with a' = a or a^dag, b' = b or b^dag
template <bool DA, bool DB>
__device__ __forceinline__ void m3mul(const zd a[9], const zd b[9], zd c[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            zd t = mkc(0.0, 0.0);
            for (int k = 0; k < 3; ++k) {
                const zd x = DA ? mkc(a[3 * k + i].r, -a[3 * k + i].i) : a[3 * i + k];
                const zd y = DB ? mkc(b[3 * j + k].r, -b[3 * j + k].i) : b[3 * k + j];
                cfma(t, x, y);
            }
            c[3 * i + j] = t;
        }
}

struct CloverBuildParams {
    Geom g;
    LinkView U[2][4];     // FP64 links
    double kc;            // kappa * c_SW
    void* out[NPREC];     // per storage format: A_e, A_o, Ainv_e, Ainv_o
    int64_t stride;
    size_t field_bytes[NPREC];
    int* bad;             // set when a block is singular or non-finite
};

__device__ void store_block(const CloverBuildParams& cp, int which, int parity, int64_t i, int blk, const double r[36]) {
    const int f = which * 2 + parity;
    {
        double2* p = reinterpret_cast<double2*>(static_cast<char*>(cp.out[P64]) + f * cp.field_bytes[P64]);
        for (int j = 0; j < 18; ++j) p[(blk * 18 + j) * cp.stride + i] = make_double2(r[2 * j], r[2 * j + 1]);
    }
    {
        float4* p = reinterpret_cast<float4*>(static_cast<char*>(cp.out[P32]) + f * cp.field_bytes[P32]);
        for (int j = 0; j < 9; ++j)
            p[(blk * 9 + j) * cp.stride + i] = make_float4((float)r[4 * j], (float)r[4 * j + 1], (float)r[4 * j + 2], (float)r[4 * j + 3]);
    }
    {
        __half* base = reinterpret_cast<__half*>(static_cast<char*>(cp.out[P16]) + f * cp.field_bytes[P16]);
        for (int k = 0; k < 36; ++k) {
            const int h = blk * 36 + k;
            base[((h >> 3) * cp.stride + i) * 8 + (h & 7)] = __double2half(r[k]);
        }
    }
    {
        float4* p = reinterpret_cast<float4*>(static_cast<char*>(cp.out[P64S]) + f * cp.field_bytes[P64S]);
        for (int j = 0; j < 18; ++j) {
            const df64 a(r[2 * j]), b(r[2 * j + 1]);
            p[(blk * 18 + j) * cp.stride + i] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
    }
}

// Gauss-Jordan inverse of a 6x6 complex matrix with partial pivoting.
__device__ bool inverse6(zd a[36], zd inv[36]) {
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) inv[6 * r + c] = mkc(r == c ? 1.0 : 0.0, 0.0);
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        double best = a[6 * c + c].r * a[6 * c + c].r + a[6 * c + c].i * a[6 * c + c].i;
        for (int r = c + 1; r < 6; ++r) {
            const double m = a[6 * r + c].r * a[6 * r + c].r + a[6 * r + c].i * a[6 * r + c].i;
            if (m > best) { best = m; piv = r; }
        }
        if (!(best > 1e-300) || !isfinite(best)) return false;
        if (piv != c)
            for (int k = 0; k < 6; ++k) {
                zd t = a[6 * c + k]; a[6 * c + k] = a[6 * piv + k]; a[6 * piv + k] = t;
                t = inv[6 * c + k]; inv[6 * c + k] = inv[6 * piv + k]; inv[6 * piv + k] = t;
            }
        const zd p = a[6 * c + c];
        const double den = 1.0 / (p.r * p.r + p.i * p.i);
        const zd pinv = mkc(p.r * den, -p.i * den);
        for (int k = 0; k < 6; ++k) { a[6 * c + k] = pinv * a[6 * c + k]; inv[6 * c + k] = pinv * inv[6 * c + k]; }
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            const zd f = a[6 * r + c];
            for (int k = 0; k < 6; ++k) {
                a[6 * r + k] = a[6 * r + k] - f * a[6 * c + k];
                inv[6 * r + k] = inv[6 * r + k] - f * inv[6 * c + k];
            }
        }
    }
    return true;
}

// Pack a Hermitian 6x6 (taking the Hermitian part) into 6 + 30 reals.
__device__ void pack6(const zd m[36], double r[36]) {
    for (int k = 0; k < 6; ++k) r[k] = m[7 * k].r;
    for (int row = 1; row < 6; ++row)
        for (int col = 0; col < row; ++col) {
            const int k = row * (row - 1) / 2 + col;
            r[6 + 2 * k] = 0.5 * (m[6 * row + col].r + m[6 * col + row].r);
            r[7 + 2 * k] = 0.5 * (m[6 * row + col].i - m[6 * col + row].i);
        }
}

__global__ void k_clover_build(CloverBuildParams cp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const Geom g = cp.g;
    if (t >= 2 * (int64_t)g.Vh) return;
    const int parity = (int)(t / g.Vh);
    const int i = (int)(t % g.Vh);
    int x[4];
    eo_coords(g, i, parity, x);
    LinkView U[2][4];
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < 4; ++m) U[p][m] = cp.U[p][m];

    zd Fh[6][9];   // planes (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
    int pl = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++pl) {
            int e[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
            e[0][mu] = 1;
            e[1][nu] = 1;
#define AT(a, b) x[0] + (a) * e[0][0] + (b) * e[1][0], x[1] + (a) * e[0][1] + (b) * e[1][1], \
                 x[2] + (a) * e[0][2] + (b) * e[1][2], x[3] + (a) * e[0][3] + (b) * e[1][3]
            zd u1[9], u2[9], u3[9], u4[9], t1[9], t2[9], leaf[9], Q[9];
            for (int k = 0; k < 9; ++k) Q[k] = mkc(0.0, 0.0);
            // U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
            load_u(nullptr, U, g, AT(0, 0), mu, u1); load_u(nullptr, U, g, AT(1, 0), nu, u2);
            load_u(nullptr, U, g, AT(0, 1), mu, u3); load_u(nullptr, U, g, AT(0, 0), nu, u4);
            m3mul<false, false>(u1, u2, t1); m3mul<false, true>(t1, u3, t2); m3mul<false, true>(t2, u4, leaf);
            for (int k = 0; k < 9; ++k) Q[k] = Q[k] + leaf[k];
            // U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
            load_u(nullptr, U, g, AT(0, 0), nu, u1); load_u(nullptr, U, g, AT(-1, 1), mu, u2);
            load_u(nullptr, U, g, AT(-1, 0), nu, u3); load_u(nullptr, U, g, AT(-1, 0), mu, u4);
            m3mul<false, true>(u1, u2, t1); m3mul<false, true>(t1, u3, t2); m3mul<false, false>(t2, u4, leaf);
            for (int k = 0; k < 9; ++k) Q[k] = Q[k] + leaf[k];
            // U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
            load_u(nullptr, U, g, AT(-1, 0), mu, u1); load_u(nullptr, U, g, AT(-1, -1), nu, u2);
            load_u(nullptr, U, g, AT(-1, -1), mu, u3); load_u(nullptr, U, g, AT(0, -1), nu, u4);
            m3mul<true, true>(u1, u2, t1); m3mul<false, false>(t1, u3, t2); m3mul<false, false>(t2, u4, leaf);
            for (int k = 0; k < 9; ++k) Q[k] = Q[k] + leaf[k];
            // U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
            load_u(nullptr, U, g, AT(0, -1), nu, u1); load_u(nullptr, U, g, AT(0, -1), mu, u2);
            load_u(nullptr, U, g, AT(1, -1), nu, u3); load_u(nullptr, U, g, AT(0, 0), mu, u4);
            m3mul<true, false>(u1, u2, t1); m3mul<false, false>(t1, u3, t2); m3mul<false, true>(t2, u4, leaf);
            for (int k = 0; k < 9; ++k) Q[k] = Q[k] + leaf[k];
#undef AT
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    Fh[pl][3 * a + b] = mkc((Q[3 * a + b].r - Q[3 * b + a].r) * 0.125, (Q[3 * a + b].i + Q[3 * b + a].i) * 0.125);
        }
    // plane index: F12=0, F13=1, F14=2, F23=3, F24=4, F34=5
    for (int blk = 0; blk < 2; ++blk) {
        const double sg = blk == 0 ? 1.0 : -1.0;
        zd X1[9], X2[9], X3[9];
        for (int k = 0; k < 9; ++k) {
            X1[k] = -(Fh[3][k] + sg * Fh[2][k]);
            X2[k] = Fh[1][k] - sg * Fh[4][k];
            X3[k] = -(Fh[0][k] + sg * Fh[5][k]);
        }
        zd A[36];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const int k = 3 * a + b;
                A[6 * a + b] = cp.kc * ix(X3[k]);
                A[6 * a + 3 + b] = cp.kc * (ix(X1[k]) + X2[k]);
                A[6 * (3 + a) + b] = cp.kc * (ix(X1[k]) - X2[k]);
                A[6 * (3 + a) + 3 + b] = -(cp.kc * ix(X3[k]));
            }
        for (int k = 0; k < 6; ++k) A[7 * k].r += 1.0;
        double r[36];
        pack6(A, r);
        store_block(cp, 0, parity, i, blk, r);
        zd Ai[36];
        if (!inverse6(A, Ai)) atomicExch(cp.bad, 1);
        pack6(Ai, r);
        for (int k = 0; k < 36; ++k)
            if (!isfinite(r[k])) atomicExch(cp.bad, 1);
        store_block(cp, 1, parity, i, blk, r);
    }
}

void clover_build(Gauge& G, double kappa, double csw, cudaStream_t st) {
    for (int p = 0; p < NPREC; ++p) {
        if (!G.clover[p]) BPP_CUDA(cudaMalloc(&G.clover[p], 4 * clover_alloc_bytes(p, G.stride)));
    }
    CloverBuildParams cp;
    cp.g = G.g;
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < 4; ++m) cp.U[p][m] = link_view(G, P64, p, m);
    cp.kc = kappa * csw;
    cp.stride = G.stride;
    for (int p = 0; p < NPREC; ++p) {
        cp.out[p] = G.clover[p];
        cp.field_bytes[p] = clover_alloc_bytes(p, G.stride);
    }
    DevBuf bad(sizeof(int), st);
    BPP_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    cp.bad = bad.as<int>();
    const int B = 128;
    ProfScope prof(PROF_CLOVER, 0.0, st);
    k_clover_build<<<(unsigned)((2 * G.Vh + B - 1) / B), B, 0, st>>>(cp);
    count_launch();
    BPP_CHECK_LAUNCH();
    int h_bad = 0;
    BPP_CUDA(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BPP_CUDA(cudaStreamSynchronize(st));
    G.has_clover = true;
    G.clov_kappa = kappa;
    G.clov_csw = csw;
    if (h_bad) {
        G.has_clover = false;
        throw Error(BPP_ERR_NONFINITE, "clover build: a 6x6 block of 1 + F is singular or not finite");
    }
}

template <int P>
__global__ void k_clover_apply(const SysDesc* sys, int parity, int inverse, char* in, char* out) {
    using real = typename PT<P>::real;
    const SysDesc& d = sys[blockIdx.y];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.g.Vh) return;
    cx<real> v[12], w[12];
    Access<P>::load_spinor(sys_view<P>(in, d), i, v);
    clover_apply_site<P>(inverse ? d.Ainv[parity] : d.A[parity], i, v, w);
    Access<P>::store_spinor(sys_view<P>(out, d), i, w);
}

static double PTC_bytes(int prec) { return (prec == P64 || prec == P64S) ? 576.0 : prec == P32 ? 288.0 : 144.0; }

void clover_apply(const Batch& b, int parity, int inverse, char* in, char* out, cudaStream_t st) {
    for (auto& s : b.sys)
        BPP_REQUIRE((inverse ? s.Ainv[parity].data : s.A[parity].data) != nullptr, BPP_ERR_UNSUPPORTED,
                    "clover term not built (call bpp_clover_build)");
    const int B = 256;
    dim3 grid((unsigned)((b.Vh_max + B - 1) / B), b.nsys());
    ProfScope prof(PROF_CLOVER, b.sites() * (2.0 * spinor_bytes(b.prec) + PTC_bytes(b.prec)), st);
    if (b.prec == P64) k_clover_apply<P64><<<grid, B, 0, st>>>(b.dev(), parity, inverse, in, out);
    else if (b.prec == P32) k_clover_apply<P32><<<grid, B, 0, st>>>(b.dev(), parity, inverse, in, out);
    else if (b.prec == P16) k_clover_apply<P16><<<grid, B, 0, st>>>(b.dev(), parity, inverse, in, out);
    else k_clover_apply<P64S><<<grid, B, 0, st>>>(b.dev(), parity, inverse, in, out);
    count_launch();
    BPP_CHECK_LAUNCH();
}

}  // namespace bpp
