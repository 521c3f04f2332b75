// Link gradient of L = Re<eta, D^-1 b> for the fermion matrix of Eq. (1),
// given x = D^-1 b and lam = D^-dag eta.  dL = -Re<lam, dD x> with dD read off
// Eq. (1), written as dL = Re sum conj(G) dU.
//
// Hopping term: G_mu(x) = kappa * bc * M_mu(x)^dag,
//   M_mu(x) = sum_spin [ x(x+mu) ((1 - gamma_mu) lam(x))^dag + ((1 + gamma_mu) lam(x+mu)) x(x)^dag ],
// colour outer products summed over spin.
//
// Clover term (F = i kappa c_SW sum_{mu<nu} sigma_{mu nu} (Q - Q^dag)/8):
//   dL = (kappa c_SW / 8) sum_x sum_{mu<nu} Im tr[ dQ_{mu nu}(x) H_{mu nu}(x) ],
//   H = W + W^dag,  W = sum_{s,t} sigma_{mu nu}[s][t] x_t(x) lam_s(x)^dag.
// A link that sits in a leaf A1 A2 A3 A4 of Q at position k enters through
// R_k = A_{k+1} .. A_4 H A_1 .. A_{k-1}: G += (kappa c_SW / 8) i R_k^dag when the
// leaf holds the link itself, G += -(kappa c_SW / 8) i R_k when it holds its
// dagger.  Each link lies in two plaquettes per plane, each a leaf of the
// clover at its four corners: 8 terms per plane, 24 per link, gathered per
// link (no atomics: the result does not depend on scheduling).
//
// Projected force: P = (i/2)(U G^dag - G U^dag) - trace/3, for which
// dL/deps = tr(T P) under U -> exp(i eps T) U.
#include "bpp_internal.h"
#include "gauge.h"
#include "kernels.h"
#include "solver.h"

namespace bpp {

typedef cx<double> zd;

__device__ __forceinline__ zd conjz(zd a) { return mkc(a.r, -a.i); }

// (1 + S gamma_mu) psi as a full four-spinor, chiral basis (see dslash.cu).
template <int S>
__device__ void proj_full(int mu, const zd psi[12], zd out[12]) {
    for (int c = 0; c < 3; ++c) {
        const zd u0 = psi[c], u1 = psi[3 + c], l0 = psi[6 + c], l1 = psi[9 + c];
        zd al0, al1, au0, au1;   // A l and A^dag u
        if (mu == 0) { al0 = ix(l1); al1 = ix(l0); au0 = -ix(u1); au1 = -ix(u0); }
        else if (mu == 1) { al0 = l1; al1 = -l0; au0 = -u1; au1 = u0; }
        else if (mu == 2) { al0 = ix(l0); al1 = -ix(l1); au0 = -ix(u0); au1 = ix(u1); }
        else { al0 = l0; al1 = l1; au0 = u0; au1 = u1; }
        out[c] = S > 0 ? u0 + al0 : u0 - al0;
        out[3 + c] = S > 0 ? u1 + al1 : u1 - al1;
        out[6 + c] = S > 0 ? l0 + au0 : l0 - au0;
        out[9 + c] = S > 0 ? l1 + au1 : l1 - au1;
    }
}

__device__ __forceinline__ void load12(const double2* p, zd v[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 t = __ldg(p + k);
        v[k] = mkc(t.x, t.y);
    }
}

__device__ __forceinline__ int64_t lex_of(const Geom& g, const int y[4]) {
    return y[0] + (int64_t)g.L[0] * (y[1] + (int64_t)g.L[1] * (y[2] + (int64_t)g.L[2] * y[3]));
}

// U_mu at the site x + da e_a + db e_b (periodic wrap), from the FP64
// internal link fields; dagger on request.
__device__ void link_at(const LinkView U[2][4], const Geom& g, const int x[4], int a, int da, int b, int db, int mu,
                        bool dag, zd u[9]) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[a] = (y[a] + da + g.L[a]) % g.L[a];
    y[b] = (y[b] + db + g.L[b]) % g.L[b];
    const int par = (y[0] + y[1] + y[2] + y[3]) & 1;
    const int64_t i = lex_of(g, y) >> 1;
    const double2* p = static_cast<const double2*>(U[par][mu].data);
    const int64_t st = U[par][mu].stride;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 t = __ldg(p + k * st + i);
        if (dag) u[3 * (k % 3) + k / 3] = mkc(t.x, -t.y);
        else u[k] = mkc(t.x, t.y);
    }
}

__device__ __forceinline__ void mm(const zd a[9], const zd b[9], zd c[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            zd t = mkc(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cfma(t, a[3 * i + k], b[3 * k + j]);
            c[3 * i + j] = t;
        }
}

// acc += a b
__device__ __forceinline__ void mm_acc(const zd a[9], const zd b[9], zd acc[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) cfma(acc[3 * i + j], a[3 * i + k], b[3 * k + j]);
}

// P = (i/2)(U G^dag - G U^dag) - tr/3 (traceless Hermitian), in place of G.
__device__ void project_su3(const zd U[9], zd G[9]) {
    zd Y[9];   // Y = U G^dag
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            zd t = mkc(0.0, 0.0);
            for (int k = 0; k < 3; ++k) cfma(t, U[3 * a + k], conjz(G[3 * b + k]));
            Y[3 * a + b] = t;
        }
    // G U^dag = (U G^dag)^dag = Y^dag
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const zd d = Y[3 * a + b] - conjz(Y[3 * b + a]);
            G[3 * a + b] = 0.5 * ix(d);
        }
    const double tr = (G[0].r + G[4].r + G[8].r) / 3.0;
    G[0].r -= tr; G[4].r -= tr; G[8].r -= tr;
    G[0].i = 0.0; G[4].i = 0.0; G[8].i = 0.0;
}

struct ForceParams {
    Geom g;
    LinkView U[2][4];
    const double2* x;      // [nrhs][V][4][3]
    const double2* lam;
    double2* out;          // [4][V][3][3]
    double kappa;
    int nrhs;
    int project;
};

// One thread per site x: the hopping-term gradient of its four links, summed
// over the right-hand sides.
__global__ void k_force(ForceParams fp) {
    const Geom g = fp.g;
    const int64_t V = 2 * (int64_t)g.Vh;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int x[4];
    {
        int64_t r = s;
        x[0] = (int)(r % g.L[0]); r /= g.L[0];
        x[1] = (int)(r % g.L[1]); r /= g.L[1];
        x[2] = (int)(r % g.L[2]); x[3] = (int)(r / g.L[2]);
    }
    for (int mu = 0; mu < 4; ++mu) {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] = (x[mu] + 1) % g.L[mu];
        const double sign = (x[mu] == g.L[mu] - 1) ? (double)g.bc[mu] : 1.0;
        const int64_t sy = lex_of(g, y);
        zd M[9];
        for (int k = 0; k < 9; ++k) M[k] = mkc(0.0, 0.0);
        for (int r = 0; r < fp.nrhs; ++r) {
            const int64_t off = (int64_t)r * V * 12;
            zd xs[12], xy[12], w[12], v[12];
            {
                zd ls[12];
                load12(fp.lam + off + s * 12, ls);
                proj_full<-1>(mu, ls, w);   // (1 - gamma) lam(x)
            }
            {
                zd ly[12];
                load12(fp.lam + off + sy * 12, ly);
                proj_full<+1>(mu, ly, v);   // (1 + gamma) lam(x+mu)
            }
            load12(fp.x + off + s * 12, xs);
            load12(fp.x + off + sy * 12, xy);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    for (int sp = 0; sp < 4; ++sp) {
                        cfma(M[3 * a + b], xy[3 * sp + a], conjz(w[3 * sp + b]));
                        cfma(M[3 * a + b], v[3 * sp + a], conjz(xs[3 * sp + b]));
                    }
        }
        const double ks = fp.kappa * sign;
        zd G[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[3 * a + b] = mkc(ks * M[3 * b + a].r, -ks * M[3 * b + a].i);
        if (fp.project) {
            zd U[9];
            link_at(fp.U, g, x, 0, 0, 1, 0, mu, false, U);
            project_su3(U, G);
        }
        double2* o = fp.out + ((int64_t)mu * V + s) * 9;
        for (int k = 0; k < 9; ++k) o[k] = make_double2(G[k].r, G[k].i);
    }
}

// ----------------------------------------------------------------------------- clover term
// Plane index of (a, b), a < b: (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).
__device__ __forceinline__ int plane_of(int a, int b) { return a == 0 ? b - 1 : a == 1 ? b + 1 : 5; }

// In the chiral basis F = kappa c_SW sum_p Fhat_p (x) T_p with T_p block
// diagonal (spins 0,1 and spins 2,3; sg = +1 / -1 for the two blocks); the
// 2x2 block of T_p is returned in t[2][2].  sigma_p = -i T_p.
__device__ void tblock(int pl, double sg, zd t[2][2]) {
    const zd z = mkc(0.0, 0.0), one = mkc(1.0, 0.0), im = mkc(0.0, 1.0);
    t[0][0] = t[0][1] = t[1][0] = t[1][1] = z;
    switch (pl) {
        case 0: t[0][0] = -im; t[1][1] = im; break;                                   // F12
        case 1: t[0][1] = one; t[1][0] = -one; break;                                 // F13
        case 2: t[0][1] = -(sg * im); t[1][0] = -(sg * im); break;                    // F14
        case 3: t[0][1] = -im; t[1][0] = -im; break;                                  // F23
        case 4: t[0][1] = -(sg * one); t[1][0] = sg * one; break;                     // F24
        default: t[0][0] = -(sg * im); t[1][1] = sg * im; break;                      // F34
    }
}

struct CloverForceParams {
    Geom g;
    LinkView U[2][4];
    const double2* x;      // [nrhs][V][4][3]
    const double2* lam;
    int nrhs;
    double2* H;            // [6 planes][9 entries][V]
    double2* G;            // [4][V][3][3], hopping-term gradient in, total out
    double c;              // kappa c_SW / 8
    int project;
};

// H_p(x) = W + W^dag, W = sum_{s,t} sigma_p[s][t] x_t lam_s^dag, summed over
// the right-hand sides, for the six planes.
__global__ void k_clover_hfield(CloverForceParams cp) {
    const int64_t V = 2 * (int64_t)cp.g.Vh;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    for (int pl = 0; pl < 6; ++pl) {
        zd W[9];
        for (int k = 0; k < 9; ++k) W[k] = mkc(0.0, 0.0);
        for (int r = 0; r < cp.nrhs; ++r) {
            const int64_t off = (int64_t)r * V * 12;
            zd xs[12], ls[12];
            load12(cp.x + off + s * 12, xs);
            load12(cp.lam + off + s * 12, ls);
            for (int blk = 0; blk < 2; ++blk) {
                zd t[2][2];
                tblock(pl, blk == 0 ? 1.0 : -1.0, t);
                for (int sl = 0; sl < 2; ++sl)
                    for (int tl = 0; tl < 2; ++tl) {
                        // sigma = -i T
                        const zd sg = mkc(t[sl][tl].i, -t[sl][tl].r);
                        if (sg.r == 0.0 && sg.i == 0.0) continue;
                        const int ss = 2 * blk + sl, tt = 2 * blk + tl;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) cfma(W[3 * a + b], sg, xs[3 * tt + a] * conjz(ls[3 * ss + b]));
                    }
            }
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const zd h = W[3 * a + b] + conjz(W[3 * b + a]);
                cp.H[((int64_t)pl * 9 + 3 * a + b) * V + s] = make_double2(h.r, h.i);
            }
    }
}

__device__ void h_at(const CloverForceParams& cp, const int x[4], int a, int da, int b, int db, int pl, zd h[9]) {
    const Geom& g = cp.g;
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[a] = (y[a] + da + g.L[a]) % g.L[a];
    y[b] = (y[b] + db + g.L[b]) % g.L[b];
    const int64_t V = 2 * (int64_t)g.Vh;
    const int64_t s = lex_of(g, y);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 t = __ldg(cp.H + ((int64_t)pl * 9 + k) * V + s);
        h[k] = mkc(t.x, t.y);
    }
}

// acc += F1 F2 F3 with H inserted at position `at` (0: before F1, 1: after F1,
// 2: after F2, 3: after F3), given the partial products F12 = F1 F2,
// F23 = F2 F3 and F123.
__device__ void staple_insert(const zd F1[9], const zd F3[9], const zd F12[9], const zd F23[9], const zd F123[9],
                              const zd H[9], int at, zd acc[9]) {
    zd t[9];
    if (at == 0) {
        mm_acc(H, F123, acc);
    } else if (at == 1) {
        mm(F1, H, t);
        mm_acc(t, F23, acc);
    } else if (at == 2) {
        mm(F12, H, t);
        mm_acc(t, F3, acc);
    } else {
        mm_acc(F123, H, acc);
    }
}

// One staple F1 F2 F3 of link U_mu(x) in the plane (a, b) and the four
// positions and sites of H along it; returns sum of the four products.
__device__ void staple_sum(const CloverForceParams& cp, const int x[4], int a, int b, int pl, const zd F1[9],
                           const zd F2[9], const zd F3[9], const int at[4], const int da[4], const int db[4], zd S[9]) {
    zd F12[9], F23[9], F123[9];
    mm(F1, F2, F12);
    mm(F2, F3, F23);
    mm(F12, F3, F123);
    for (int k = 0; k < 9; ++k) S[k] = mkc(0.0, 0.0);
    for (int q = 0; q < 4; ++q) {
        zd H[9];
        h_at(cp, x, a, da[q], b, db[q], pl, H);
        staple_insert(F1, F3, F12, F23, F123, H, at[q], S);
    }
}

// One thread per site x: adds the clover term's gradient to G_mu(x) for the
// four directions, then projects when asked.
__global__ void k_clover_force(CloverForceParams cp) {
    const Geom g = cp.g;
    const int64_t V = 2 * (int64_t)g.Vh;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int x[4];
    {
        int64_t r = s;
        x[0] = (int)(r % g.L[0]); r /= g.L[0];
        x[1] = (int)(r % g.L[1]); r /= g.L[1];
        x[2] = (int)(r % g.L[2]); x[3] = (int)(r / g.L[2]);
    }
    for (int mu = 0; mu < 4; ++mu) {
        zd A[9], B[9];   // A: sum of products entering as i R^dag, B: as -i R
        for (int k = 0; k < 9; ++k) A[k] = B[k] = mkc(0.0, 0.0);
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            const int a = mu < nu ? mu : nu, b = mu < nu ? nu : mu;
            const int pl = plane_of(a, b);
            zd F1[9], F2[9], F3[9], S[9];
            if (mu == a) {
                // U_b(x+a) U_a(x+b)^dag U_b(x)^dag, H at x+a, x+a+b, x+b, x: leaf
                // positions of the link itself
                link_at(cp.U, g, x, a, 1, b, 0, b, false, F1);
                link_at(cp.U, g, x, a, 0, b, 1, a, true, F2);
                link_at(cp.U, g, x, a, 0, b, 0, b, true, F3);
                {
                    const int at[4] = {0, 1, 2, 3}, da[4] = {1, 1, 0, 0}, db[4] = {0, 1, 1, 0};
                    staple_sum(cp, x, a, b, pl, F1, F2, F3, at, da, db, S);
                }
                for (int k = 0; k < 9; ++k) A[k] = A[k] + S[k];
                // U_b(x-b)^dag U_a(x-b) U_b(x+a-b), H at x, x-b, x+a-b, x+a: its dagger
                link_at(cp.U, g, x, a, 0, b, -1, b, true, F1);
                link_at(cp.U, g, x, a, 0, b, -1, a, false, F2);
                link_at(cp.U, g, x, a, 1, b, -1, b, false, F3);
                {
                    const int at[4] = {0, 1, 2, 3}, da[4] = {0, 0, 1, 1}, db[4] = {0, -1, -1, 0};
                    staple_sum(cp, x, a, b, pl, F1, F2, F3, at, da, db, S);
                }
                for (int k = 0; k < 9; ++k) B[k] = B[k] + S[k];
            } else {
                // U_a(x) U_b(x+a) U_a(x+b)^dag, H at x, x+a, x+a+b, x+b: its dagger
                link_at(cp.U, g, x, a, 0, b, 0, a, false, F1);
                link_at(cp.U, g, x, a, 1, b, 0, b, false, F2);
                link_at(cp.U, g, x, a, 0, b, 1, a, true, F3);
                {
                    const int at[4] = {0, 1, 2, 3}, da[4] = {0, 1, 1, 0}, db[4] = {0, 0, 1, 1};
                    staple_sum(cp, x, a, b, pl, F1, F2, F3, at, da, db, S);
                }
                for (int k = 0; k < 9; ++k) B[k] = B[k] + S[k];
                // U_a(x-a+b)^dag U_b(x-a)^dag U_a(x-a), H at x+b, x-a+b, x-a, x: the link itself
                link_at(cp.U, g, x, a, -1, b, 1, a, true, F1);
                link_at(cp.U, g, x, a, -1, b, 0, b, true, F2);
                link_at(cp.U, g, x, a, -1, b, 0, a, false, F3);
                {
                    const int at[4] = {0, 1, 2, 3}, da[4] = {0, -1, -1, 0}, db[4] = {1, 1, 0, 0};
                    staple_sum(cp, x, a, b, pl, F1, F2, F3, at, da, db, S);
                }
                for (int k = 0; k < 9; ++k) A[k] = A[k] + S[k];
            }
        }
        // G += c (i A^dag - i B)
        double2* o = cp.G + ((int64_t)mu * V + s) * 9;
        zd G[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const double2 t = o[3 * i + j];
                const zd d = conjz(A[3 * j + i]) - B[3 * i + j];
                G[3 * i + j] = mkc(t.x, t.y) + cp.c * ix(d);
            }
        if (cp.project) {
            zd U[9];
            link_at(cp.U, g, x, 0, 0, 1, 0, mu, false, U);
            project_su3(U, G);
        }
        for (int k = 0; k < 9; ++k) o[k] = make_double2(G[k].r, G[k].i);
    }
}

void force(const Gauge& G, const void* x, const void* lam, double kappa, double csw, int nrhs, void* dU, int project,
           cudaStream_t st) {
    const bool clover = csw != 0.0;
    ForceParams fp;
    fp.g = G.g;
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < 4; ++m) fp.U[p][m] = link_view(G, P64, p, m);
    fp.x = static_cast<const double2*>(x);
    fp.lam = static_cast<const double2*>(lam);
    fp.out = static_cast<double2*>(dU);
    fp.kappa = kappa;
    fp.nrhs = nrhs;
    fp.project = clover ? 0 : project;
    const int B = 128;
    const unsigned grid = (unsigned)((G.V + B - 1) / B);
    {
        ProfScope prof(PROF_FORCE, (double)G.V * (nrhs * 2 * 192.0 + 4 * 144.0 * (fp.project ? 2 : 1)), st);
        k_force<<<grid, B, 0, st>>>(fp);
        count_launch();
        BPP_CHECK_LAUNCH();
    }
    if (!clover) return;
    DevBuf hbuf((size_t)G.V * 6 * 9 * sizeof(double2), st);
    CloverForceParams cp;
    cp.g = G.g;
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < 4; ++m) cp.U[p][m] = link_view(G, P64, p, m);
    cp.x = fp.x;
    cp.lam = fp.lam;
    cp.nrhs = nrhs;
    cp.H = hbuf.as<double2>();
    cp.G = fp.out;
    cp.c = kappa * csw / 8.0;
    cp.project = project;
    {
        ProfScope prof(PROF_FORCE, (double)G.V * (nrhs * 2 * 192.0 + 6 * 144.0), st);
        k_clover_hfield<<<grid, B, 0, st>>>(cp);
        count_launch();
        BPP_CHECK_LAUNCH();
    }
    {
        ProfScope prof(PROF_FORCE, (double)G.V * (6 * 144.0 + 4 * 144.0 * 2 + 4 * 144.0 * (project ? 2 : 1)), st);
        k_clover_force<<<grid, B, 0, st>>>(cp);
        count_launch();
        BPP_CHECK_LAUNCH();
    }
}

}  // namespace bpp
