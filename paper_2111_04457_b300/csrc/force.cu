// Link gradient of L = Re<eta, D^-1 b> for the Wilson hopping term of Eq. (1):
// with x = D^-1 b and lam = D^-dag eta, dL = -Re<lam, dD x> gives
//   G_mu(x) = kappa * bc * M_mu(x)^dag,
//   M_mu(x) = sum_spin [ x(x+mu) ((1 - gamma_mu) lam(x))^dag + ((1 + gamma_mu) lam(x+mu)) x(x)^dag ],
// colour outer products summed over spin.  The projected force is the
// traceless Hermitian P = (i kappa bc / 2)(U M - (U M)^dag) - trace/3, for which
// dL/deps = tr(T P) under U -> exp(i eps T) U.
#include "bpp_internal.h"
#include "gauge.h"
#include "kernels.h"
#include "solver.h"

namespace bpp {

typedef cx<double> zd;

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

struct ForceParams {
    Geom g;
    LinkView U[2][4];
    const double2* x;
    const double2* lam;
    double2* out;
    double kappa;
    int project;
};

__global__ void k_force(ForceParams fp) {
    const Geom g = fp.g;
    const int64_t V = 2 * (int64_t)g.Vh;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const int64_t s = t % V;
    int x[4];
    {
        int64_t r = s;
        x[0] = (int)(r % g.L[0]); r /= g.L[0];
        x[1] = (int)(r % g.L[1]); r /= g.L[1];
        x[2] = (int)(r % g.L[2]); x[3] = (int)(r / g.L[2]);
    }
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = (x[mu] + 1) % g.L[mu];
    const double sign = (x[mu] == g.L[mu] - 1) ? (double)g.bc[mu] : 1.0;
    const int64_t sy = y[0] + (int64_t)g.L[0] * (y[1] + (int64_t)g.L[1] * (y[2] + (int64_t)g.L[2] * y[3]));
    zd xs[12], xy[12], ls[12], ly[12], w[12], v[12];
    for (int k = 0; k < 12; ++k) {
        double2 a = fp.x[s * 12 + k], b = fp.x[sy * 12 + k], c = fp.lam[s * 12 + k], d = fp.lam[sy * 12 + k];
        xs[k] = mkc(a.x, a.y); xy[k] = mkc(b.x, b.y); ls[k] = mkc(c.x, c.y); ly[k] = mkc(d.x, d.y);
    }
    proj_full<-1>(mu, ls, w);   // (1 - gamma) lam(x)
    proj_full<+1>(mu, ly, v);   // (1 + gamma) lam(x+mu)
    zd M[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            zd acc = mkc(0.0, 0.0);
            for (int sp = 0; sp < 4; ++sp) {
                cfma(acc, xy[3 * sp + a], mkc(w[3 * sp + b].r, -w[3 * sp + b].i));
                cfma(acc, v[3 * sp + a], mkc(xs[3 * sp + b].r, -xs[3 * sp + b].i));
            }
            M[3 * a + b] = acc;
        }
    const double ks = fp.kappa * sign;
    double2* o = fp.out + ((int64_t)mu * V + s) * 9;
    if (!fp.project) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) o[3 * a + b] = make_double2(ks * M[3 * b + a].r, -ks * M[3 * b + a].i);
        return;
    }
    // Y = U M with U = U_mu(x)
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const double2* up = static_cast<const double2*>(fp.U[par][mu].data);
    zd U[9], Y[9];
    for (int k = 0; k < 9; ++k) {
        double2 q = up[k * fp.U[par][mu].stride + (s >> 1)];
        U[k] = mkc(q.x, q.y);
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            zd acc = mkc(0.0, 0.0);
            for (int k = 0; k < 3; ++k) cfma(acc, U[3 * a + k], M[3 * k + b]);
            Y[3 * a + b] = acc;
        }
    // P = (i ks / 2)(Y - Y^dag) - tr/3
    zd P[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const zd d = mkc(Y[3 * a + b].r - Y[3 * b + a].r, Y[3 * a + b].i + Y[3 * b + a].i);
            P[3 * a + b] = (0.5 * ks) * ix(d);
        }
    const double tr = (P[0].r + P[4].r + P[8].r) / 3.0;
    P[0].r -= tr; P[4].r -= tr; P[8].r -= tr;
    for (int k = 0; k < 9; ++k) o[k] = make_double2(P[k].r, P[k].i);
}

void force(const Gauge& G, const void* x, const void* lam, double kappa, void* dU, int project, cudaStream_t st) {
    ForceParams fp;
    fp.g = G.g;
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < 4; ++m) fp.U[p][m] = link_view(G, P64, p, m);
    fp.x = static_cast<const double2*>(x);
    fp.lam = static_cast<const double2*>(lam);
    fp.out = static_cast<double2*>(dU);
    fp.kappa = kappa;
    fp.project = project;
    const int64_t n = 4 * G.V;
    const int B = 128;
    k_force<<<(unsigned)((n + B - 1) / B), B, 0, st>>>(fp);
    count_launch();
    BPP_CHECK_LAUNCH();
}

}  // namespace bpp
