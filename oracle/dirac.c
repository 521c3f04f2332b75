/*
 * FP64 CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct restatement of the Wilson / Wilson-clover
 * fermion matrix of Eq. (1) of "General purpose lattice QCD code set Bridge++
 * 2.0 for high performance computing" (Sec. 3), used only by the tests, by
 * __graft_entry__.smoke() and by the benchmark's CPU-baseline leg.  Nothing in
 * the CUDA library calls, links or includes this file, and this file shares no
 * code, tables or constants with it.
 *
 *   D_{x,y} = [1 + F(x)] delta_{x,y}
 *             - kappa sum_mu [ (1 - gamma_mu) U_mu(x)      delta_{x+mu,y}
 *                            + (1 + gamma_mu) U_mu^dag(x-mu) delta_{x-mu,y} ]
 *
 * No half-spinor trick, no even-odd tables: every hop applies the full 4x4
 * spin matrix (1 -/+ gamma_mu), passed in by the caller, and the 3x3 link.
 * Neighbours come from modular arithmetic; a hop across the boundary in
 * direction mu picks up bc[mu] (+1 periodic, -1 antiperiodic).  When L_mu = 2
 * the forward and backward neighbours are the same site and both terms add,
 * as the sum in Eq. (1) says.
 *
 * Layouts (complex128): site s = x1 + L1*(x2 + L2*(x3 + L3*x4));
 *   U[((mu*V + s)*3 + a)*3 + b], psi[(s*4 + spin)*3 + colour],
 *   F[(s*12 + i)*12 + j] with i = spin*3 + colour, gamma[(mu*4 + s)*4 + t].
 */
#include <complex.h>
#include <stddef.h>
#include <stdint.h>

typedef double complex cplx;

static void site_coords(const int L[4], int64_t s, int x[4])
{
    x[0] = (int)(s % L[0]); s /= L[0];
    x[1] = (int)(s % L[1]); s /= L[1];
    x[2] = (int)(s % L[2]); s /= L[2];
    x[3] = (int)s;
}

static int64_t site_index(const int L[4], const int x[4])
{
    return x[0] + (int64_t)L[0] * (x[1] + (int64_t)L[1] * (x[2] + (int64_t)L[2] * x[3]));
}

/* neighbour of x one step along mu in direction dir (+1 / -1) */
static int64_t neighbour(const int L[4], const int x[4], int mu, int dir)
{
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = (x[mu] + dir + L[mu]) % L[mu];
    return site_index(L, y);
}

/* D psi (dagger = 0) or D^dagger psi (dagger = 1) at the listed sites.
 * D^dagger_{x,y} = conj(D_{y,x}) swaps (1 - gamma) and (1 + gamma); U enters the
 * same way because transposing the hop also swaps U_mu(x) and U_mu^dag(x-mu).
 * sites == NULL means all V sites, out then has V entries; otherwise out[k]
 * holds the result at sites[k]. */
void oracle_dirac_apply(const int L[4], const int bc[4], const cplx *gamma,
                        const cplx *U, const cplx *F, double kappa, int dagger,
                        const cplx *psi, cplx *out, int64_t nsites, const int64_t *sites)
{
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    if (sites == NULL) nsites = V;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nsites; ++k) {
        const int64_t s = sites ? sites[k] : k;
        int x[4];
        site_coords(L, s, x);
        cplx acc[12];
        /* [1 + F(x)] psi(x) */
        for (int i = 0; i < 12; ++i) {
            acc[i] = psi[s * 12 + i];
            if (F)
                for (int j = 0; j < 12; ++j) acc[i] += F[(s * 12 + i) * 12 + j] * psi[s * 12 + j];
        }
        for (int mu = 0; mu < 4; ++mu) {
            const cplx *g = &gamma[mu * 16];
            /* forward: (1 - gamma_mu) U_mu(x) psi(x+mu)   [dagger: (1 + gamma_mu)] */
            {
                const int64_t y = neighbour(L, x, mu, +1);
                const double sign = (x[mu] == L[mu] - 1) ? (double)bc[mu] : 1.0;
                const cplx *u = &U[(mu * V + s) * 9];
                cplx chi[12];
                for (int sp = 0; sp < 4; ++sp)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = 0.0;
                        for (int b = 0; b < 3; ++b) t += u[a * 3 + b] * psi[y * 12 + sp * 3 + b];
                        chi[sp * 3 + a] = t;
                    }
                const double gs = dagger ? +1.0 : -1.0;
                for (int sp = 0; sp < 4; ++sp)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = chi[sp * 3 + a];
                        for (int tp = 0; tp < 4; ++tp) t += gs * g[sp * 4 + tp] * chi[tp * 3 + a];
                        acc[sp * 3 + a] -= kappa * sign * t;
                    }
            }
            /* backward: (1 + gamma_mu) U_mu^dag(x-mu) psi(x-mu)   [dagger: (1 - gamma_mu)] */
            {
                const int64_t y = neighbour(L, x, mu, -1);
                const double sign = (x[mu] == 0) ? (double)bc[mu] : 1.0;
                const cplx *u = &U[(mu * V + y) * 9];
                cplx chi[12];
                for (int sp = 0; sp < 4; ++sp)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = 0.0;
                        for (int b = 0; b < 3; ++b) t += conj(u[b * 3 + a]) * psi[y * 12 + sp * 3 + b];
                        chi[sp * 3 + a] = t;
                    }
                const double gs = dagger ? -1.0 : +1.0;
                for (int sp = 0; sp < 4; ++sp)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = chi[sp * 3 + a];
                        for (int tp = 0; tp < 4; ++tp) t += gs * g[sp * 4 + tp] * chi[tp * 3 + a];
                        acc[sp * 3 + a] -= kappa * sign * t;
                    }
            }
        }
        for (int i = 0; i < 12; ++i) out[k * 12 + i] = acc[i];
    }
}

static void m3_mul(const cplx *a, const cplx *b, cplx *c)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx t = 0.0;
            for (int k = 0; k < 3; ++k) t += a[i * 3 + k] * b[k * 3 + j];
            c[i * 3 + j] = t;
        }
}

static void m3_dag(const cplx *a, cplx *c)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c[i * 3 + j] = conj(a[j * 3 + i]);
}

/* product of four 3x3 matrices a*b*c*d */
static void m3_mul4(const cplx *a, const cplx *b, const cplx *c, const cplx *d, cplx *out)
{
    cplx t1[9], t2[9];
    m3_mul(a, b, t1);
    m3_mul(t1, c, t2);
    m3_mul(t2, d, out);
}

/* Clover leaf Q_{mu nu}(x): the four plaquettes in the mu-nu plane that touch x,
 * each traversed in the same orientation (mu first, then nu). */
void oracle_clover_leaf(const int L[4], const cplx *U, int mu, int nu, int64_t s, cplx *Q)
{
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    int x[4];
    site_coords(L, s, x);
    const int64_t xpm = neighbour(L, x, mu, +1);
    const int64_t xpn = neighbour(L, x, nu, +1);
    const int64_t xmm = neighbour(L, x, mu, -1);
    const int64_t xmn = neighbour(L, x, nu, -1);
    int y[4];
    site_coords(L, xmm, y);
    const int64_t xmm_pn = neighbour(L, y, nu, +1);
    const int64_t xmm_mn = neighbour(L, y, nu, -1);
    site_coords(L, xmn, y);
    const int64_t xmn_pm = neighbour(L, y, mu, +1);
#define LINK(d, site) (&U[((int64_t)(d) * V + (site)) * 9])
    cplx a[9], b[9], c[9], d[9], leaf[9];
    for (int i = 0; i < 9; ++i) Q[i] = 0.0;
    /* U_mu(x) U_nu(x+mu) U_mu^dag(x+nu) U_nu^dag(x) */
    m3_dag(LINK(mu, xpn), c);
    m3_dag(LINK(nu, s), d);
    m3_mul4(LINK(mu, s), LINK(nu, xpm), c, d, leaf);
    for (int i = 0; i < 9; ++i) Q[i] += leaf[i];
    /* U_nu(x) U_mu^dag(x+nu-mu) U_nu^dag(x-mu) U_mu(x-mu) */
    m3_dag(LINK(mu, xmm_pn), b);
    m3_dag(LINK(nu, xmm), c);
    m3_mul4(LINK(nu, s), b, c, LINK(mu, xmm), leaf);
    for (int i = 0; i < 9; ++i) Q[i] += leaf[i];
    /* U_mu^dag(x-mu) U_nu^dag(x-mu-nu) U_mu(x-mu-nu) U_nu(x-nu) */
    m3_dag(LINK(mu, xmm), a);
    m3_dag(LINK(nu, xmm_mn), b);
    m3_mul4(a, b, LINK(mu, xmm_mn), LINK(nu, xmn), leaf);
    for (int i = 0; i < 9; ++i) Q[i] += leaf[i];
    /* U_nu^dag(x-nu) U_mu(x-nu) U_nu(x-nu+mu) U_mu^dag(x) */
    m3_dag(LINK(nu, xmn), a);
    m3_dag(LINK(mu, s), d);
    m3_mul4(a, LINK(mu, xmn), LINK(nu, xmn_pm), d, leaf);
    for (int i = 0; i < 9; ++i) Q[i] += leaf[i];
#undef LINK
}

/* F(x) = i kappa c_SW sum_{mu<nu} sigma_{mu nu} (x) Fhat_{mu nu}(x), a 12x12
 * Hermitian matrix per site, with sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] and
 * Fhat = (Q - Q^dag)/8 from the clover leaf.  Links enter without boundary
 * signs.  Output F[(k*12 + i)*12 + j] for the k-th listed site (all sites
 * when sites == NULL). */
void oracle_clover_field_sites(const int L[4], const cplx *gamma, const cplx *U, double kappa,
                               double csw, cplx *F, int64_t nsites, const int64_t *sites)
{
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    if (sites == NULL) nsites = V;
    cplx sigma[6][16];
    int pmu[6], pnu[6];
    int np = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    cplx c = 0.0;
                    for (int r = 0; r < 4; ++r)
                        c += gamma[mu * 16 + s * 4 + r] * gamma[nu * 16 + r * 4 + t]
                           - gamma[nu * 16 + s * 4 + r] * gamma[mu * 16 + r * 4 + t];
                    sigma[np][s * 4 + t] = 0.5 * I * c;
                }
            pmu[np] = mu; pnu[np] = nu; ++np;
        }
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nsites; ++k) {
        const int64_t s = sites ? sites[k] : k;
        cplx *f = &F[k * 144];
        for (int i = 0; i < 144; ++i) f[i] = 0.0;
        for (int p = 0; p < 6; ++p) {
            cplx Q[9], Fh[9];
            oracle_clover_leaf(L, U, pmu[p], pnu[p], s, Q);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Fh[a * 3 + b] = (Q[a * 3 + b] - conj(Q[b * 3 + a])) / 8.0;
            for (int sp = 0; sp < 4; ++sp)
                for (int tp = 0; tp < 4; ++tp)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            f[(sp * 3 + a) * 12 + tp * 3 + b] += I * kappa * csw * sigma[p][sp * 4 + tp] * Fh[a * 3 + b];
        }
    }
}

/* F(x) at every site (F[s*144 + ...]). */
void oracle_clover_field(const int L[4], const cplx *gamma, const cplx *U,
                         double kappa, double csw, cplx *F)
{
    oracle_clover_field_sites(L, gamma, U, kappa, csw, F, 0, NULL);
}

/* Unconstrained link gradient of L = Re<eta, D^{-1} b> for the Wilson hopping
 * term (the clover term is not differentiated), given x = D^{-1} b and
 * lam = D^{-dag} eta:
 *   G_mu(x) = kappa * bc * M_mu(x)^dag,
 *   M_mu(x) = sum_spin [ x(x+mu) ((1 - gamma_mu) lam(x))^dag
 *                      + ((1 + gamma_mu) lam(x+mu)) x(x)^dag ],
 * colour outer products summed over spin; bc is the boundary sign of the link.
 * This follows from dL = -Re<lam, dD x> with dD read off Eq. (1).
 * Output G[((mu*V + s)*3 + a)*3 + b]. */
void oracle_link_gradient(const int L[4], const int bc[4], const cplx *gamma,
                          const cplx *x, const cplx *lam, double kappa, cplx *G)
{
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < V; ++s) {
        int xc[4];
        site_coords(L, s, xc);
        for (int mu = 0; mu < 4; ++mu) {
            const cplx *g = &gamma[mu * 16];
            const int64_t y = neighbour(L, xc, mu, +1);
            const double sign = (xc[mu] == L[mu] - 1) ? (double)bc[mu] : 1.0;
            cplx w[12], v[12];        /* w = (1 - gamma) lam(x), v = (1 + gamma) lam(x+mu) */
            for (int sp = 0; sp < 4; ++sp)
                for (int a = 0; a < 3; ++a) {
                    cplx tw = lam[s * 12 + sp * 3 + a], tv = lam[y * 12 + sp * 3 + a];
                    for (int tp = 0; tp < 4; ++tp) {
                        tw -= g[sp * 4 + tp] * lam[s * 12 + tp * 3 + a];
                        tv += g[sp * 4 + tp] * lam[y * 12 + tp * 3 + a];
                    }
                    w[sp * 3 + a] = tw;
                    v[sp * 3 + a] = tv;
                }
            cplx M[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    cplx t = 0.0;
                    for (int sp = 0; sp < 4; ++sp)
                        t += x[y * 12 + sp * 3 + a] * conj(w[sp * 3 + b])
                           + v[sp * 3 + a] * conj(x[s * 12 + sp * 3 + b]);
                    M[a * 3 + b] = t;
                }
            cplx *out = &G[((int64_t)mu * V + s) * 9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) out[a * 3 + b] = kappa * sign * conj(M[b * 3 + a]);
        }
    }
}

/* Clover-term part of the link gradient of L = Re<eta, D^{-1} b> (added to G).
 * With x = D^{-1} b, lam = D^{-dag} eta and F = i kappa c_SW sum_{mu<nu}
 * sigma_{mu nu} (Q - Q^dag)/8, dL = -Re sum_x lam^dag dF x gives
 *   dL = (kappa c_SW / 8) sum_x sum_{mu<nu} Im tr[dQ_{mu nu}(x) H_{mu nu}(x)],
 *   H = W + W^dag,  W = sum_{s,t} sigma_{mu nu}[s][t] x_t(x) lam_s(x)^dag.
 * For a leaf A1 A2 A3 A4 (each a link or its dagger) the link of A_k enters
 * through R_k = A_{k+1} .. A4 H A1 .. A_{k-1}: with dL = Re sum conj(G) dU,
 * G += (kappa c_SW / 8) (i R_k^dag) for an undaggered link and
 * G += (kappa c_SW / 8) (-i R_k) for a daggered one.  Serial scatter loops. */
static void m3_mul_to(const cplx *a, const cplx *b, cplx *c) { m3_mul(a, b, c); }

void oracle_clover_gradient(const int L[4], const cplx *gamma, const cplx *U, const cplx *x, const cplx *lam,
                            double kappa, double csw, cplx *G)
{
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    const double c = kappa * csw / 8.0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
            cplx sigma[16];
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    cplx v = 0.0;
                    for (int r = 0; r < 4; ++r)
                        v += gamma[mu * 16 + s * 4 + r] * gamma[nu * 16 + r * 4 + t]
                           - gamma[nu * 16 + s * 4 + r] * gamma[mu * 16 + r * 4 + t];
                    sigma[s * 4 + t] = 0.5 * I * v;
                }
            for (int64_t s0 = 0; s0 < V; ++s0) {
                /* W = sum_{s,t} sigma[s][t] x_t lam_s^dag,  H = W + W^dag */
                cplx W[9], H[9];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        cplx v = 0.0;
                        for (int s = 0; s < 4; ++s)
                            for (int t = 0; t < 4; ++t)
                                v += sigma[s * 4 + t] * x[s0 * 12 + t * 3 + a] * conj(lam[s0 * 12 + s * 3 + b]);
                        W[a * 3 + b] = v;
                    }
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) H[a * 3 + b] = W[a * 3 + b] + conj(W[b * 3 + a]);
                /* the four leaves of Q_{mu nu}(x): links (direction, site, daggered) */
                int xc[4], y[4];
                site_coords(L, s0, xc);
                const int64_t xpm = neighbour(L, xc, mu, +1), xpn = neighbour(L, xc, nu, +1);
                const int64_t xmm = neighbour(L, xc, mu, -1), xmn = neighbour(L, xc, nu, -1);
                site_coords(L, xmm, y);
                const int64_t xmm_pn = neighbour(L, y, nu, +1), xmm_mn = neighbour(L, y, nu, -1);
                site_coords(L, xmn, y);
                const int64_t xmn_pm = neighbour(L, y, mu, +1);
                const int dir[4][4] = {{mu, nu, mu, nu}, {nu, mu, nu, mu}, {mu, nu, mu, nu}, {nu, mu, nu, mu}};
                const int64_t site[4][4] = {{s0, xpm, xpn, s0}, {s0, xmm_pn, xmm, xmm},
                                            {xmm, xmm_mn, xmm_mn, xmn}, {xmn, xmn, xmn_pm, s0}};
                const int dag[4][4] = {{0, 0, 1, 1}, {0, 1, 1, 0}, {1, 1, 0, 0}, {1, 0, 0, 1}};
                for (int leaf = 0; leaf < 4; ++leaf) {
                    cplx A[4][9];
                    for (int k = 0; k < 4; ++k) {
                        const cplx *u = &U[((int64_t)dir[leaf][k] * V + site[leaf][k]) * 9];
                        if (dag[leaf][k]) m3_dag(u, A[k]);
                        else for (int e = 0; e < 9; ++e) A[k][e] = u[e];
                    }
                    for (int k = 0; k < 4; ++k) {
                        /* R = A_{k+1} .. A_4 H A_1 .. A_{k-1} */
                        cplx R[9], T[9];
                        for (int e = 0; e < 9; ++e) R[e] = (e % 4 == 0) ? 1.0 : 0.0;
                        for (int j = k + 1; j < 4; ++j) { m3_mul_to(R, A[j], T); for (int e = 0; e < 9; ++e) R[e] = T[e]; }
                        m3_mul_to(R, H, T);
                        for (int e = 0; e < 9; ++e) R[e] = T[e];
                        for (int j = 0; j < k; ++j) { m3_mul_to(R, A[j], T); for (int e = 0; e < 9; ++e) R[e] = T[e]; }
                        cplx *g = &G[((int64_t)dir[leaf][k] * V + site[leaf][k]) * 9];
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) {
                                if (dag[leaf][k]) g[a * 3 + b] += c * (-I) * R[a * 3 + b];
                                else g[a * 3 + b] += c * I * conj(R[b * 3 + a]);
                            }
                    }
                }
            }
        }
}
