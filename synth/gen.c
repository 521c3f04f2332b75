/*
 * Seeded synthetic inputs: counter-based normal deviates and random SU(3) link
 * fields.  This file holds no arithmetic of the fermion matrix; it only makes
 * the inputs that both the FP64 oracle and the CUDA path consume.
 *
 * Random numbers
 *   splitmix64 (Steele, Lea, Flood 2014) used as a counter-based generator:
 *   the n-th 64-bit output for seed s is mix(s + (n+1) * 0x9E3779B97F4A7C15).
 *   A uniform in (0,1] is ((out >> 11) + 1) * 2^-53.  The j-th normal pair is
 *   Box-Muller on the uniforms with counters 2j and 2j+1.  Every value depends
 *   only on (seed, counter), so results do not depend on the thread count.
 *
 * Links (the "exp(i*eps*H), reunitarised" recipe)
 *   For link l = site*4 + mu (site in lexicographic order, x1 fastest) the nine
 *   complex entries of a Gaussian matrix A take normal pairs l*9 .. l*9+8.
 *   H = (A + A^dag)/2 - tr(.)/3, U = exp(i*eps*H) by a Taylor series with
 *   scaling and squaring in long double, then Gram-Schmidt on rows 1 and 2 and
 *   row 3 = conj(row1 x row2), so det U = 1.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t splitmix_at(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1ULL) * GOLDEN_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline double uniform_at(uint64_t seed, uint64_t n)
{
    return ((double)(splitmix_at(seed, n) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

static inline void normal_pair(uint64_t seed, uint64_t j, double *z0, double *z1)
{
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = uniform_at(seed, 2 * j);
    double u2 = uniform_at(seed, 2 * j + 1);
    double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(two_pi * u2);
    *z1 = r * sin(two_pi * u2);
}

/* out[k] = uniform (offset + k) in (0,1], k < n. */
void synth_uniforms(uint64_t seed, uint64_t offset, int64_t n, double *out)
{
    for (int64_t k = 0; k < n; ++k) out[k] = uniform_at(seed, offset + (uint64_t)k);
}

/* out[2k], out[2k+1] = normal pair (offset + k), k < n. */
void synth_normal_pairs(uint64_t seed, uint64_t offset, int64_t n, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k)
        normal_pair(seed, offset + (uint64_t)k, &out[2 * k], &out[2 * k + 1]);
}

typedef struct { long double re, im; } lcx;

static inline lcx lc_mul(lcx a, lcx b) { lcx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static inline lcx lc_add(lcx a, lcx b) { lcx r = {a.re + b.re, a.im + b.im}; return r; }

static void mat_mul(const lcx a[9], const lcx b[9], lcx c[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            lcx s = {0.0L, 0.0L};
            for (int k = 0; k < 3; ++k) s = lc_add(s, lc_mul(a[3 * i + k], b[3 * k + j]));
            c[3 * i + j] = s;
        }
}

/* exp(X) for a 3x3 matrix X by scaling and squaring with a 24-term Taylor series. */
static void mat_exp(const lcx x_in[9], lcx out[9])
{
    long double nrm = 0.0L;
    for (int i = 0; i < 9; ++i) nrm += x_in[i].re * x_in[i].re + x_in[i].im * x_in[i].im;
    nrm = sqrtl(nrm);
    int s = 0;
    while (nrm > 0.25L) { nrm *= 0.5L; ++s; }
    long double scale = ldexpl(1.0L, -s);
    lcx x[9];
    for (int i = 0; i < 9; ++i) { x[i].re = x_in[i].re * scale; x[i].im = x_in[i].im * scale; }
    /* Horner: e = 1 + x(1 + x/2(1 + x/3(...))) */
    lcx e[9], t[9];
    for (int i = 0; i < 9; ++i) { e[i].re = (i % 4 == 0) ? 1.0L : 0.0L; e[i].im = 0.0L; }
    for (int k = 24; k >= 1; --k) {
        mat_mul(x, e, t);
        for (int i = 0; i < 9; ++i) {
            e[i].re = t[i].re / (long double)k + ((i % 4 == 0) ? 1.0L : 0.0L);
            e[i].im = t[i].im / (long double)k;
        }
    }
    for (int k = 0; k < s; ++k) { mat_mul(e, e, t); memcpy(e, t, sizeof(t)); }
    memcpy(out, e, sizeof(e));
}

static void reunitarise(lcx u[9])
{
    long double n0 = 0.0L;
    for (int j = 0; j < 3; ++j) n0 += u[j].re * u[j].re + u[j].im * u[j].im;
    n0 = 1.0L / sqrtl(n0);
    for (int j = 0; j < 3; ++j) { u[j].re *= n0; u[j].im *= n0; }
    /* row1 -= <row0,row1> row0 */
    lcx d = {0.0L, 0.0L};
    for (int j = 0; j < 3; ++j) {
        d.re += u[j].re * u[3 + j].re + u[j].im * u[3 + j].im;
        d.im += u[j].re * u[3 + j].im - u[j].im * u[3 + j].re;
    }
    for (int j = 0; j < 3; ++j) {
        lcx p = lc_mul(d, u[j]);
        u[3 + j].re -= p.re; u[3 + j].im -= p.im;
    }
    long double n1 = 0.0L;
    for (int j = 0; j < 3; ++j) n1 += u[3 + j].re * u[3 + j].re + u[3 + j].im * u[3 + j].im;
    n1 = 1.0L / sqrtl(n1);
    for (int j = 0; j < 3; ++j) { u[3 + j].re *= n1; u[3 + j].im *= n1; }
    /* row2 = conj(row0 x row1) */
    for (int j = 0; j < 3; ++j) {
        int a = (j + 1) % 3, b = (j + 2) % 3;
        lcx c1 = lc_mul(u[a], u[3 + b]);
        lcx c2 = lc_mul(u[b], u[3 + a]);
        u[6 + j].re = c1.re - c2.re;
        u[6 + j].im = -(c1.im - c2.im);
    }
}

/* One SU(3) matrix exp(i*eps*H) from the normal pairs base .. base+8. */
static void su3_from_pairs(uint64_t seed, uint64_t base, double eps, double *out18)
{
    lcx a[9], h[9], x[9], u[9];
    for (int k = 0; k < 9; ++k) {
        double z0, z1;
        normal_pair(seed, base + (uint64_t)k, &z0, &z1);
        a[k].re = z0; a[k].im = z1;
    }
    /* H = (A + A^dag)/2 with the trace removed */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            h[3 * i + j].re = 0.5L * (a[3 * i + j].re + a[3 * j + i].re);
            h[3 * i + j].im = 0.5L * (a[3 * i + j].im - a[3 * j + i].im);
        }
    long double tr = (h[0].re + h[4].re + h[8].re) / 3.0L;
    h[0].re -= tr; h[4].re -= tr; h[8].re -= tr;
    /* X = i*eps*H */
    for (int i = 0; i < 9; ++i) { x[i].re = -(long double)eps * h[i].im; x[i].im = (long double)eps * h[i].re; }
    mat_exp(x, u);
    reunitarise(u);
    for (int i = 0; i < 9; ++i) { out18[2 * i] = (double)u[i].re; out18[2 * i + 1] = (double)u[i].im; }
}

/* Links in canonical order out[((mu*V + site)*9 + entry)*2 + reim]; the random
 * stream is consumed in the order site, then mu, then entry. */
void synth_su3_links(uint64_t seed, int64_t volume, double eps, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t site = 0; site < volume; ++site)
        for (int mu = 0; mu < 4; ++mu) {
            uint64_t l = (uint64_t)site * 4 + (uint64_t)mu;
            su3_from_pairs(seed, l * 9, eps, &out[((int64_t)mu * volume + site) * 18]);
        }
}

/* One SU(3) matrix per site (a gauge transformation g(x)), out[site*18 + ...]. */
void synth_su3_sites(uint64_t seed, int64_t volume, double eps, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t site = 0; site < volume; ++site)
        su3_from_pairs(seed, (uint64_t)site * 9, eps, &out[site * 18]);
}
