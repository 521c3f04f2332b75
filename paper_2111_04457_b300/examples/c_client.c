/*
 * A C client of libbpp (include/bpp.h): no Python, no PyTorch.  Builds a
 * random-ish gauge field on the host (here: the free field times a
 * site-dependent U(1) phase, which keeps every link unitary), solves D x = b
 * on an 8^4 lattice in mixed precision, and checks the true residual with
 * bpp_dirac_apply.  Prints one line "c_client ok <resid>" and returns 0 on
 * success.
 *
 *   gcc -O2 -I include -o c_client c_client.c -L<dir of libbpp.so> -lbpp -lcudart
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "bpp.h"

#define CHECK(x)                                                                 \
    do {                                                                         \
        int rc_ = (x);                                                           \
        if (rc_ != BPP_OK) {                                                     \
            char msg[512];                                                       \
            bpp_last_error(msg, sizeof msg);                                     \
            fprintf(stderr, "%s failed (%d): %s\n", #x, rc_, msg);               \
            return 1;                                                            \
        }                                                                        \
    } while (0)

int main(void)
{
    const bpp_lattice lat = {{8, 8, 8, 8}, {1, 1, 1, -1}};
    const long V = 8L * 8 * 8 * 8;
    const double kappa = 0.12;
    const size_t nlink = (size_t)4 * V * 9, nspin = (size_t)V * 12;
    double *U = calloc(2 * nlink, sizeof(double)), *b = malloc(2 * nspin * sizeof(double));
    if (!U || !b) return 1;
    for (int mu = 0; mu < 4; ++mu)
        for (long s = 0; s < V; ++s) {
            const double ph = 0.3 * sin(0.7 * (double)(s + 13 * mu));
            for (int a = 0; a < 3; ++a) {
                double* z = &U[2 * (((size_t)mu * V + s) * 9 + 4 * a)];
                z[0] = cos(ph + a);
                z[1] = sin(ph + a);
            }
        }
    for (size_t k = 0; k < 2 * nspin; ++k) b[k] = cos(0.37 * (double)k) + 0.1 * sin(1.3 * (double)k);

    bpp_gauge g;
    CHECK(bpp_gauge_create(&lat, U, NULL, &g));   /* host links: copied in */
    void *db, *dx, *dr;
    if (cudaMalloc(&db, 16 * nspin) || cudaMalloc(&dx, 16 * nspin) || cudaMalloc(&dr, 16 * nspin)) return 1;
    cudaMemcpy(db, b, 16 * nspin, cudaMemcpyHostToDevice);

    bpp_solve_opts o;
    bpp_solve_opts_default(&o);
    o.inner_prec = BPP_F16;
    bpp_solve_stats st;
    CHECK(bpp_solve(g, db, dx, kappa, 0.0, 1e-10, 1, &o, &st, NULL));
    CHECK(bpp_dirac_apply(g, dx, dr, kappa, 0.0, 0, 1, NULL));

    double* r = malloc(16 * nspin);
    cudaMemcpy(r, dr, 16 * nspin, cudaMemcpyDeviceToHost);
    double nr = 0.0, nb = 0.0;
    for (size_t k = 0; k < 2 * nspin; ++k) {
        nr += (b[k] - r[k]) * (b[k] - r[k]);
        nb += b[k] * b[k];
    }
    const double res = sqrt(nr / nb);
    CHECK(bpp_gauge_destroy(g));
    cudaFree(db);
    cudaFree(dx);
    cudaFree(dr);
    free(U);
    free(b);
    free(r);
    if (!(res <= 1e-10) || !st.converged) {
        fprintf(stderr, "residual %g converged %d\n", res, st.converged);
        return 1;
    }
    printf("c_client ok %.3e outer %d inner %d\n", res, st.outer_iters, st.inner_iters);
    return 0;
}
