// Domain decomposition in x4 (see dd.cu).
#pragma once

#include "bpp_internal.h"

struct bpp_dd_s;

namespace bpp {

void dd_create(const bpp_lattice* lat, const void* U_lex, int ndom, cudaStream_t st, bpp_dd_s** out);
void dd_destroy(bpp_dd_s* dd);
void dd_dslash(const bpp_dd_s* dd, const void* psi, void* out, double kappa, int parity, int prec, int nrhs,
               cudaStream_t st);
void dd_schur(const bpp_dd_s* dd, const void* in, void* out, double kappa, int dagger, int prec, int nrhs,
              cudaStream_t st);
int dd_solve(const bpp_dd_s* dd, const void* b_canon, void* x_canon, double kappa, double tol, int nrhs,
             const bpp_solve_opts& o, bpp_solve_stats* stats, cudaStream_t st);
void dd_set_reducer(bpp_dd_s* dd, bpp_dd_reducer fn, void* ctx);

}  // namespace bpp
