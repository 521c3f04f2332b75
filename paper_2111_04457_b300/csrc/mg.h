// Two-level aggregation multigrid (see mg.cu).
#pragma once

#include "bpp_internal.h"

struct bpp_mg_s;

namespace bpp {

void mg_create(bpp_gauge G, double kappa, double csw, const int bs[4], const void* vecs, int refine,
               const bpp_mg_params* prm, cudaStream_t st, bpp_mg_s** out);
void mg_destroy(bpp_mg_s* mg);
void mg_apply_op(const bpp_mg_s* mg, int op, const void* in, void* out, int nrhs, cudaStream_t st);
int mg_solve(const bpp_mg_s* mg, const void* b_canon, void* x_canon, double tol, int nrhs, const bpp_solve_opts& o,
             bpp_solve_stats* stats, cudaStream_t st);

}  // namespace bpp
