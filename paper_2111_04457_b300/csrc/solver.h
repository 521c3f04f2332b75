// Schur operator and the batched mixed-precision solve.
#pragma once

#include <vector>

#include "bpp_internal.h"
#include "gauge.h"

namespace bpp {

// out_e = Mhat in_e (dag: Mhat^dag) with the odd temporary tmp_o.
void schur(const Batch& b, bool clover, int dag, char* in_e, char* out_e, char* tmp_o, cudaStream_t st);

// Solves D[G_s] x_s = b_s (canonical complex128 full fields on the device) for
// every system s; returns BPP_OK or the first per-system error.
int solve_batch(const std::vector<const Gauge*>& G, const std::vector<double>& kappa, bool clover,
                const std::vector<const void*>& b_canon, const std::vector<void*>& x_canon, double tol,
                const bpp_solve_opts& o, bpp_solve_stats* stats, cudaStream_t st);

// Full-lattice (lexical) solve of A x = b, A = D, D^dag or D^dag D (mode
// bpp_lex_mode), FP64 defect correction around an FP64 or FP32 inner solve.
int solve_lex(const Gauge& G, double kappa, bool clover, const std::vector<const void*>& b_canon,
              const std::vector<void*>& x_canon, int mode, double tol, const bpp_solve_opts& o,
              bpp_solve_stats* stats, cudaStream_t st);

// Releases cached solver plans that use gauge G (all plans for G == nullptr).
void drop_plans(const Gauge* G);

// Link gradient / projected force (see bpp_force).
void force(const Gauge& G, const void* x, const void* lam, double kappa, double csw, int nrhs, void* dU, int project,
           cudaStream_t st);

}  // namespace bpp
