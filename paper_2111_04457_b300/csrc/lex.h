// Full-lattice ("lexical") fields and operator (see lex.cu): a full field is
// one structure-of-arrays vector whose planes hold 2 * stride entries, the
// even sites in the first half and the odd sites in the second.
#pragma once

#include "gauge.h"
#include "kernels.h"

namespace bpp {

struct LexBatches {
    Batch hop;             // half views, real geometry, plane stride 2 * stride
    Batch vec;             // whole fields: 2 * stride sites
    size_t half_off = 0;   // byte offset of the odd half inside a field
};

// nrhs systems on gauge G in precision prec (P64 or P32).
void lex_batches(LexBatches& lb, const Gauge& G, int prec, double kappa, bool clover, int nrhs, cudaStream_t st);
// out = D in (dag = 0) or D^dag in (dag = 1) on full fields, every system
// (skipping systems whose done flag is set).
void lex_apply(const LexBatches& lb, bool clover, int dag, char* in, char* out, cudaStream_t st,
               const int* done = nullptr, int ds = 0);

}  // namespace bpp
