// Device building blocks of one hop of Eq. (1) in the chiral basis, shared by
// the even-odd hopping kernels and the multigrid coarse-operator build:
// spin projection to the two-spin half spinor, the SU(3) multiplication, and
// the reconstruction of the four-spinor.  gamma_mu = [[0, A_mu], [A_mu^dag, 0]]
// with A_k = i sigma_k, A_4 = 1, so (1 + S gamma_mu) psi = (h, S A_mu^dag h)
// with h = u + S A_mu l (u, l the upper and lower spin pairs).
#pragma once

#include "bpp_internal.h"

namespace bpp {

// h = u + S A_mu l for the four-spinor psi (u = spins 0,1; l = spins 2,3).
template <int MU, int S, class real>
__device__ __forceinline__ void project(const cx<real> psi[12], cx<real> h[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<real> u0 = psi[c], u1 = psi[3 + c], l0 = psi[6 + c], l1 = psi[9 + c];
        if (MU == 0) {          // A l = (i l1, i l0)
            h[c] = S > 0 ? u0 + ix(l1) : u0 - ix(l1);
            h[3 + c] = S > 0 ? u1 + ix(l0) : u1 - ix(l0);
        } else if (MU == 1) {   // A l = (l1, -l0)
            h[c] = S > 0 ? u0 + l1 : u0 - l1;
            h[3 + c] = S > 0 ? u1 - l0 : u1 + l0;
        } else if (MU == 2) {   // A l = (i l0, -i l1)
            h[c] = S > 0 ? u0 + ix(l0) : u0 - ix(l0);
            h[3 + c] = S > 0 ? u1 - ix(l1) : u1 + ix(l1);
        } else {                // A l = (l0, l1)
            h[c] = S > 0 ? u0 + l0 : u0 - l0;
            h[3 + c] = S > 0 ? u1 + l1 : u1 - l1;
        }
    }
}

// acc += (g, S A_mu^dag g) for the colour-multiplied half spinor g.
template <int MU, int S, class real>
__device__ __forceinline__ void reconstruct(cx<real> acc[12], const cx<real> g[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<real> g0 = g[c], g1 = g[3 + c];
        acc[c] = acc[c] + g0;
        acc[3 + c] = acc[3 + c] + g1;
        if (MU == 0) {          // A^dag g = (-i g1, -i g0)
            acc[6 + c] = S > 0 ? acc[6 + c] - ix(g1) : acc[6 + c] + ix(g1);
            acc[9 + c] = S > 0 ? acc[9 + c] - ix(g0) : acc[9 + c] + ix(g0);
        } else if (MU == 1) {   // A^dag g = (-g1, g0)
            acc[6 + c] = S > 0 ? acc[6 + c] - g1 : acc[6 + c] + g1;
            acc[9 + c] = S > 0 ? acc[9 + c] + g0 : acc[9 + c] - g0;
        } else if (MU == 2) {   // A^dag g = (-i g0, i g1)
            acc[6 + c] = S > 0 ? acc[6 + c] - ix(g0) : acc[6 + c] + ix(g0);
            acc[9 + c] = S > 0 ? acc[9 + c] + ix(g1) : acc[9 + c] - ix(g1);
        } else {                // A^dag g = (g0, g1)
            acc[6 + c] = S > 0 ? acc[6 + c] + g0 : acc[6 + c] - g0;
            acc[9 + c] = S > 0 ? acc[9 + c] + g1 : acc[9 + c] - g1;
        }
    }
}

// g = U h (BACK = false) or U^dag h (BACK = true) on both spins of h.
template <bool BACK, class real>
__device__ __forceinline__ void link_mul(const cx<real> U[9], const cx<real> h[6], cx<real> g[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<real> t = mkc<real>(0, 0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (BACK) cfmac(t, U[3 * b + a], h[3 * s + b]);
                else cfma(t, U[3 * a + b], h[3 * s + b]);
            }
            g[3 * s + a] = t;
        }
}

}  // namespace bpp
