/*
 * bpp.h -- C ABI of the B300 Wilson / Wilson-clover fermion-matrix library.
 *
 * The library applies the fermion matrix of Eq. (1) of "General purpose lattice
 * QCD code set Bridge++ 2.0 for high performance computing" (arXiv:2111.04457,
 * Sec. 3):
 *
 *   D_{x,y} = [1 + F(x)] delta_{x,y}
 *             - kappa sum_mu [ (1 - gamma_mu) U_mu(x) delta_{x+mu,y}
 *                            + (1 + gamma_mu) U_mu^dag(x-mu) delta_{x-mu,y} ]
 *
 * and solves D x = b (the linear problem Sec. 2 names as the main bottleneck)
 * with the operator modes D / Ddag of Fig. 1 and float / double fields
 * (Sec. 2, the AField<double>/AField<float> pair).  Work runs as CUDA kernels
 * for sm_103a on one GPU; there is no CPU fallback.
 *
 * Conventions
 *   - Euclidean Hermitian gamma matrices in the chiral basis:
 *       gamma_k = [[0, i sigma_k], [-i sigma_k, 0]] (k = 1, 2, 3),
 *       gamma_4 = [[0, 1], [1, 0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(-1,-1,1,1).
 *   - Directions mu = 0..3 are x1..x4; the site index is
 *       s = x1 + L1*(x2 + L2*(x3 + L3*x4));  parity (x1+x2+x3+x4) mod 2, even = 0.
 *   - Boundary: a hop across the lattice boundary in direction mu is multiplied
 *     by bc[mu] (+1 periodic, -1 antiperiodic); links themselves are periodic.
 *   - Clover term: F = i kappa c_SW sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu},
 *     sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], Fhat = (Q - Q^dag)/8 from the
 *     four-plaquette clover leaf Q.
 *   - Canonical spinor layout: complex [nrhs][V][4][3] (spin, then colour),
 *     lexicographic sites.  Half-lattice ("even-odd") fields hold the Vh = V/2
 *     sites of one parity in lexicographic order.  Every extent must be even.
 *   - Canonical link layout: complex128 [4][V][3][3], row-major U_mu(x)[a][b].
 *   - The complex element type of a canonical field is complex128 for BPP_F64
 *     and BPP_F64DF and complex64 for BPP_F32 and BPP_F16 (FP16 is a storage
 *     format: the library converts at the boundary and computes in FP32).
 *
 * Errors: every function returns an int status, 0 = BPP_OK, < 0 an error code
 * below.  No C++ exception crosses the ABI.  bpp_last_error() copies the
 * message of the calling thread's last failure.  Calls are asynchronous on the
 * given stream unless documented otherwise; a NULL stream is the legacy default
 * stream.  The library never frees or keeps caller memory.
 */
#ifndef BPP_H_
#define BPP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* bpp_stream; /* the same type as cudaStream_t */

enum {
    BPP_OK = 0,
    BPP_ERR_INVALID_ARG = -1,   /* bad pointer, size, parity, precision or lattice */
    BPP_ERR_UNSUPPORTED = -2,   /* valid request the library does not implement */
    BPP_ERR_CUDA = -3,          /* a CUDA runtime call failed; see bpp_last_error */
    BPP_ERR_OOM = -4,           /* device allocation failed */
    BPP_ERR_NOT_CONVERGED = -5, /* solver hit max iterations or broke down; x is the best iterate */
    BPP_ERR_NONFINITE = -6,     /* NaN or Inf met in an input or a residual */
    BPP_ERR_TIMEOUT = -7        /* reserved: a bounded device-side wait ran out (the library's
                                   loops are graph conditionals with iteration caps and it has
                                   no device-side waits, so this is not returned today) */
};

/* BPP_F64DF: FP64 values (complex128 at the boundary) with double-float
 * arithmetic inside (each real held as an FP32 hi + lo pair, ~48-bit
 * significand), which runs on the FP32 pipe; accepted by bpp_dslash and
 * bpp_schur_apply. */
typedef enum { BPP_F64 = 0, BPP_F32 = 1, BPP_F16 = 2, BPP_F64DF = 3 } bpp_prec;
typedef enum { BPP_EVEN = 0, BPP_ODD = 1, BPP_FULL = 2 } bpp_parity;
typedef enum { BPP_BICGSTAB = 0, BPP_CGNR = 1 } bpp_solver;

/* Lattice extents L[mu] (every L[mu] even and >= 2: the even-odd decomposition
 * needs neighbours of opposite parity) and boundary signs bc[mu]
 * in {+1, -1}; the paper's workloads use bc = {1, 1, 1, -1}. */
typedef struct {
    int L[4];
    int bc[4];
} bpp_lattice;

/* Opaque gauge handle: owns device copies of the links in the internal
 * even-odd structure-of-arrays layout in all four storage formats, plus the clover
 * term and its inverse once bpp_clover_build() ran. */
typedef struct bpp_gauge_s* bpp_gauge;

/* Library version (major*10000 + minor*100 + patch). */
int bpp_version(void);

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to n bytes); returns the status code of that error (BPP_OK if none). */
int bpp_last_error(char* buf, size_t n);

/* Gauge field U_mu(x) of Eq. (1) (Sec. 2: "link variable U_mu(x) in SU(3)").
 * U_lex: complex128 [4][V][3][3] in device or host memory (detected); copied,
 * the caller keeps ownership.  Synchronises `stream` before returning.
 * When every link is SU(3) to 1e-10 (|U U^dag - 1| and |row3 -
 * conj(row1 x row2)|), the FP32 hopping kernels read only rows 1 and 2 and
 * rebuild row 3 (48 instead of 72 bytes per link); the environment variable
 * BPP_LINK_COMPRESSION=0, read when a solve plan or an operator call is set
 * up, keeps the 18-real links.
 * Errors: INVALID_ARG (NULL pointer, odd L[mu], L[mu] < 2, bc not +-1),
 * OOM, CUDA. */
int bpp_gauge_create(const bpp_lattice* lat, const void* U_lex, bpp_stream stream, bpp_gauge* out);

/* Frees the gauge handle and everything it owns (synchronises the device). */
int bpp_gauge_destroy(bpp_gauge g);

/* Builds the clover term F(x) of Eq. (1) ("a 12x12 Hermitian matrix made of
 * the link variables", Sec. 3) as two 6x6 Hermitian chiral blocks per site,
 * A = 1 + F and A^{-1} (per block, FP64 Gauss-Jordan), cached on the handle for
 * this (kappa, c_SW).  Must be called before any clover use (csw != 0).
 * Errors: INVALID_ARG, NONFINITE (a block is singular), OOM, CUDA. */
int bpp_clover_build(bpp_gauge g, double kappa, double csw, bpp_stream stream);

/* Hopping term of Eq. (1) between parities, or the full Wilson matrix.
 *   parity BPP_EVEN/BPP_ODD: out_p = -kappa H_{p,pbar} psi_pbar, where psi is
 *     the half field of the opposite parity and out the half field of parity p,
 *     both canonical [nrhs][Vh][4][3].  The clover term is not applied.
 *   parity BPP_FULL: out = D_W psi = psi - kappa H psi on the full lattice
 *     (F = 0), canonical [nrhs][V][4][3].
 * psi, out: device memory, caller-owned, of element type complex<prec>; out
 * must not alias psi.  The arithmetic is done in `prec` (BPP_F16: FP16 storage
 * of fields and links, FP32 arithmetic).
 * Errors: INVALID_ARG (NULL, nrhs < 1, bad parity/prec), OOM, CUDA. */
int bpp_dslash(bpp_gauge U, const void* psi, void* out, double kappa, int parity, int prec,
               int nrhs, bpp_stream stream);

/* bpp_dslash for the EVEN/ODD modes, for callers that cannot allocate device
 * memory (a host application whose own memory manager owns the device and
 * does not let libraries call cudaMalloc, or code that must not risk an
 * allocation failing or stalling partway through).  No counterpart in the
 * paper: it is the same hopping term as bpp_dslash, with the call's working
 * storage (the system table and the two internal half fields) taken from one
 * file-scope device array of 32 MiB, placed on a GPU when the first gauge field
 * is created there and held until the process exits, instead of being
 * allocated.  Arguments, layouts and results are
 * those of bpp_dslash with parity BPP_EVEN or BPP_ODD (BPP_FULL is rejected).
 * Needs 256-byte-rounded 64 system descriptors plus 2 * nrhs half fields of
 * (Vh rounded up to 64) * {192, 96, 52} bytes for F64/F32/F16; larger requests
 * return BPP_ERR_INVALID_ARG with the sizes in the message.  The current device
 * must be the gauge field's device.  The array's device address is looked up
 * (cudaGetSymbolAddress, which also places the array on the device under lazy
 * module loading) when a gauge field is created on that device, so this call
 * itself finds it in place.  The system table is written by a kernel from a
 * descriptor passed by value: no host buffer is read after the call returns.
 * All calls share the one array: calls that can overlap on the GPU (different
 * streams without ordering between them) race and give wrong results; calls
 * on one stream are ordered and safe.  Calls no
 * cudaMalloc, cudaFree or other allocating routine. */
int bpp_dslash_noalloc(bpp_gauge U, const void* psi, void* out, double kappa, int parity, int prec,
                       int nrhs, bpp_stream stream);

/* Clover term of Eq. (1) on one parity: out = (1 + F) in, or (1 + F)^{-1} in
 * when inverse != 0.  in/out: device, canonical half fields [nrhs][Vh][4][3]
 * of complex<prec>; parity BPP_EVEN or BPP_ODD.  Requires bpp_clover_build.
 * Errors: INVALID_ARG, UNSUPPORTED (no clover built), OOM, CUDA. */
int bpp_clover_apply(bpp_gauge U, const void* in, void* out, int parity, int inverse, int prec,
                     int nrhs, bpp_stream stream);

/* Even-odd preconditioned operator on the even half lattice,
 *   Mhat = A_ee - kappa^2 H_eo A_oo^{-1} H_oe   (A = 1 + F, A = 1 when csw = 0),
 * or its adjoint Mhat^dag = gamma5 Mhat gamma5 when dagger != 0.  csw != 0
 * requires bpp_clover_build with the same kappa and csw.  in/out: device,
 * canonical even half fields [nrhs][Vh][4][3] of complex<prec>.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
int bpp_schur_apply(bpp_gauge U, const void* in, void* out, double kappa, double csw, int dagger,
                    int prec, int nrhs, bpp_stream stream);

/* The full matrix D of Eq. (1) (clover included when csw != 0), or D^dag when
 * dagger != 0, in FP64 on canonical full fields complex128 [nrhs][V][4][3],
 * device memory.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
int bpp_dirac_apply(bpp_gauge U, const void* in, void* out, double kappa, double csw, int dagger,
                    int nrhs, bpp_stream stream);

/* Solver options.  The outer loop is FP64 defect correction (Sec. 2, Fig. 1:
 * the double/float mixed-precision propagator solver; Sec. 3: float plays the
 * main role in multi-precision solvers): r = bhat - Mhat x in FP64, an inner
 * Krylov solve of Mhat e = r/|r| in inner_prec to relative tolerance
 * inner_tol, x += |r| e.  inner_prec = BPP_F64 is the plain FP64 solve. */
typedef struct {
    int solver;       /* bpp_solver: BPP_BICGSTAB or BPP_CGNR on the Schur system */
    int inner_prec;   /* bpp_prec of the inner Krylov solve */
    double inner_tol; /* relative residual reduction per inner solve (ignored for F64);
                         <= 0 selects the default: 1e-6 for F32, 2e-3 for F16 */
    int max_inner;    /* iteration cap of one inner solve */
    int max_outer;    /* cap on defect-correction steps */
    int use_x0;       /* nonzero: x holds the initial guess on entry */
    int dagger;       /* nonzero: solve D^dag x = b (through gamma5-hermiticity) */
    int check_every;  /* inner iterations between host-side convergence checks (eager mode) */
    int use_graph;    /* 0: host-driven loops; 1: each inner solve is one CUDA graph
                         launch whose conditional while node repeats one Krylov iteration
                         until every system has converged; 2: the whole correction loop
                         (outer decisions by device control kernels, inner solves,
                         defect updates, true-residual checks) is one graph launch with
                         nested conditional nodes.  With 2 the first solve of a
                         configuration runs host-driven (autotuning) and captures the
                         graph; later solves replay it.  All modes compute identical
                         results. */
    int outer_arith;  /* 0: every outer-loop operator application in FP64 arithmetic;
                         1: the even-odd preparation and the intermediate defects
                         bhat - Mhat x in double-float arithmetic (FP64 values held as
                         FP32 hi + lo pairs, ~48-bit significands, on the FP32 pipe),
                         while the solution, its accumulation, all norms and the final
                         true residual stay FP64;
                         2: as 1, and the true-residual check and the iterate x in
                         double-float too: x_o = A_oo^-1 (b_o + kappa H_oe x_e) and
                         the even residual b_e - (A_ee x_e - kappa H_eo x_o) are
                         computed in double-float (the odd residual vanishes by
                         construction), and the returned x is the checked iterate
                         (scaled back by ||b|| to ~1e-14).  The check's rounding error
                         is of order 1e-14 ||x|| / ||b|| relative; it avoids the FP64
                         pipe, which runs at 1/74 of the FP32 rate on this GPU
                         (measured, bpp_fma_peak).  Ignored (FP64) when inner_prec is
                         F64; other values: INVALID_ARG */
} bpp_solve_opts;

/* Per right-hand side statistics of a solve. */
typedef struct {
    int outer_iters;    /* defect-correction steps */
    int inner_iters;    /* total inner Krylov iterations */
    int converged;      /* 1 if true_resid <= tol */
    int status;         /* BPP_OK or the per-RHS error code */
    double true_resid;  /* ||b - D x|| / ||b|| with the full D recomputed from x (FP64, or
                           double-float with outer_arith 2) */
    double seconds;     /* wall time of the whole call (same for every RHS); the first call
                           of a configuration includes the block-size autotuner's timing
                           launches and the CUDA-graph capture */
    double hop_bytes;   /* algorithmic bytes of every hopping-kernel launch of the call (all RHS) */
    double hop_gbs;     /* hop_bytes / seconds / 1e9: the dslash GB/s the call sustained */
} bpp_solve_stats;

/* Fills opts with defaults: BiCGStab, FP32 inner, inner_tol 0 (per precision),
 * max_inner 20000, max_outer 50, use_x0 0, dagger 0, check_every 4, use_graph 2,
 * outer_arith 2.
 * BiCGStab forms <rhat, v>, <t, s> and ||t||^2 inside the second hopping
 * kernel of each Schur application (per-warp partial sums in a fixed order);
 * the environment variable BPP_FUSED_DOTS=0, read when a solve plan is set
 * up, selects separate vector kernels instead.  Both are deterministic and
 * independent of batching; they group the sums differently. */
void bpp_solve_opts_default(bpp_solve_opts* opts);

/* Solves D x = b (or D^dag x = b) for nrhs right-hand sides sharing the gauge
 * field, to a true residual ||b - D x|| / ||b|| <= tol per RHS (D applied to
 * the returned x in FP64 or, with outer_arith 2, in double-float), through
 * the even-odd Schur complement: bhat_e = b_e - D_eo D_oo^{-1} b_o,
 * Mhat x_e = bhat_e, x_o = D_oo^{-1}(b_o - D_oe x_e).
 * b, x: complex128 [nrhs][V][4][3], in device memory or in host memory (then
 * copied in and out inside the call).  csw != 0 requires bpp_clover_build with
 * the same kappa and csw.  stats: NULL or an array of nrhs entries.
 * Synchronises `stream` (convergence decisions are taken on the host).
 * Errors: INVALID_ARG, UNSUPPORTED, NOT_CONVERGED (x holds the best iterate),
 * NONFINITE, OOM, CUDA. */
int bpp_solve(bpp_gauge U, const void* b, void* x, double kappa, double csw, double tol, int nrhs,
              const bpp_solve_opts* opts, bpp_solve_stats* stats, bpp_stream stream);

/* Operator modes of the lexical solve (Fig. 1: "mode is D, Ddag, DdagD"). */
typedef enum { BPP_LEX_D = 0, BPP_LEX_DDAG = 1, BPP_LEX_DDAGD = 2 } bpp_lex_mode;

/* Lexical propagator solve (Fig. 1, Fprop_Standard_lex with the double/float
 * mixed-precision solver of Sec. 2): A x = b on the full lattice, without
 * even-odd preconditioning, for nrhs right-hand sides sharing the gauge field:
 *   mode BPP_LEX_D:     A = D      (opts->solver BPP_BICGSTAB: BiCGStab on D;
 *                                   BPP_CGNR: CG on D^dag D x = D^dag b, the
 *                                   normal-equation propagator x = D^{-1} b)
 *   mode BPP_LEX_DDAG:  A = D^dag  (likewise)
 *   mode BPP_LEX_DDAGD: A = D^dag D (CG; opts->solver is ignored)
 * D is Eq. (1) with the clover term when csw != 0 (requires bpp_clover_build
 * with the same kappa and csw).  Outer loop: FP64 defect correction
 * r = b - A x with the full FP64 operator, inner solve of A e = r/|r| in
 * opts->inner_prec (BPP_F32, or BPP_F64 for the plain solve; BPP_F16 and
 * BPP_F64DF return BPP_ERR_UNSUPPORTED), x += |r| e, until
 * |b - A x| / |b| <= tol (FP64, recomputed from scratch), reported per RHS
 * as stats[r].true_resid.  opts->use_graph and opts->outer_arith are ignored
 * (host-driven loop, convergence read every check_every inner iterations).
 * b, x: complex128 [nrhs][V][4][3], device or host memory.  Synchronises
 * `stream`.  Errors: as bpp_solve. */
int bpp_solve_lex(bpp_gauge U, const void* b, void* x, double kappa, double csw, double tol, int nrhs, int mode,
                  const bpp_solve_opts* opts, bpp_solve_stats* stats, bpp_stream stream);

/* Batched solve over nlat independent lattices (each with its own gauge
 * handle, hopping parameter kappa[i] and one right-hand side), run together so
 * every kernel launch covers all lattices.  The paper has no counterpart (its
 * solver objects take one lattice per call); the batch is this library's
 * extension for many small independent problems on one GPU, each system
 * following the bpp_solve algorithm of Sec. 2 on its own.  csw != 0: Wilson-clover, each
 * gauge handle must hold its clover term built with (kappa[i], csw).
 * b[i], x[i]: device complex128 [V_i][4][3].  stats: NULL or nlat entries.
 * Errors: as bpp_solve. */
int bpp_solve_batch(int nlat, const bpp_gauge* U, const void* const* b, void* const* x,
                    const double* kappa, double csw, double tol, const bpp_solve_opts* opts,
                    bpp_solve_stats* stats, bpp_stream stream);

/* Link gradient of L = Re<eta, D^{-1} b> (the fermion force of the HMC use of
 * the solve, Sec. 2) for the matrix of Eq. (1), given x = D^{-1} b and
 * lam = D^{-dag} eta for nrhs right-hand sides (complex128 [nrhs][V][4][3],
 * device), summed over the right-hand sides.  From dL = -Re<lam, dD x>,
 * written dL = Re sum conj(G) dU:
 *   hopping term:  G_mu(x) = kappa * bc * M_mu(x)^dag,
 *     M_mu(x) = sum_spin [ x(x+mu) ((1 - gamma_mu) lam(x))^dag + ((1 + gamma_mu) lam(x+mu)) x(x)^dag ];
 *   clover term (csw != 0; the links of its four-plaquette leaves, no
 *   boundary signs):  dL = (kappa c_SW / 8) sum_x sum_{mu<nu} Im tr[dQ_{mu nu}(x) H_{mu nu}(x)],
 *     H = W + W^dag, W = sum_{s,t} sigma_{mu nu}[s][t] x_t(x) lam_s(x)^dag,
 *     so a link in leaf position k adds (kappa c_SW / 8) i R_k^dag (or
 *     -(kappa c_SW / 8) i R_k where the leaf holds its dagger), R_k the leaf
 *     product cycled to start after the link, with H inserted at the leaf's
 *     base site.
 * With project_su3 != 0 the output is instead the traceless Hermitian force
 *   P_mu(x) = (i/2)(U G^dag - G U^dag) - trace/3,  so that dL/deps = tr(T P)
 * for U_mu(x) -> exp(i eps T) U_mu(x).  The clover part needs no
 * bpp_clover_build (it uses the links only).
 * dU: complex128 [4][V][3][3], device, caller-owned, overwritten.
 * Errors: INVALID_ARG (NULL or host pointer, nrhs outside 1..64, non-finite
 * kappa or csw), OOM (the clover part's 864 B per site of scratch), CUDA. */
int bpp_force(bpp_gauge U, const void* x, const void* lam, double kappa, double csw, int nrhs, void* dU,
              int project_su3, bpp_stream stream);

/* ---- Domain decomposition (Sec. 2 and Sec. 3.1: sub-lattices per process,
 * boundary exchange, global sums), here with every sub-lattice on the current
 * GPU.  The lattice is cut in x4 into ndom slabs of L[3] / ndom time slices
 * (an even number, so each slab keeps the global even-odd split); each slab
 * holds only its own links.  A decomposed hop packs each slab's two faces of
 * the input field (the bottom face's (1 + SF gamma_4) projections and the top
 * face's U_4^dag (1 - SF gamma_4) projections, 12 reals per face site;
 * SF = -1 for D, +1 for D^dag), copies them into the neighbouring slabs' own
 * buffers (device-to-device copies standing in for the messages), and runs
 * the hopping kernel on every slab with the face terms from those buffers.
 * The face values carry exactly the arithmetic of the undecomposed kernel, so
 * the decomposed hopping term and Schur operator equal bpp_dslash and
 * bpp_schur_apply bit for bit when those read the 18-real links (always in
 * FP64 and FP16; in FP32 with BPP_LINK_COMPRESSION=0, see bpp_gauge_create).
 * Wilson fermions (no clover term). */
typedef struct bpp_dd_s* bpp_dd;

/* Combines per-slab sums: in holds nparts blocks of n doubles (slab order),
 * out receives their element-wise sum (n doubles); returns 0 on success.  The
 * hook where a multi-process run adds its cross-process sum. */
typedef int (*bpp_dd_reducer)(const double* in, double* out, int nparts, int n, void* ctx);

/* Cuts the lattice lat (links U_lex as in bpp_gauge_create, device or host)
 * into ndom slabs in x4.  Errors: INVALID_ARG (ndom outside 2..64, L[3] / ndom
 * not an even whole number, or the bpp_gauge_create conditions), OOM, CUDA. */
int bpp_dd_create(const bpp_lattice* lat, const void* U_lex, int ndom, bpp_stream stream, bpp_dd* out);
int bpp_dd_destroy(bpp_dd dd);

/* Registers the reducer of the decomposed solve's sums (NULL: the library sums
 * the slabs on the device, in slab order).  The library calls it from the
 * calling thread with host buffers, after synchronising the stream. */
int bpp_dd_set_reducer(bpp_dd dd, bpp_dd_reducer fn, void* ctx);

/* The hopping term of bpp_dslash (parity BPP_EVEN or BPP_ODD, prec BPP_F64,
 * BPP_F32 or BPP_F16, canonical global half fields [nrhs][Vh][4][3] in device
 * memory) through the decomposition.  Errors: INVALID_ARG, OOM, CUDA. */
int bpp_dd_dslash(bpp_dd dd, const void* psi, void* out, double kappa, int parity, int prec, int nrhs,
                  bpp_stream stream);

/* The Wilson Schur operator Mhat = 1 - kappa^2 H_eo H_oe (or Mhat^dag) of
 * bpp_schur_apply through the decomposition (two decomposed hops). */
int bpp_dd_schur_apply(bpp_dd dd, const void* in, void* out, double kappa, int dagger, int prec, int nrhs,
                       bpp_stream stream);

/* Solves D x = b (opts->dagger: D^dag x = b) for the Wilson matrix through the
 * decomposition: FP64 BiCGStab on the even-odd Schur system
 * (opts->inner_prec must be BPP_F64, opts->solver BPP_BICGSTAB), every inner
 * product reduced per slab and combined across slabs (see the reducer), then
 * x_o reconstructed and the full FP64 residual ||b - D x|| / ||b|| computed
 * the same way (stats[r].true_resid).  b, x: device complex128
 * [nrhs][V][4][3].  Synchronises `stream`.  Errors: as bpp_solve. */
int bpp_dd_solve(bpp_dd dd, const void* b, void* x, double kappa, double tol, int nrhs, const bpp_solve_opts* opts,
                 bpp_solve_stats* stats, bpp_stream stream);

/* ---- Multigrid (the multi-grid solver of Sec. 1 and Sec. 4), two levels,
 * for the full-lattice matrix D of Eq. (1) (Wilson or Wilson-clover):
 *   prolongator P: the lattice is cut into blocks of block[0..3] sites; on
 *     every block and chirality (spins 0,1 / spins 2,3) six near-null vectors
 *     restricted there are orthonormalised (Gram-Schmidt, fixed order), so a
 *     block carries 12 coarse degrees of freedom (chirality-major, then
 *     vector); restriction is P^dag;
 *   coarse operator D_c = P^dag D P: a nearest-neighbour stencil on the block
 *     lattice (a self term and one term per direction and sense, 12x12 each);
 *   V-cycle: nu_pre minimal-residual steps on D, restriction, BiCGStab on D_c
 *     to coarse_tol (at most coarse_maxiter iterations), prolongation, the
 *     residual recomputed, nu_post minimal-residual steps;
 *   solve: flexible GCR(gcr_restart) on D preconditioned by the V-cycle in
 *     FP32, inside FP64 defect correction until ||b - D x|| / ||b|| <= tol.
 * The preconditioner works in FP32. */
typedef struct bpp_mg_s* bpp_mg;

typedef struct {
    int nu_pre, nu_post;   /* minimal-residual smoothing steps before / after the coarse correction */
    double coarse_tol;     /* relative residual of the coarse BiCGStab */
    int coarse_maxiter;    /* iteration cap of the coarse BiCGStab */
    int gcr_restart;       /* GCR directions kept before a restart (1..64) */
    double setup_tol;      /* relative residual of the solves that improve the near-null vectors */
} bpp_mg_params;

/* Defaults: nu_pre 4, nu_post 4, coarse_tol 0.2, coarse_maxiter 15,
 * gcr_restart 12, setup_tol 0.05 (a cheap, loose coarse solve and more
 * smoothing: on 16^3x32 near the critical kappa the fastest of the settings
 * measured). */
void bpp_mg_params_default(bpp_mg_params* p);

/* Builds the prolongator and the coarse operator for D on gauge U (kappa,
 * csw; csw != 0 requires bpp_clover_build with the same kappa and csw).
 * vectors: six canonical complex128 full fields [6][V][4][3] (device or host),
 * the near-null vectors, or the starting vectors when refine > 0: each of the
 * refine passes replaces them by approximate solutions of D v' = v (mixed
 * precision, relative residual setup_tol), one inverse-iteration step.  The
 * library draws no random numbers.  block: extents dividing L, 32..256 sites
 * per block (a multiple of 32).  params: NULL for the defaults.  U must
 * outlive the handle.  Synchronises `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
int bpp_mg_create(bpp_gauge U, double kappa, double csw, const int block[4], const void* vectors, int refine,
                  const bpp_mg_params* params, bpp_stream stream, bpp_mg* out);
int bpp_mg_destroy(bpp_mg mg);

/* The multigrid operators on canonical complex64 fields (device memory), for
 * checking and for use as building blocks:
 *   BPP_MG_PROLONG:  out = P in,     in [nrhs][Vc][12], out [nrhs][V][4][3]
 *   BPP_MG_RESTRICT: out = P^dag in, in [nrhs][V][4][3], out [nrhs][Vc][12]
 *   BPP_MG_COARSE:   out = D_c in,   coarse fields
 *   BPP_MG_VCYCLE:   out = M in (the preconditioner), full fields
 * Coarse index: block b = b0 + Lc0 (b1 + Lc1 (b2 + Lc2 b3)), Lc = L / block;
 * component chirality * 6 + vector.  Synchronises `stream`. */
enum { BPP_MG_PROLONG = 0, BPP_MG_RESTRICT = 1, BPP_MG_COARSE = 2, BPP_MG_VCYCLE = 3 };
int bpp_mg_apply(bpp_mg mg, int op, const void* in, void* out, int nrhs, bpp_stream stream);

/* Solves D x = b (opts->dagger: D^dag x = b, through gamma5-hermiticity) with
 * the multigrid-preconditioned GCR under FP64 defect correction;
 * opts->inner_tol (<= 0: 1e-6) is the relative reduction per inner solve,
 * opts->max_inner caps the GCR iterations of one inner solve, opts->max_outer
 * the corrections.  b, x: device complex128 [nrhs][V][4][3].  stats as
 * bpp_solve (inner_iters counts preconditioned GCR iterations).
 * Synchronises `stream`.  Errors: as bpp_solve. */
int bpp_mg_solve(bpp_mg mg, const void* b, void* x, double tol, int nrhs, const bpp_solve_opts* opts,
                 bpp_solve_stats* stats, bpp_stream stream);

/* Number of kernels this library has launched since load (or since the last
 * reset when reset != 0); graph launches count each kernel node they run. */
int64_t bpp_launch_count(int reset);

/* Kernel timing: while enabled, every kernel launch of the library outside a
 * CUDA graph is bracketed by CUDA events on its stream and credited to its
 * kernel class. */
int bpp_prof_enable(int enable);
/* Reads (and with reset != 0 clears) the accumulated timings of kernel class
 * `prec`: number of launches, total milliseconds, total algorithmic bytes
 * (each operand and result counted once per launch).  Classes: 0..3 the
 * even-odd hopping kernels in BPP_F64 / BPP_F32 / BPP_F16 / BPP_F64DF (bytes:
 * 8 links + input + output spinor per site, + fused operands); 4 the Krylov
 * vector kernels (fused updates and reductions); 5 the outer defect-
 * correction vector kernels (residuals, down-conversion, accumulation);
 * 6 the boundary layout conversion; 7 the single-warp control kernels (no
 * bytes); 8 the clover apply (and build, no bytes); 9 the force kernel.
 * Synchronises the device.  Errors: INVALID_ARG (class out of range). */
int bpp_prof_read(int prec, int64_t* launches, double* ms, double* bytes, int reset);

/* Reads (and with reset != 0 clears) the work done by the even-odd hopping
 * kernels of precision prec since load: launches and algorithmic bytes (per
 * output site: 8 links + input and output spinor, + the xpay operand and
 * clover blocks of fused epilogues; right-hand sides that share a gauge field
 * count its links once per launch).  Graph-executed iterations are credited
 * per system for the iterations that system was active.  Does not synchronise. */
int bpp_work_read(int prec, int64_t* launches, double* bytes, int reset);

/* Releases cached device workspace (synchronises the device). */
int bpp_release_workspace(void);

/* Measures the throughput of the FMA pipe of prec (BPP_F64 or BPP_F32) with a
 * synthetic kernel (8 resp. 16 independent FMA chains per thread, 8 blocks of
 * 256 threads per SM, best of 5 launches of tens of ms) and stores it in
 * *tflops (an FMA counted as 2 flop).  The roofline denominator of the
 * ALU-bound hopping kernels (the FP64 hop on the FP64 pipe, the double-float
 * hop on the FP32 pipe), which the measurement of Sec. 3.3's kernels needs
 * beside the memory bandwidth.  Synchronises `stream`.  Errors: INVALID_ARG,
 * CUDA. */
int bpp_fma_peak(int prec, double* tflops, bpp_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* BPP_H_ */
