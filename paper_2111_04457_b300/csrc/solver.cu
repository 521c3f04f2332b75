// Even-odd preconditioned solve of D x = b with a mixed-precision defect
// correction (Sec. 2, Fig. 1: a double-precision outer solver around a
// single-precision inner solver; Sec. 3: single precision "plays a main role
// in multi-precision solver algorithms").
//
//   bhat_e = b_e - D_eo D_oo^-1 b_o = b_e + kappa H_eo A_oo^-1 b_o
//   Mhat   = A_ee - kappa^2 H_eo A_oo^-1 H_oe
//   outer (FP64): r = bhat - Mhat x; stop when ||r|| <= tol ||b||;
//                 e = Mhat^-1 (r/||r||) to inner_tol in the inner precision;
//                 x += ||r|| e
//   x_o = A_oo^-1 (b_o + kappa H_oe x_e)
//   true residual ||b - D x|| / ||b|| recomputed with the full FP64 D.
//
// The inner solver is BiCGStab (van der Vorst 1992) or CGNR (CG on
// Mhat^dag Mhat with Mhat^dag = gamma5 Mhat gamma5) on the Schur system, over a
// batch of systems (right-hand sides and/or lattices) that every launch covers;
// the host only reads the per-system scalars every check_every iterations.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <memory>
#include <mutex>
#include <vector>

#include "blas.h"
#include "kernels.h"
#include "outer.h"
#include "solver.h"

namespace bpp {

int work_read(int prec, int64_t* n, double* bytes, int reset);

void schur(const Batch& b, bool clover, int dag, char* in_e, char* out_e, char* tmp_o, cudaStream_t st) {
    // tmp_o = A_oo^-1 (-kappa H_oe in);  out_e = A_ee in + kappa H_eo tmp_o
    hop(b, 1, dag, clover ? HOP_INV : HOP_PLAIN, -1.0, in_e, tmp_o, nullptr, st);
    hop(b, 0, dag, clover ? HOP_CLOV_XPAY : HOP_XPAY, +1.0, tmp_o, out_e, in_e, st);
}

// Batch vector of `bt` (all systems, one parity).
struct Vec {
    DevBuf buf;
    char* p() const { return buf.as<char>(); }
};

static void read_scalars(const DevBuf& d, std::vector<KScal>& h, cudaStream_t st) {
    BPP_CUDA(cudaMemcpyAsync(h.data(), d.p, h.size() * sizeof(KScal), cudaMemcpyDeviceToHost, st));
    BPP_CUDA(cudaStreamSynchronize(st));
}
static void write_scalars(DevBuf& d, const std::vector<KScal>& h, cudaStream_t st) {
    BPP_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(KScal), cudaMemcpyHostToDevice, st));
}

// Loop control of the graph-captured inner solve: keep iterating while any
// system is active, at most max_loops times.
// Sets a graph condition.  A handle's default value is applied when the
// top-level graph is launched, not each time an enclosing body runs again, so
// a nested while loop is re-armed explicitly before it is reached.
__global__ void k_set_cond(cudaGraphConditionalHandle h, unsigned v) { cudaGraphSetConditional(h, v); }

// loops[0] counts the passes of this inner solve, loops[1] all passes since
// the solve started.
__global__ void k_loop_ctl(const KScal* sc, int n, int* loops, int max_loops, cudaGraphConditionalHandle h) {
    bool active = false;
    for (int s = threadIdx.x; s < n; s += 32) active = active || !sc[s].done;
    active = __any_sync(0xffffffffu, active);
    if (threadIdx.x == 0) {
        const int l = loops[0] + 1;
        loops[0] = l;
        loops[1] += 1;
        cudaGraphSetConditional(h, (active && l < max_loops) ? 1u : 0u);
    }
}

// Everything one configuration of systems needs, kept across calls so that
// repeated solves (a propagator's 12 sources, a benchmark loop) reuse the
// vectors, the reduction buffers and the instantiated inner-solve graph.
struct Plan {
    std::vector<const Gauge*> G;
    std::vector<double> kappa;
    bool clover = false;
    int prec = P32, solver = BPP_BICGSTAB;
    bool split = false;                  // double-float defects (split-FP64 vectors)
    bool dfcheck = false;                // the true-residual check in double-float too (x split only)
    bool reliable = false;               // FP32 recursive defect updates between recomputations
    Batch b64, bP, b64s, b32;
    Vec e32, m32, tmp32;
    Vec be, bo, bhat, xe, xo, r, tmpo;
    Vec be_s, bo_s, bhat_s, xe_s, m_s, tmpo_s, r_s;
    Vec w[9];
    RedBuf rb;
    DevBuf hred;                         // per-warp partials of the fused BiCGStab inner products
    int hred_wstride = 0;                // 0: inner products in separate vector kernels
    DevBuf d64, dP, dloops, dod, doc;
    std::vector<KScal> h64, hP;
    bool warmed = false;                 // one eager inner solve ran (autotuner populated)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_max_iter = -1;
    int body_kernels = 0;
    std::vector<double> iter_bytes;      // hopping-kernel bytes of one iteration, per system
    // the whole solve (outer loop included) as one graph launch
    cudaGraph_t wgraph = nullptr;
    cudaGraphExec_t wexec = nullptr;
    int wgraph_max_iter = -1;
    bool whole_warm = false;             // one host-driven solve ran (every branch kernel tuned)
    std::vector<double> w_iter_bytes;    // per system, inner precision
    double w_full_bytes[NPREC] = {}, w_rel_bytes[NPREC] = {}, w_schur_bytes[NPREC] = {};
    int64_t w_full_hops[NPREC] = {}, w_rel_hops[NPREC] = {}, w_schur_hops[NPREC] = {}, w_iter_hops = 0;
    int64_t w_full_launch = 0, w_rel_launch = 0, w_schur_launch = 0, w_iter_launch = 0;
    int64_t w_inner_launch = 0, w_pass_launch = 0;
    size_t bytes = 0;
    uint64_t last_use = 0;
    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (wexec) cudaGraphExecDestroy(wexec);
        if (wgraph) cudaGraphDestroy(wgraph);
    }
};

// The BiCGStab inner products fused into the hopping kernels (default), or
// in separate vector kernels with BPP_FUSED_DOTS=0; both are deterministic,
// with sums grouped differently.
static bool fused_dots() {
    const char* e = std::getenv("BPP_FUSED_DOTS");
    return !(e && e[0] == '0');
}

static std::mutex g_plan_mu;
static std::vector<std::unique_ptr<Plan>> g_plans;
static uint64_t g_plan_clock = 0;
static const size_t PLAN_BUDGET = (size_t)48 << 30;
static const size_t MAX_PLANS = 16;

static void alloc_vec(Plan& pl, Vec& v, const Batch& b) {
    v.buf.alloc_persistent(b.vec_bytes);
    pl.bytes += b.vec_bytes;
}

static Plan& get_plan(const std::vector<const Gauge*>& G, const std::vector<double>& kappa, bool clover, int prec,
                      int solver, bool split, bool dfcheck, cudaStream_t st) {
    ++g_plan_clock;
    for (auto& p : g_plans)
        if (p->G == G && p->kappa == kappa && p->clover == clover && p->prec == prec && p->solver == solver &&
            p->split == split && p->dfcheck == dfcheck) {
            p->last_use = g_plan_clock;
            return *p;
        }
    std::unique_ptr<Plan> pl(new Plan());
    pl->G = G;
    pl->kappa = kappa;
    pl->clover = clover;
    pl->prec = prec;
    pl->solver = solver;
    pl->split = split;
    pl->dfcheck = dfcheck;
    pl->b64.prec = P64;
    pl->bP.prec = prec;
    pl->b64s.prec = P64S;
    pl->b32.prec = P32;
    pl->reliable = split && prec == P16;
    // two-row links for the reduced-precision hops when every gauge is SU(3)
    pl->bP.comp = pl->b32.comp = true;
    for (auto* g : G) {
        pl->bP.comp = pl->bP.comp && link_compression(*g, prec);
        pl->b32.comp = pl->b32.comp && link_compression(*g, P32);
    }
    for (size_t s = 0; s < G.size(); ++s) {
        batch_add(pl->b64, *G[s], kappa[s], clover);
        batch_add(pl->bP, *G[s], kappa[s], clover);
        batch_add(pl->b64s, *G[s], kappa[s], clover);
        batch_add(pl->b32, *G[s], kappa[s], clover);
    }
    // evict least recently used plans beyond the count or byte budget
    const size_t need = (split ? 14 : 7) * pl->b64.vec_bytes + 9 * pl->bP.vec_bytes +
                        (pl->reliable ? 3 * pl->b32.vec_bytes : 0);
    for (;;) {
        size_t total = need;
        for (auto& p : g_plans) total += p->bytes;
        if (g_plans.empty() || (g_plans.size() < MAX_PLANS && total <= PLAN_BUDGET)) break;
        size_t lru = 0;
        for (size_t i = 1; i < g_plans.size(); ++i)
            if (g_plans[i]->last_use < g_plans[lru]->last_use) lru = i;
        BPP_CUDA(cudaDeviceSynchronize());
        g_plans.erase(g_plans.begin() + lru);
    }
    for (Batch* b : {&pl->b64, &pl->bP, &pl->b64s, &pl->b32}) {
        b->dsys.alloc_persistent(b->sys.size() * sizeof(SysDesc));
        BPP_CUDA(cudaMemcpy(b->dsys.p, b->sys.data(), b->sys.size() * sizeof(SysDesc), cudaMemcpyHostToDevice));
    }
    for (Vec* v : {&pl->be, &pl->bo, &pl->bhat, &pl->xe, &pl->xo, &pl->r, &pl->tmpo}) alloc_vec(*pl, *v, pl->b64);
    if (split)
        for (Vec* v : {&pl->be_s, &pl->bo_s, &pl->bhat_s, &pl->xe_s, &pl->m_s, &pl->tmpo_s, &pl->r_s})
            alloc_vec(*pl, *v, pl->b64s);
    if (pl->reliable)
        for (Vec* v : {&pl->e32, &pl->m32, &pl->tmp32}) alloc_vec(*pl, *v, pl->b32);
    for (auto& v : pl->w) alloc_vec(*pl, v, pl->bP);
    const int n = (int)G.size();
    pl->rb.persistent = true;
    if (solver == BPP_BICGSTAB && fused_dots()) {
        pl->hred_wstride = (pl->bP.Vh_max + 31) / 32;
        const size_t hb = (size_t)n * (pl->hred_wstride + hop_red_chunks(pl->hred_wstride)) * 4 * sizeof(double);
        pl->hred.alloc_persistent(hb);
        pl->bytes += hb;
    }
    pl->d64.alloc_persistent(n * sizeof(KScal));
    pl->dP.alloc_persistent(n * sizeof(KScal));
    pl->dloops.alloc_persistent(2 * sizeof(int));
    pl->dod.alloc_persistent(n * sizeof(OuterDev));
    pl->doc.alloc_persistent(sizeof(OuterCtl));
    BPP_CUDA(cudaMemset(pl->d64.p, 0, n * sizeof(KScal)));
    BPP_CUDA(cudaMemset(pl->dP.p, 0, n * sizeof(KScal)));
    pl->h64.resize(n);
    pl->hP.resize(n);
    pl->last_use = g_plan_clock;
    (void)st;
    g_plans.push_back(std::move(pl));
    return *g_plans.back();
}

void drop_plans(const Gauge* G) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    bool any = false;
    for (auto& p : g_plans)
        for (auto* g : p->G) any = any || G == nullptr || g == G;
    if (!any) return;
    cudaDeviceSynchronize();
    g_plans.erase(std::remove_if(g_plans.begin(), g_plans.end(),
                                 [&](const std::unique_ptr<Plan>& p) {
                                     if (G == nullptr) return true;
                                     for (auto* g : p->G)
                                         if (g == G) return true;
                                     return false;
                                 }),
                  g_plans.end());
}

// One iteration of the inner Krylov method on every active system.
static void inner_iteration(Plan& pl, const BlasVecs& v, char* tmp, cudaStream_t st) {
    const Batch& bP = pl.bP;
    KScal* sc = pl.dP.as<KScal>();
    const int* done = &sc[0].done;
    const int ds = (int)(sizeof(KScal) / sizeof(int));
    auto schur_s = [&](int dag, char* in, char* out, const HopRed* red = nullptr) {
        hop(bP, 1, dag, pl.clover ? HOP_INV : HOP_PLAIN, -1.0, in, tmp, nullptr, st, done, ds);
        hop(bP, 0, dag, pl.clover ? HOP_CLOV_XPAY : HOP_XPAY, +1.0, tmp, out, in, st, done, ds, red);
    };
    if (pl.solver == BPP_BICGSTAB && pl.hred_wstride > 0) {
        // <rhat, v> and <t, s>, ||t||^2 come from the second hop of each Schur
        // application (it holds v or t in registers and reads s as its xpay
        // operand): 15 vector passes per iteration instead of 18
        HopRed red;
        red.part = pl.hred.as<double>();
        red.wstride = pl.hred_wstride;
        red.op = HRED_ALPHA;
        red.rhat = v.rhat;
        double* chunks = red.part + (size_t)bP.nsys() * red.wstride * 4;
        schur_s(0, v.p, v.v, &red);
        hop_red_fin(bP, B_ALPHA, red.part, red.wstride, sc, pl.rb, chunks, st);
        blas(bP, B_S, v, sc, pl.rb, st);
        red.op = HRED_OMEGA;
        red.rhat = nullptr;
        schur_s(0, v.s, v.t, &red);
        hop_red_fin(bP, B_OMEGA, red.part, red.wstride, sc, pl.rb, chunks, st);
        blas(bP, B_XR, v, sc, pl.rb, st);
        blas(bP, B_P, v, sc, pl.rb, st);
    } else if (pl.solver == BPP_BICGSTAB) {
        schur_s(0, v.p, v.v);
        blas(bP, B_ALPHA, v, sc, pl.rb, st);
        blas(bP, B_S, v, sc, pl.rb, st);
        schur_s(0, v.s, v.t);
        blas(bP, B_OMEGA, v, sc, pl.rb, st);
        blas(bP, B_XR, v, sc, pl.rb, st);
        blas(bP, B_P, v, sc, pl.rb, st);
    } else {
        schur_s(0, v.p, v.w);
        blas(bP, B_CG_ALPHA, v, sc, pl.rb, st);
        blas(bP, B_CG_XR, v, sc, pl.rb, st);
        schur_s(1, v.r, v.z);
        blas(bP, B_CG_BETA, v, sc, pl.rb, st);
    }
}

static BlasVecs inner_vecs(Plan& pl) {
    BlasVecs v;
    if (pl.solver == BPP_BICGSTAB) {
        v.b = pl.w[0].p(); v.x = pl.w[1].p(); v.r = pl.w[2].p(); v.rhat = pl.w[3].p(); v.p = pl.w[4].p();
        v.v = pl.w[5].p(); v.s = pl.w[6].p(); v.t = pl.w[7].p();
    } else {
        v.b = pl.w[0].p(); v.x = pl.w[1].p(); v.r = pl.w[2].p(); v.z = pl.w[3].p(); v.p = pl.w[4].p();
        v.w = pl.w[5].p();
    }
    return v;
}

static void inner_init(Plan& pl, const BlasVecs& v, char* tmp, cudaStream_t st) {
    KScal* sc = pl.dP.as<KScal>();
    if (pl.solver == BPP_BICGSTAB) {
        blas(pl.bP, B_INIT_BICG, v, sc, pl.rb, st);
    } else {
        blas(pl.bP, B_CG_INIT, v, sc, pl.rb, st);
        schur(pl.bP, pl.clover, 1, v.r, v.z, tmp, st);
        blas(pl.bP, B_CG_PZ, v, sc, pl.rb, st);
    }
}

static int body_kernel_count(const Plan& pl) {
    // hop launches + blas launches per iteration (+ the loop control kernel);
    // the fused BiCGStab form replaces two vector kernels by two finalize kernels
    return pl.solver == BPP_BICGSTAB ? 4 + 5 + 1 : 4 + 4 + 1;
}

// Captures one iteration plus the loop control into the body of a while node.
static void build_graph(Plan& pl, int max_iter) {
    if (pl.exec) { cudaGraphExecDestroy(pl.exec); pl.exec = nullptr; }
    if (pl.graph) { cudaGraphDestroy(pl.graph); pl.graph = nullptr; }
    cudaStream_t cs;
    BPP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    try {
        BPP_CUDA(cudaGraphCreate(&pl.graph, 0));
        cudaGraphConditionalHandle handle;
        BPP_CUDA(cudaGraphConditionalHandleCreate(&handle, pl.graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        BPP_CUDA(cudaGraphAddNode(&node, pl.graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        BPP_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        capture_work_reset(pl.bP.nsys());
        set_capturing(true);
        try {
            BlasVecs v = inner_vecs(pl);
            inner_iteration(pl, v, pl.w[8].p(), cs);
            k_loop_ctl<<<1, 32, 0, cs>>>(pl.dP.as<KScal>(), pl.bP.nsys(), pl.dloops.as<int>(), max_iter + 1, handle);
            BPP_CHECK_LAUNCH();
        } catch (...) {
            set_capturing(false);
            cudaGraph_t dummy;
            cudaStreamEndCapture(cs, &dummy);
            throw;
        }
        set_capturing(false);
        pl.iter_bytes = capture_work_bytes(pl.prec);
        cudaGraph_t captured;
        BPP_CUDA(cudaStreamEndCapture(cs, &captured));
        BPP_CUDA(cudaGraphInstantiate(&pl.exec, pl.graph, 0));
        pl.graph_max_iter = max_iter;
        pl.body_kernels = body_kernel_count(pl);
    } catch (...) {
        cudaStreamDestroy(cs);
        throw;
    }
    BPP_CUDA(cudaStreamDestroy(cs));
}

// Inner Krylov solve Mhat e = rhs (in w[0]) on batch bP into w[1].
static void inner_solve(Plan& pl, const bpp_solve_opts& o, cudaStream_t st) {
    BlasVecs v = inner_vecs(pl);
    char* tmp = pl.w[8].p();
    inner_init(pl, v, tmp, st);
    if (o.use_graph && pl.warmed) {
        if (!pl.exec || pl.graph_max_iter != o.max_inner) build_graph(pl, o.max_inner);
        BPP_CUDA(cudaMemsetAsync(pl.dloops.p, 0, sizeof(int), st));   // this solve's pass counter
        BPP_CUDA(cudaGraphLaunch(pl.exec, st));
        int loops = 0;
        BPP_CUDA(cudaMemcpyAsync(&loops, pl.dloops.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        read_scalars(pl.dP, pl.hP, st);
        count_launch((int64_t)loops * pl.body_kernels);
        double bytes = 0.0;
        for (int s = 0; s < pl.bP.nsys() && s < (int)pl.iter_bytes.size(); ++s) bytes += pl.hP[s].iter * pl.iter_bytes[s];
        add_hop_work(pl.prec, (int64_t)loops * 4, bytes);
        return;
    }
    // eager: host checks every check_every iterations; the hopping kernels and
    // the vector updates skip systems that have converged
    const int max_chunks = o.max_inner / o.check_every + 2;
    for (int chunk = 0; chunk < max_chunks; ++chunk) {
        for (int k = 0; k < o.check_every; ++k) inner_iteration(pl, v, tmp, st);
        read_scalars(pl.dP, pl.hP, st);
        bool all = true;
        for (auto& k : pl.hP) all = all && k.done;
        if (all) break;
    }
    pl.warmed = true;
}

// ----------------------------------------------------------------------------- capture helpers
// Graph currently captured on stream cs.
static cudaGraph_t capture_graph(cudaStream_t cs) {
    cudaStreamCaptureStatus stt;
    cudaGraph_t g = nullptr;
    BPP_CUDA(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &g, nullptr, nullptr, nullptr));
    BPP_REQUIRE(stt == cudaStreamCaptureStatusActive && g, BPP_ERR_CUDA, "stream is not capturing");
    return g;
}

static unsigned long long new_handle(cudaStream_t cs, unsigned dflt) {
    cudaGraphConditionalHandle h;
    BPP_CUDA(cudaGraphConditionalHandleCreate(&h, capture_graph(cs), dflt, cudaGraphCondAssignDefault));
    return (unsigned long long)h;
}

// Appends a conditional node after everything captured so far on cs and
// returns its body graphs.
static std::vector<cudaGraph_t> add_conditional(cudaStream_t cs, unsigned long long h, cudaGraphConditionalNodeType type,
                                                unsigned size) {
    cudaStreamCaptureStatus stt;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t nd = 0;
    BPP_CUDA(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &g, &deps, &edata, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = (cudaGraphConditionalHandle)h;
    cp.conditional.type = type;
    cp.conditional.size = size;
    cudaGraphNode_t node;
    BPP_CUDA(cudaGraphAddNode(&node, g, deps, edata, nd, &cp));
    BPP_CUDA(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    std::vector<cudaGraph_t> bodies(cp.conditional.phGraph_out, cp.conditional.phGraph_out + size);
    return bodies;
}

// Captures f(stream) into the (empty) body graph.
template <class F>
static void capture_body(cudaGraph_t body, F f) {
    cudaStream_t cs;
    BPP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    BPP_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        f(cs);
    } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(cs, &dummy);
        cudaStreamDestroy(cs);
        throw;
    }
    cudaGraph_t captured;
    const cudaError_t e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    BPP_CUDA(e);
}

struct CapSnap {
    double bytes[NPREC];
    int64_t hops[NPREC];
    int64_t launches;
};
static CapSnap cap_snap(int n) {
    CapSnap c;
    for (int p = 0; p < NPREC; ++p) {
        c.bytes[p] = 0.0;
        const auto& v = capture_work_bytes(p);
        for (int s = 0; s < n && s < (int)v.size(); ++s) c.bytes[p] += v[s];
        c.hops[p] = capture_hop_launches(p);
    }
    c.launches = capture_launches();
    return c;
}

int solve_batch(const std::vector<const Gauge*>& G, const std::vector<double>& kappa, bool clover,
                const std::vector<const void*>& b_canon, const std::vector<void*>& x_canon, double tol,
                const bpp_solve_opts& o, bpp_solve_stats* stats, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    double work0 = 0.0;
    for (int q = 0; q < NPREC; ++q) {
        double by = 0.0;
        work_read(q, nullptr, &by, 0);
        work0 += by;
    }
    const int n = (int)G.size();
    BPP_REQUIRE(n >= 1 && n <= MAXSYS, BPP_ERR_INVALID_ARG, "number of systems must be 1..64");
    BPP_REQUIRE(tol > 0.0, BPP_ERR_INVALID_ARG, "tol must be positive");
    BPP_REQUIRE(o.solver == BPP_BICGSTAB || o.solver == BPP_CGNR, BPP_ERR_INVALID_ARG, "unknown solver");
    BPP_REQUIRE(o.inner_prec >= BPP_F64 && o.inner_prec <= BPP_F16, BPP_ERR_INVALID_ARG, "unknown inner precision");
    BPP_REQUIRE(o.max_inner > 0 && o.max_outer > 0 && o.check_every > 0, BPP_ERR_INVALID_ARG, "iteration caps must be positive");
    BPP_REQUIRE(o.outer_arith >= 0 && o.outer_arith <= 2, BPP_ERR_INVALID_ARG, "outer_arith must be 0, 1 or 2");

    std::lock_guard<std::mutex> lk(g_plan_mu);
    // a plain FP64 solve (FP64 inner) stays FP64 throughout
    const bool split = o.outer_arith != 0 && o.inner_prec != BPP_F64;
    // outer_arith 2: the true-residual check in double-float as well, the split
    // copy of x the only iterate (the returned solution)
    const bool dfcheck = split && o.outer_arith >= 2;
    Plan& pl = get_plan(G, kappa, clover, o.inner_prec, o.solver, split, dfcheck, st);
    const Batch& b64 = pl.b64;
    const Batch& bP = pl.bP;
    KScal* sc64 = pl.d64.as<KScal>();
    std::vector<KScal>& h64 = pl.h64;
    pl.rb.ensure(1, n, st);   // tickets

    // b -> even/odd FP64 (gamma5 b for the adjoint solve)
    const Batch& b64s = pl.b64s;
    for (int s = 0; s < n; ++s) full_to_eo(b64, s, 1, b_canon[s], 1, 0, pl.be.p(), pl.bo.p(), o.dagger ? 1 : 0, st);
    const int dag = 0;
    // ||b||^2 = ||b_e||^2 + ||b_o||^2
    std::vector<double> bnorm2(n), bscale(n, 1.0);
    {
        BlasVecs v;
        v.x = pl.be.p();
        v.r = pl.bo.p();
        blas(b64, B_NORM2X2, v, sc64, pl.rb, st);
        read_scalars(pl.d64, h64, st);
        for (int s = 0; s < n; ++s) bnorm2[s] = h64[s].bb;
    }
    for (int s = 0; s < n; ++s)
        BPP_REQUIRE(std::isfinite(bnorm2[s]), BPP_ERR_NONFINITE, "non-finite right-hand side");
    // The system is linear: solve D x' = b / ||b|| and return x = ||b|| x'.  The
    // normalised right-hand side keeps every split-FP64 value inside the FP32
    // exponent range whatever the scale of b.
    for (int s = 0; s < n; ++s) {
        if (bnorm2[s] > 0.0) {
            bscale[s] = std::sqrt(bnorm2[s]);
            bnorm2[s] = 1.0;
        }
        h64[s].scale = 1.0 / bscale[s];
    }
    write_scalars(pl.d64, h64, st);
    // (with the double-float check only the split copies of b are read later)
    scale_split(b64, pl.be.p(), split ? pl.be_s.p() : nullptr, sc64, st, !dfcheck);
    scale_split(b64, pl.bo.p(), split ? pl.bo_s.p() : nullptr, sc64, st, !dfcheck);
    // bhat = b_e + kappa H_eo A_oo^-1 b_o (double-float when split)
    {
        const Batch& bb = split ? b64s : b64;
        char* be_ = split ? pl.be_s.p() : pl.be.p();
        char* bo_ = split ? pl.bo_s.p() : pl.bo.p();
        char* tmp_ = split ? pl.tmpo_s.p() : pl.tmpo.p();
        char* bh_ = split ? pl.bhat_s.p() : pl.bhat.p();
        if (clover) {
            clover_apply(bb, 1, 1, bo_, tmp_, st);
            hop(bb, 0, dag, HOP_XPAY, +1.0, tmp_, bh_, be_, st);
        } else {
            hop(bb, 0, dag, HOP_XPAY, +1.0, bo_, bh_, be_, st);
        }
    }

    // initial guess (scaled like b)
    bool x_zero = !o.use_x0;
    if (o.use_x0) {
        for (int s = 0; s < n; ++s) full_to_eo(b64, s, 1, x_canon[s], 1, 0, pl.xe.p(), pl.xo.p(), o.dagger ? 1 : 0, st);
        scale_split(b64, pl.xe.p(), split ? pl.xe_s.p() : nullptr, sc64, st, !dfcheck);
    } else {
        if (!dfcheck) BPP_CUDA(cudaMemsetAsync(pl.xe.p(), 0, b64.vec_bytes, st));
        if (split) BPP_CUDA(cudaMemsetAsync(pl.xe_s.p(), 0, b64s.vec_bytes, st));
    }

    // Outer loop.  r (FP64) or r_s (split) holds the even defect; after a
    // "full" residual it is the even part of b - D x (equal to bhat - Mhat x_e,
    // since x_o is reconstructed from x_e) and rr_o the odd part, so the full
    // FP64 true residual is known.  The decisions are taken by the control
    // kernels of outer.cu on device state (OuterDev / OuterCtl): the host-driven
    // loop reads their flags back and launches the chosen branch; the
    // whole-solve graph branches on the same flags with conditional nodes.
    OuterDev* od = pl.dod.as<OuterDev>();
    OuterCtl* oc = pl.doc.as<OuterCtl>();
    KScal* scP = pl.dP.as<KScal>();
    const double eps32 = 4.0 * 5.96e-8;   // per-update error bound of a reliable FP32 defect update
    std::vector<OuterDev> hod(n);
    OuterCtl hoc{};

    // the branch kernel sequences (host-driven and captured alike)
    auto full_kernels = [&](cudaStream_t cs) {
        if (dfcheck) {
            // The same check in double-float arithmetic on the split iterate:
            // x_o = A_oo^-1 (b_o + kappa H_oe x_e) in one hop (kept in tmpo_s
            // for the returned x), De = A_ee x_e - kappa H_eo x_o, and the even
            // residual b_e - De as the next split defect.  The odd residual
            // vanishes by construction and is not recomputed.
            hop(b64s, 1, dag, clover ? HOP_INV_XPAY : HOP_XPAY, +1.0, pl.xe_s.p(), pl.tmpo_s.p(), pl.bo_s.p(), cs);
            hop(b64s, 0, dag, clover ? HOP_CLOV_XPAY : HOP_XPAY, -1.0, pl.tmpo_s.p(), pl.m_s.p(), pl.xe_s.p(), cs);
            split_residual(b64, pl.be_s.p(), pl.m_s.p(), pl.r_s.p(), sc64, pl.rb, cs);
            oc_full_even(od, oc, sc64, cs, true);
            return;
        }
        // The true residual of the returned x with the full FP64 D: h = kappa
        // H_oe x_e once, x_o = A_oo^-1 (b_o + h) and the odd residual
        // b_o - (A_oo x_o - h) from it, then De = A_ee x_e - kappa H_eo x_o and
        // the even residual b_e - De.
        hop(b64, 1, dag, HOP_PLAIN, +1.0, pl.xe.p(), pl.tmpo.p(), nullptr, cs);
        odd_reconstruct(b64, clover, pl.bo.p(), pl.tmpo.p(), pl.xo.p(), sc64, pl.rb, cs);
        oc_full_odd(od, sc64, n, cs);
        hop(b64, 0, dag, clover ? HOP_CLOV_XPAY : HOP_XPAY, -1.0, pl.xo.p(), pl.r.p(), pl.xe.p(), cs);
        outer_residual(b64, pl.be.p(), pl.r.p(), sc64, pl.rb, cs);
        oc_full_even(od, oc, sc64, cs);
    };
    auto reliable_kernels = [&](cudaStream_t cs) {
        to_f32(bP, pl.b32, pl.w[1].p(), pl.e32.p(), cs);
        schur(pl.b32, clover, dag, pl.e32.p(), pl.m32.p(), pl.tmp32.p(), cs);
        defect_update(b64, pl.b32, pl.r_s.p(), pl.m32.p(), sc64, pl.rb, cs);
        oc_after_reliable(od, oc, sc64, cs);
    };
    auto schur_kernels = [&](cudaStream_t cs) {
        if (split) {
            schur(b64s, clover, dag, pl.xe_s.p(), pl.m_s.p(), pl.tmpo_s.p(), cs);
            split_residual(b64, pl.bhat_s.p(), pl.m_s.p(), pl.r_s.p(), sc64, pl.rb, cs);
        } else {
            schur(b64, clover, dag, pl.xe.p(), pl.r.p(), pl.tmpo.p(), cs);
            outer_residual(b64, pl.bhat.p(), pl.r.p(), sc64, pl.rb, cs);
        }
        oc_after_schur(od, oc, sc64, cs);
    };
    auto downcast = [&](bool from_split, cudaStream_t cs) {
        outer_downcast(b64, bP, from_split ? pl.r_s.p() : pl.r.p(), pl.w[0].p(), sc64, cs, from_split);
    };
    auto read_state = [&]() {
        BPP_CUDA(cudaMemcpyAsync(hod.data(), od, n * sizeof(OuterDev), cudaMemcpyDeviceToHost, st));
        BPP_CUDA(cudaMemcpyAsync(&hoc, oc, sizeof(OuterCtl), cudaMemcpyDeviceToHost, st));
        BPP_CUDA(cudaStreamSynchronize(st));
    };

    // initial defect
    bool defect_split = false;
    if (x_zero) {
        if (split) {
            split_residual(b64, pl.bhat_s.p(), nullptr, pl.r_s.p(), sc64, pl.rb, st);
            defect_split = true;
        } else {
            BPP_CUDA(cudaMemsetAsync(pl.r.p(), 0, b64.vec_bytes, st));
            outer_residual(b64, pl.bhat.p(), pl.r.p(), sc64, pl.rb, st);
        }
    } else if (split) {
        schur(b64s, clover, dag, pl.xe_s.p(), pl.m_s.p(), pl.tmpo_s.p(), st);
        split_residual(b64, pl.bhat_s.p(), pl.m_s.p(), pl.r_s.p(), sc64, pl.rb, st);
        defect_split = true;
    } else {
        schur(b64, clover, dag, pl.xe.p(), pl.r.p(), pl.tmpo.p(), st);
        outer_residual(b64, pl.bhat.p(), pl.r.p(), sc64, pl.rb, st);
    }
    read_scalars(pl.d64, h64, st);
    for (int s = 0; s < n; ++s) {
        OuterDev d{};
        d.rr_e = h64[s].rr;
        d.target = tol;
        d.bnorm2 = bnorm2[s];
        d.status = BPP_OK;
        hod[s] = d;
    }
    hoc.tol = tol;
    hoc.inner_tol = o.inner_tol;
    hoc.eps32 = eps32;
    hoc.n = n;
    hoc.max_outer = o.max_outer;
    hoc.max_passes = o.max_outer + 8;
    hoc.max_inner = o.max_inner;
    hoc.prec = bP.prec;
    hoc.split = split;
    hoc.reliable = pl.reliable;
    hoc.defect_split = defect_split;
    BPP_CUDA(cudaMemcpyAsync(od, hod.data(), n * sizeof(OuterDev), cudaMemcpyHostToDevice, st));
    BPP_CUDA(cudaMemcpyAsync(oc, &hoc, sizeof(OuterCtl), cudaMemcpyHostToDevice, st));

    if (o.use_graph == 2 && pl.whole_warm) {
        // the whole correction loop as one graph launch
        if (!pl.wexec || pl.wgraph_max_iter != o.max_inner) {
            if (pl.wexec) { cudaGraphExecDestroy(pl.wexec); pl.wexec = nullptr; }
            if (pl.wgraph) { cudaGraphDestroy(pl.wgraph); pl.wgraph = nullptr; }
            BPP_CUDA(cudaStreamSynchronize(st));
            cudaStream_t s0;
            BPP_CUDA(cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking));
            BPP_CUDA(cudaGraphCreate(&pl.wgraph, 0));
            capture_work_reset(n);
            set_capturing(true);
            try {
                BPP_CUDA(cudaStreamBeginCaptureToGraph(s0, pl.wgraph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
                const unsigned long long h_outer = new_handle(s0, 1);
                auto outer_body = add_conditional(s0, h_outer, cudaGraphCondTypeWhile, 1);
                capture_body(outer_body[0], [&](cudaStream_t s1) {
                    const unsigned long long h_check = new_handle(s1, 0), h_inner = new_handle(s1, 0);
                    const CapSnap p0 = cap_snap(n);
                    oc_classify(od, oc, h_check, h_inner, s1);
                    const CapSnap p1 = cap_snap(n);
                    capture_body(add_conditional(s1, h_check, cudaGraphCondTypeIf, 1)[0], full_kernels);
                    const CapSnap p2 = cap_snap(n);
                    for (int q = 0; q < NPREC; ++q) {
                        pl.w_full_bytes[q] = p2.bytes[q] - p1.bytes[q];
                        pl.w_full_hops[q] = p2.hops[q] - p1.hops[q];
                    }
                    pl.w_full_launch = p2.launches - p1.launches;
                    capture_body(add_conditional(s1, h_inner, cudaGraphCondTypeIf, 1)[0], [&](cudaStream_t s2) {
                        const unsigned long long h_split = new_handle(s2, 0), h_branch = new_handle(s2, 0);
                        const CapSnap i0 = cap_snap(n);
                        oc_inner_setup(od, oc, sc64, scP, h_split, s2);
                        auto dc = add_conditional(s2, h_split, cudaGraphCondTypeIf, 2);
                        capture_body(dc[0], [&](cudaStream_t s3) { downcast(true, s3); });
                        capture_body(dc[1], [&](cudaStream_t s3) { downcast(false, s3); });
                        BlasVecs v = inner_vecs(pl);
                        inner_init(pl, v, pl.w[8].p(), s2);
                        BPP_CUDA(cudaMemsetAsync(pl.dloops.p, 0, sizeof(int), s2));
                        const unsigned long long h_it = new_handle(s2, 1);
                        k_set_cond<<<1, 1, 0, s2>>>((cudaGraphConditionalHandle)h_it, 1u);
                        count_launch();
                        BPP_CHECK_LAUNCH();
                        const CapSnap i1 = cap_snap(n);
                        const std::vector<double> before = capture_work_bytes(bP.prec);
                        capture_body(add_conditional(s2, h_it, cudaGraphCondTypeWhile, 1)[0], [&](cudaStream_t s3) {
                            inner_iteration(pl, v, pl.w[8].p(), s3);
                            k_loop_ctl<<<1, 32, 0, s3>>>(scP, n, pl.dloops.as<int>(), o.max_inner + 1,
                                                         (cudaGraphConditionalHandle)h_it);
                            count_launch();
                            BPP_CHECK_LAUNCH();
                        });
                        const CapSnap i2 = cap_snap(n);
                        pl.w_iter_bytes.assign(n, 0.0);
                        {
                            const auto& after = capture_work_bytes(bP.prec);
                            for (int s = 0; s < n; ++s)
                                pl.w_iter_bytes[s] = (s < (int)after.size() ? after[s] : 0.0) -
                                                     (s < (int)before.size() ? before[s] : 0.0);
                        }
                        pl.w_iter_launch = i2.launches - i1.launches;
                        pl.w_iter_hops = i2.hops[bP.prec] - i1.hops[bP.prec];
                        outer_accumulate(b64, bP, dfcheck ? nullptr : pl.xe.p(), pl.w[1].p(), sc64, s2, split ? pl.xe_s.p() : nullptr);
                        oc_decide(od, oc, scP, h_branch, s2);
                        const CapSnap i3 = cap_snap(n);
                        // both downcast variants were captured, one runs
                        pl.w_inner_launch = (i1.launches - i0.launches) - 1 + (i3.launches - i2.launches);
                        auto br = add_conditional(s2, h_branch, cudaGraphCondTypeSwitch, 3);
                        const CapSnap b0 = cap_snap(n);
                        capture_body(br[OB_FULL], full_kernels);
                        const CapSnap b1 = cap_snap(n);
                        if (pl.reliable) capture_body(br[OB_RELIABLE], reliable_kernels);
                        const CapSnap b2 = cap_snap(n);
                        capture_body(br[OB_SCHUR], schur_kernels);
                        const CapSnap b3 = cap_snap(n);
                        for (int q = 0; q < NPREC; ++q) {
                            pl.w_rel_bytes[q] = b2.bytes[q] - b1.bytes[q];
                            pl.w_schur_bytes[q] = b3.bytes[q] - b2.bytes[q];
                            pl.w_rel_hops[q] = b2.hops[q] - b1.hops[q];
                            pl.w_schur_hops[q] = b3.hops[q] - b2.hops[q];
                        }
                        pl.w_rel_launch = b2.launches - b1.launches;
                        pl.w_schur_launch = b3.launches - b2.launches;
                    });
                    oc_loop(oc, h_outer, s1);
                    pl.w_pass_launch = 2;
                    (void)p0;
                });
                cudaGraph_t captured;
                BPP_CUDA(cudaStreamEndCapture(s0, &captured));
            } catch (...) {
                set_capturing(false);
                cudaGraph_t dummy;
                cudaStreamEndCapture(s0, &dummy);
                cudaStreamDestroy(s0);
                if (pl.wgraph) { cudaGraphDestroy(pl.wgraph); pl.wgraph = nullptr; }
                throw;
            }
            set_capturing(false);
            cudaStreamDestroy(s0);
            BPP_CUDA(cudaGraphInstantiate(&pl.wexec, pl.wgraph, 0));
            pl.wgraph_max_iter = o.max_inner;
        }
        BPP_CUDA(cudaMemsetAsync(pl.dloops.p, 0, 2 * sizeof(int), st));
        BPP_CUDA(cudaGraphLaunch(pl.wexec, st));
        read_state();
        int loops[2] = {0, 0};
        BPP_CUDA(cudaMemcpy(loops, pl.dloops.p, 2 * sizeof(int), cudaMemcpyDeviceToHost));
        // credit the work the graph did: every inner iteration of an active
        // system, and every executed branch for all systems
        for (int q = 0; q < NPREC; ++q) {
            double by = hoc.n_full * pl.w_full_bytes[q] + hoc.n_rel * pl.w_rel_bytes[q] + hoc.n_schur * pl.w_schur_bytes[q];
            int64_t hops = hoc.n_full * pl.w_full_hops[q] + hoc.n_rel * pl.w_rel_hops[q] + hoc.n_schur * pl.w_schur_hops[q];
            if (q == bP.prec) {
                for (int s = 0; s < n; ++s) by += hod[s].inner_it * pl.w_iter_bytes[s];
                hops += (int64_t)loops[1] * pl.w_iter_hops;
            }
            if (by > 0 || hops > 0) add_hop_work(q, hops, by);
        }
        count_launch((int64_t)hoc.passes * pl.w_pass_launch + (int64_t)hoc.n_inner * pl.w_inner_launch +
                     (int64_t)loops[1] * pl.w_iter_launch + (int64_t)hoc.n_full * pl.w_full_launch +
                     (int64_t)hoc.n_rel * pl.w_rel_launch + (int64_t)hoc.n_schur * pl.w_schur_launch);
    } else {
        for (int pass = 0; pass < hoc.max_passes; ++pass) {
            oc_classify(od, oc, 0, 0, st);
            read_state();
            if (hoc.check) {
                full_kernels(st);
            } else if (hoc.inner) {
                oc_inner_setup(od, oc, sc64, scP, 0, st);
                downcast(hoc.defect_split != 0, st);
                inner_solve(pl, o, st);
                outer_accumulate(b64, bP, dfcheck ? nullptr : pl.xe.p(), pl.w[1].p(), sc64, st, split ? pl.xe_s.p() : nullptr);
                oc_decide(od, oc, scP, 0, st);
                read_state();
                if (hoc.branch == OB_FULL) full_kernels(st);
                else if (hoc.branch == OB_RELIABLE) reliable_kernels(st);
                else schur_kernels(st);
            }
            oc_loop(oc, 0, st);
            if (!hoc.check && !hoc.inner) break;
        }
        pl.whole_warm = true;
    }
    read_state();
    std::vector<double> rr_e(n), rr_o(n), true_res(n);
    std::vector<int> outer(n), inner_it(n), conv(n), status(n);
    for (int s = 0; s < n; ++s) {
        rr_e[s] = hod[s].rr_e;
        rr_o[s] = hod[s].rr_o;
        true_res[s] = hod[s].true_res;
        outer[s] = hod[s].outer;
        inner_it[s] = hod[s].inner_it;
        conv[s] = hod[s].conv;
        status[s] = hod[s].status;
    }
    bool have_full = hoc.have_full != 0;
    if (!have_full) {
        full_kernels(st);
        read_state();
        for (int s = 0; s < n; ++s) {
            rr_e[s] = hod[s].rr_e;
            rr_o[s] = hod[s].rr_o;
        }
        have_full = true;
        for (int s = 0; s < n; ++s) {
            if (status[s] != BPP_OK || bnorm2[s] == 0.0) continue;
            true_res[s] = std::sqrt((rr_e[s] + rr_o[s]) / bnorm2[s]);
            conv[s] = true_res[s] <= tol;
        }
    } else {
        for (int s = 0; s < n; ++s)
            if (status[s] == BPP_OK && bnorm2[s] > 0.0) true_res[s] = std::sqrt((rr_e[s] + rr_o[s]) / bnorm2[s]);
    }
    // x = ||b|| x' (with the double-float check the checked split iterate is
    // the solution: x_e, and x_o in tmpo_s, converted on the way out)
    for (int s = 0; s < n; ++s) {
        if (dfcheck)
            eo_to_full(b64s, s, 1, pl.xe_s.p(), pl.tmpo_s.p(), x_canon[s], 1, 0, o.dagger ? 1 : 0, st, bscale[s]);
        else
            eo_to_full(b64, s, 1, pl.xe.p(), pl.xo.p(), x_canon[s], 1, 0, o.dagger ? 1 : 0, st, bscale[s]);
    }
    BPP_CUDA(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    double work1 = 0.0;
    for (int q = 0; q < NPREC; ++q) {
        double by = 0.0;
        work_read(q, nullptr, &by, 0);
        work1 += by;
    }
    int rc = BPP_OK;
    for (int s = 0; s < n; ++s) {
        if (status[s] == BPP_OK && !conv[s]) status[s] = BPP_ERR_NOT_CONVERGED;
        if (status[s] != BPP_OK && rc == BPP_OK) rc = status[s];
        if (stats) {
            stats[s].outer_iters = outer[s];
            stats[s].inner_iters = inner_it[s];
            stats[s].converged = conv[s];
            stats[s].status = status[s];
            stats[s].true_resid = true_res[s];
            stats[s].seconds = secs;
            stats[s].hop_bytes = work1 - work0;
            stats[s].hop_gbs = secs > 0.0 ? (work1 - work0) / secs / 1e9 : 0.0;
        }
    }
    return rc;
}

}  // namespace bpp
