// Library runtime: thread-local last error, launch counter, block-size
// autotuner with an optional cache file, hopping-kernel timing, stream-ordered
// scratch memory.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <vector>

#include "bpp_internal.h"

namespace bpp {

static std::atomic<int64_t> g_launches{0};
static thread_local bool t_capturing = false;

void set_capturing(bool on) { t_capturing = on; }
bool thread_capturing() { return t_capturing; }

static std::mutex g_work_mu;
static int64_t g_work_n[NPREC] = {};
static double g_work_bytes[NPREC] = {};
static thread_local std::vector<double> t_cap_bytes[NPREC];
static thread_local int64_t t_cap_launches = 0;
static thread_local int64_t t_cap_hops[NPREC] = {};

void add_hop_work(int prec, int64_t launches, double bytes) {
    std::lock_guard<std::mutex> lk(g_work_mu);
    g_work_n[prec] += launches;
    g_work_bytes[prec] += bytes;
}
void capture_hop_work(int prec, int sys, double bytes) {
    if ((int)t_cap_bytes[prec].size() <= sys) t_cap_bytes[prec].resize(sys + 1, 0.0);
    t_cap_bytes[prec][sys] += bytes;
}
void capture_work_reset(int nsys) {
    for (auto& v : t_cap_bytes) v.assign(nsys, 0.0);
    for (auto& h : t_cap_hops) h = 0;
    t_cap_launches = 0;
}
void capture_hop_launch(int prec) { t_cap_hops[prec] += 1; }
int64_t capture_hop_launches(int prec) { return t_cap_hops[prec]; }
const std::vector<double>& capture_work_bytes(int prec) { return t_cap_bytes[prec]; }
int64_t capture_launches() { return t_cap_launches; }

int work_read(int prec, int64_t* n, double* bytes, int reset) {
    if (prec < 0 || prec >= NPREC) return BPP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_work_mu);
    if (n) *n = g_work_n[prec];
    if (bytes) *bytes = g_work_bytes[prec];
    if (reset) { g_work_n[prec] = 0; g_work_bytes[prec] = 0; }
    return 0;
}

void count_launch(int64_t n) {
    if (!t_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
    else t_cap_launches += n;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// ----------------------------------------------------------------------------- autotuner
static std::mutex g_tune_mu;
static std::map<std::string, int>* g_tune = nullptr;

static const char* tune_file() { return std::getenv("BPP_TUNE_CACHE"); }

static void tune_load_locked() {
    if (g_tune) return;
    g_tune = new std::map<std::string, int>();
    const char* f = tune_file();
    if (!f) return;
    std::ifstream in(f);
    std::string k;
    int b;
    while (in >> k >> b) (*g_tune)[k] = b;
}

int tune_lookup(const std::string& key) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune->find(key);
    return it == g_tune->end() ? 0 : it->second;
}

void tune_store(const std::string& key, int block) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    (*g_tune)[key] = block;
    const char* f = tune_file();
    if (!f) return;
    std::ofstream out(f, std::ios::trunc);
    for (auto& kv : *g_tune) out << kv.first << " " << kv.second << "\n";
}

// ----------------------------------------------------------------------------- profiling
struct ProfRec {
    int prec;
    double bytes;
    cudaEvent_t e0, e1;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static int64_t g_prof_n[NPROF] = {};
static double g_prof_ms[NPROF] = {};
static double g_prof_bytes[NPROF] = {};

ProfScope::ProfScope(int p, double b, cudaStream_t st) : prec(p), bytes(b), s(st), on(false) {
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_prof_on) return;
    }
    if (capturing(st)) return;
    if (cudaEventCreate(&e0) != cudaSuccess) return;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
    cudaEventRecord(e0, s);
    on = true;
}

ProfScope::~ProfScope() {
    if (!on) return;
    cudaEventRecord(e1, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back({prec, bytes, e0, e1});
}

static void prof_drain_locked() {
    for (auto& r : g_prof) {
        float ms = 0.f;
        cudaEventSynchronize(r.e1);
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        g_prof_n[r.prec] += 1;
        g_prof_ms[r.prec] += ms;
        g_prof_bytes[r.prec] += r.bytes;
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    g_prof.clear();
}

int prof_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return 0;
}

int prof_read(int prec, int64_t* n, double* ms, double* bytes, int reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain_locked();
    if (prec < 0 || prec >= NPROF) return BPP_ERR_INVALID_ARG;
    if (n) *n = g_prof_n[prec];
    if (ms) *ms = g_prof_ms[prec];
    if (bytes) *bytes = g_prof_bytes[prec];
    if (reset) {
        g_prof_n[prec] = 0;
        g_prof_ms[prec] = 0;
        g_prof_bytes[prec] = 0;
    }
    return 0;
}

int64_t launch_count(int reset) {
    return reset ? g_launches.exchange(0) : g_launches.load();
}

// ----------------------------------------------------------------------------- scratch
static std::once_flag g_pool_once;

static void pool_setup() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;   // keep freed blocks cached in the pool
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

void DevBuf::alloc(size_t bytes, cudaStream_t st) {
    release();
    std::call_once(g_pool_once, pool_setup);
    s = st;
    n = bytes;
    if (bytes == 0) return;
    BPP_CUDA(cudaMallocAsync(&p, bytes, st));
}

void DevBuf::alloc_persistent(size_t bytes) {
    release();
    persistent = true;
    n = bytes;
    if (bytes == 0) return;
    BPP_CUDA(cudaMalloc(&p, bytes));
}

void DevBuf::release() {
    if (p) {
        if (persistent) cudaFree(p);
        else cudaFreeAsync(p, s);
    }
    p = nullptr;
    n = 0;
    persistent = false;
}

int release_workspace() {
    cudaDeviceSynchronize();
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    return 0;
}

}  // namespace bpp
