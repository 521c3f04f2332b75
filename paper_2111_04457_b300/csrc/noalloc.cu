// bpp_dslash_noalloc: the even-odd hopping term (the bpp_dslash EVEN/ODD mode)
// for callers that cannot allocate device memory -- for example a host
// application whose memory manager owns the whole device and forbids other
// libraries from calling cudaMalloc, or code running where an allocation
// could fail or stall at an unpredictable point.  The working storage of the
// call (the system table and the two internal half fields) lives in one
// file-scope device array of fixed size instead of being allocated.
#include <cstdio>
#include <mutex>
#include <string>

#include "gauge.h"
#include "kernels.h"

namespace bpp {
void hop_fixed(int prec, const SysDesc* dsys, int nsys, int Vh, int parity, int mode, double a_sign, char* in,
               char* out, char* y, cudaStream_t st);
void half_to_int_fixed(int prec, const SysDesc* dsys, int nsys, int Vh, const void* canon, int canon_f64, char* out,
                       cudaStream_t st);
void int_to_half_fixed(int prec, const SysDesc* dsys, int nsys, int Vh, const char* in, void* canon, int canon_f64,
                       cudaStream_t st);
int set_error(int code, const char* msg);
}  // namespace bpp

using namespace bpp;

// 32 MiB per device.  The library is built without relocatable device code,
// so this file's device code is a module of its own; the array is placed on a
// device when that module is loaded there (at the first gauge handle created
// on the device, see noalloc_prepare) and stays until the process exits.
#define BPP_NOALLOC_SCRATCH_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[BPP_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {};

// Writes the call's system table: n copies of d, the copy for right-hand side
// r at byte offset r * field of the scratch vectors.  The descriptor travels
// as a kernel parameter, so no host buffer has to outlive the call.
__global__ void k_noalloc_table(SysDesc d, int n, int64_t field, SysDesc* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    SysDesc e = d;
    e.vec_off = (int64_t)r * field;
    out[r] = e;
}

namespace bpp {
// Device address of the scratch array on device `dev` (which must be the
// current device).  In host code the array's name is only a host-side
// stand-in, so the address is looked up with cudaGetSymbolAddress and cached
// per device.  The lookup also loads the module that holds the array: the
// library is built without relocatable device code, so this file's device
// code is a module of its own and, under lazy module loading, its 32 MiB
// array is only placed on the device at this point.  bpp_gauge_create calls
// this for its device (it allocates anyway), so a later bpp_dslash_noalloc
// call, which needs a gauge handle of the same device, finds the array in
// place and causes no device allocation.
int noalloc_prepare(int dev, cudaStream_t st, std::string* err, void** ptr) {
    if (dev < 0 || dev >= 64) {
        if (err) *err = "device ordinal >= 64";
        return BPP_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev]) {
        if (ptr) *ptr = g_noalloc_ptr[dev];
        return BPP_OK;
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        if (err) *err = std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e);
        return BPP_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
    // one launch that writes nothing loads the table kernel as well
    k_noalloc_table<<<1, 32, 0, st>>>(SysDesc{}, 0, 0, nullptr);
    count_launch();
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        if (err) *err = std::string("launch of the table kernel failed: ") + cudaGetErrorString(le);
        return BPP_ERR_CUDA;
    }
    if (ptr) *ptr = p;
    return BPP_OK;
}
}  // namespace bpp

extern "C" int bpp_dslash_noalloc(bpp_gauge U, const void* psi, void* out, double kappa, int parity, int prec,
                                  int nrhs, bpp_stream stream) {
    if (!U || !psi || !out || psi == out) return set_error(BPP_ERR_INVALID_ARG, "bpp_dslash_noalloc: NULL or aliased field");
    if (parity != BPP_EVEN && parity != BPP_ODD)
        return set_error(BPP_ERR_INVALID_ARG, "bpp_dslash_noalloc: parity must be BPP_EVEN or BPP_ODD");
    if (prec != BPP_F64 && prec != BPP_F32 && prec != BPP_F16)
        return set_error(BPP_ERR_INVALID_ARG, "bpp_dslash_noalloc: unknown precision");
    if (nrhs < 1 || nrhs > MAXSYS) return set_error(BPP_ERR_INVALID_ARG, "bpp_dslash_noalloc: nrhs must be 1..64");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(BPP_ERR_CUDA, "bpp_dslash_noalloc: cudaGetDevice failed");
    if (dev != U->device)
        return set_error(BPP_ERR_INVALID_ARG, "bpp_dslash_noalloc: the current device is not the gauge field's device");
    // scratch layout: [system table, 256-byte aligned][input half fields][output half fields]
    const size_t table = ((size_t)MAXSYS * sizeof(SysDesc) + 255) / 256 * 256;
    const size_t field = spinor_alloc_bytes(prec, U->stride);
    const size_t need = table + 2 * (size_t)nrhs * field;
    if (need > BPP_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "bpp_dslash_noalloc: needs %zu bytes of scratch for this lattice, precision and nrhs; the "
                      "static maximum is %u bytes (use bpp_dslash)",
                      need, (unsigned)BPP_NOALLOC_SCRATCH_BYTES);
        return set_error(BPP_ERR_INVALID_ARG, msg);
    }
    std::string err;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    const int rc = noalloc_prepare(dev, st, &err, &scratch);
    if (rc != BPP_OK) return set_error(rc, ("bpp_dslash_noalloc: " + err).c_str());
    unsigned char* base = static_cast<unsigned char*>(scratch);

    SysDesc d;
    d.g = U->g;
    for (int p = 0; p < 2; ++p) {
        for (int mu = 0; mu < 4; ++mu) d.U[p][mu] = link_view(*U, prec, p, mu);
        d.A[p] = CloverView{nullptr, U->stride};
        d.Ainv[p] = CloverView{nullptr, U->stride};
    }
    d.kappa = kappa;
    d.vec_off = 0;
    d.stride = U->stride;
    k_noalloc_table<<<1, MAXSYS, 0, st>>>(d, nrhs, (int64_t)field, reinterpret_cast<SysDesc*>(base));
    count_launch();
    const SysDesc* dsys = reinterpret_cast<const SysDesc*>(base);
    char* vin = reinterpret_cast<char*>(base + table);
    char* vout = vin + (size_t)nrhs * field;
    const int f64 = prec == BPP_F64;
    half_to_int_fixed(prec, dsys, nrhs, U->g.Vh, psi, f64, vin, st);
    hop_fixed(prec, dsys, nrhs, U->g.Vh, parity, HOP_PLAIN, -1.0, vin, vout, nullptr, st);
    int_to_half_fixed(prec, dsys, nrhs, U->g.Vh, vout, out, f64, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof(msg), "bpp_dslash_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
        return set_error(BPP_ERR_CUDA, msg);
    }
    return BPP_OK;
}
