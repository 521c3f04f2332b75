// Throughput of the FMA pipes (FP64 and FP32) measured with a synthetic
// kernel: the roofline denominators of the ALU-bound hopping kernels (the
// FP64 hop runs on the FP64 FMA pipe, the double-float hop on the FP32 one;
// cuBLAS DGEMM runs on the FP64 tensor cores instead and is no peak for them).
#include <algorithm>

#include "bpp_internal.h"

namespace bpp {

// Every thread runs NA independent chains a = a * b + c for `iters` rounds;
// the result is stored only if it hits an impossible value, so the compiler
// keeps the arithmetic and nothing is written.
template <class T, int NA>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, T b, T c, int iters) {
    T a[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NA; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < NA; ++k) s += a[k];
    if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

double fma_peak(int prec, cudaStream_t st) {
    BPP_REQUIRE(prec == P64 || prec == P32, BPP_ERR_INVALID_ARG, "fma peak: prec must be F64 or F32");
    int dev = 0, sms = 0;
    BPP_CUDA(cudaGetDevice(&dev));
    BPP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = sms * 8;
    constexpr int NA64 = 8, NA32 = 16;
    const int iters = prec == P64 ? 4000 : 40000;
    DevBuf out((size_t)blocks * threads * sizeof(double), st);
    cudaEvent_t e0, e1;
    BPP_CUDA(cudaEventCreate(&e0));
    BPP_CUDA(cudaEventCreate(&e1));
    auto run = [&]() {
        if (prec == P64) k_fma_peak<double, NA64><<<blocks, threads, 0, st>>>(out.as<double>(), 0.999999, 1e-7, iters);
        else k_fma_peak<float, NA32><<<blocks, threads, 0, st>>>(out.as<float>(), 0.999999f, 1e-7f, iters);
        BPP_CHECK_LAUNCH();
    };
    run();
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        BPP_CUDA(cudaEventRecord(e0, st));
        run();
        BPP_CUDA(cudaEventRecord(e1, st));
        BPP_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        BPP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)blocks * threads * iters * (prec == P64 ? NA64 : NA32);
    return 2.0 * fmas / (best * 1e-3) / 1e12;
}

}  // namespace bpp
