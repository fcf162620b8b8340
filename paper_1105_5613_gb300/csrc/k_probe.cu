// Peak FP32 / FP64 fused multiply-add rate of the current device, measured: the roofline
// denominator of the pair-force kernels, which are bound by arithmetic issue rather than
// by memory (the paper's own timings are whole-machine; it has no counterpart of this).
//
// Every thread runs kChains independent dependent chains a <- a * b + c; with enough
// resident warps the FMA pipes never wait on a chain's latency, and nothing is loaded or
// stored in the loop.  The flops counted are 2 per FMA.
#include <algorithm>

#include "bbmd_internal.cuh"

namespace bbmd {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chain(T b, T c, int iters, T* sink) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = a[k] * b + c;
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // a data-dependent store keeps the chains alive; in practice never taken
    if (s == (T)12345.678) sink[blockIdx.x] = s;
}

template <typename T>
double measure(int nsm, int iters, int repeats, T* sink) {
    const int blocks = nsm * 8;  // 2048 threads per SM
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b slightly below 1 and c small keep the values finite and normal
    const T b = (T)0.999999, c = (T)1e-3;
    k_fma_chain<T><<<blocks, kProbeThreads>>>(b, c, std::max(1, iters / 10), sink);  // warm-up
    float best = 0.f;
    for (int r = 0; r < repeats; ++r) {
        cudaEventRecord(e0);
        k_fma_chain<T><<<blocks, kProbeThreads>>>(b, c, iters, sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * kChains * 16.0 * (double)iters * (double)blocks * kProbeThreads;
    return best > 0.f ? flops / (best * 1e-3) / 1e12 : 0.0;
}

}  // namespace
}  // namespace bbmd

extern "C" bbmd_status bbmd_fma_peak(int32_t precision, int32_t* sm_count, double* tflops) {
    if (!tflops || (precision != BBMD_PREC_MIXED && precision != BBMD_PREC_FP64))
        return BBMD_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm <= 0) {
        cudaGetLastError();
        return BBMD_ERR_CUDA;
    }
    if (sm_count) *sm_count = nsm;
    void* sink = nullptr;
    if (cudaMalloc(&sink, (size_t)nsm * 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return BBMD_ERR_OOM;
    }
    // about 0.1 s per timed FP32 launch at 80 TFLOP/s; FP64 issues far fewer per clock
    *tflops = precision == BBMD_PREC_FP64
                  ? bbmd::measure<double>(nsm, 2000, 3, (double*)sink)
                  : bbmd::measure<float>(nsm, 100000, 3, (float*)sink);
    cudaFree(sink);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess && *tflops > 0.0 ? BBMD_OK : BBMD_ERR_CUDA;
}
