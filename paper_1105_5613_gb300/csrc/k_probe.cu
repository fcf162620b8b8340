// Hardware rates the kernels' design rests on, measured on the current device (the paper's
// own timings are whole-machine; it has no counterpart of these):
//   - the peak FP32 / FP64 fused multiply-add rate: the roofline denominator of the
//     pair-force kernels, which are bound by arithmetic issue rather than by memory;
//   - the rate of shared-memory scatter-adds: the cost of the reaction update a Newton's
//     third law (half list) force kernel would add to every pair.
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

// Shared-memory scatter: every thread adds into a 2048-entry shared array at addresses
// that differ across the lanes of a warp (no bank conflicts: the most favourable case of
// a reaction scatter).  KIND 0: 64-bit integer adds of a float converted to 2^32 fixed
// point; 1: 32-bit integer adds; 2: FP32 adds.
constexpr int kScatterN = 2048;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_scatter(int iters, float x0,
                                                           unsigned long long* sink) {
    __shared__ unsigned long long a64[kScatterN];
    __shared__ unsigned int a32[kScatterN];
    __shared__ float af[kScatterN];
    for (int i = threadIdx.x; i < kScatterN; i += blockDim.x) {
        a64[i] = 0;
        a32[i] = 0;
        af[i] = 0.f;
    }
    __syncthreads();
    float x = x0 + 0.37f * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
        const int idx = (threadIdx.x * 37 + it * 101) & (kScatterN - 1);
        if (KIND == 0) atomicAdd(&a64[idx], (unsigned long long)__float2ll_rn(x * 4294967296.0f));
        if (KIND == 1) atomicAdd(&a32[idx], (unsigned)(it + threadIdx.x));
        if (KIND == 2) atomicAdd(&af[idx], x);
        x += 1e-3f;
    }
    __syncthreads();
    unsigned long long s = 0;
    for (int i = threadIdx.x; i < kScatterN; i += blockDim.x) s += a64[i] + a32[i] + (unsigned long long)af[i];
    if (s == 12345ull) sink[blockIdx.x] = s;
}

template <int KIND>
double scatter_rate(int nsm, unsigned long long* sink) {
    const int blocks = nsm * 4, iters = 20000;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_scatter<KIND><<<blocks, kProbeThreads>>>(iters / 10, 1.f, sink);  // warm-up
    float best = 0.f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        k_scatter<KIND><<<blocks, kProbeThreads>>>(iters, 1.f, sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best > 0.f ? (double)blocks * kProbeThreads * iters / (best * 1e-3) : 0.0;
}

}  // namespace
}  // namespace bbmd

extern "C" bbmd_status bbmd_smem_scatter_rate(int32_t kind, double* adds_per_s) {
    if (!adds_per_s || kind < 0 || kind > 2) return BBMD_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm <= 0) {
        cudaGetLastError();
        return BBMD_ERR_CUDA;
    }
    void* sink = nullptr;
    if (cudaMalloc(&sink, (size_t)nsm * 4 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return BBMD_ERR_OOM;
    }
    unsigned long long* s = (unsigned long long*)sink;
    *adds_per_s = kind == 0 ? bbmd::scatter_rate<0>(nsm, s)
                            : kind == 1 ? bbmd::scatter_rate<1>(nsm, s) : bbmd::scatter_rate<2>(nsm, s);
    cudaFree(sink);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess && *adds_per_s > 0.0 ? BBMD_OK : BBMD_ERR_CUDA;
}

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
