// Measured arithmetic peaks for the roofline of the Legendre kernels: FP32
// and FP64 fused multiply-add throughput of this GPU at its current clocks.
// Each thread runs NCH independent FMA chains (enough to hide the pipe
// latency) for a fixed trip count; the grid fills every SM with several
// CTAs.  The result is stored so that the compiler keeps every chain.
#include <chrono>

#include "common.cuh"

namespace shtg {
namespace {

constexpr int NCH = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T a, T b) {
    T x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) x[c] = x[c] * a + b;
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(int iters, int *sms, double *tflops, cudaStream_t st) {
    int dev = 0;
    SHTG_CUDA(cudaGetDevice(&dev));
    int nsm = 0, per_sm = 0;
    SHTG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SHTG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, 256, 0));
    const int blocks = nsm * (per_sm > 0 ? per_sm : 1);
    T *out = nullptr;
    SHTG_CUDA(cudaMallocAsync((void **)&out, sizeof(T) * (size_t)blocks * 256, st));
    cudaEvent_t e0, e1;
    SHTG_CUDA(cudaEventCreate(&e0));
    SHTG_CUDA(cudaEventCreate(&e1));
    // warm-up launch, then the timed one
    k_fma_probe<T><<<blocks, 256, 0, st>>>(out, iters / 4 + 1, T(0.999999), T(1e-7));
    SHTG_CUDA(cudaEventRecord(e0, st));
    k_fma_probe<T><<<blocks, 256, 0, st>>>(out, iters, T(0.999999), T(1e-7));
    SHTG_CUDA(cudaEventRecord(e1, st));
    SHTG_CHECK_LAUNCH("k_fma_probe");
    SHTG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SHTG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SHTG_CUDA(cudaFreeAsync(out, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    const double flops = 2.0 * NCH * 16.0 * iters * (double)blocks * 256.0;
    *sms = nsm;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return SHTG_OK;
}

}  // namespace
}  // namespace shtg

using namespace shtg;

extern "C" int shtg_probe_fma_peak(int precision, int *sm_count, double *tflops, void *stream) {
    if ((precision != SHTG_FP32 && precision != SHTG_FP64) || !sm_count || !tflops) {
        set_error("probe: precision must be SHTG_FP32 or SHTG_FP64, outputs non-null");
        return SHTG_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // about 10-50 ms of work per launch at the GB300's FP32 / FP64 rates
    if (precision == SHTG_FP32) return probe<float>(16384, sm_count, tflops, st);
    return probe<double>(512, sm_count, tflops, st);
}
