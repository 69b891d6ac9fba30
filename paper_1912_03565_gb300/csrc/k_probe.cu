// hs_fp64_fma_rate: the device's FP64 fused multiply-add throughput, measured.
// A diagnostic for the FP64-pipe roofline of the FP64 transforms (no paper
// counterpart): every thread runs CHAINS independent DFMA recurrences so the
// pipe never waits on a result, and the rate is timed with CUDA events.
#include "hs_internal.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int ITERS = 4096;

// written only when the (positive) chains sum below zero, which never happens:
// the store keeps the compiler from discarding the chains
__device__ double g_probe_sink;

__global__ void __launch_bounds__(256) dfma_kernel(double a, double b) {
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s < 0.0) g_probe_sink = s;
}

}  // namespace

extern "C" hs_status hs_fp64_fma_rate(void *stream, double *tflops) {
    if (!tflops) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    const unsigned blocks = (unsigned)sms * 8;   // 2048 threads per SM
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return HS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HS_ERR_CUDA;
    }
    // a = 1 - 2^-30 and b = 2^-40 keep the values positive, bounded and normal
    const double a = 1.0 - 0x1p-30, b = 0x1p-40;
    dfma_kernel<<<blocks, 256, 0, s>>>(a, b);   // warm-up
    cudaEventRecord(e0, s);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) dfma_kernel<<<blocks, 256, 0, s>>>(a, b);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || cudaGetLastError() != cudaSuccess) return HS_ERR_CUDA;
    const double flops = 2.0 * CHAINS * ITERS * 256.0 * blocks * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return HS_OK;
}
