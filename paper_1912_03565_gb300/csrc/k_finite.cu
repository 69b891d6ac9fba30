// hs_check_finite: the number of NaN or infinite values in a device array of
// FP64 or FP32 values (a right-hand side, face data or a result), by one
// grid-stride pass, warp sums and one atomic per warp that met such a value.
// Input validation only (the paper assumes finite data): hs_solve runs it on f
// in its synchronous (hs_info) mode and returns HS_ERR_NONFINITE instead of a
// NaN field.  The count lives in the plan's reduction scratch (d_red[62]), so a
// check is ordered with the plan's other work on the same stream.
#include "hs_internal.cuh"

namespace {

template <typename T>
__device__ __forceinline__ bool bad(T v) {
    return !isfinite(v);
}

template <typename T>
__global__ void __launch_bounds__(256) nonfinite_kernel(const T *__restrict__ x, size_t n,
                                                        unsigned long long *count) {
    unsigned c = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        c += bad(x[i]) ? 1u : 0u;
    // warp sums, then one atomic per warp that saw something (rare)
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

}  // namespace

// Enqueues the count of non-finite values of x[0..n) into *dcount (device, not
// cleared here) on stream s.
hs_status hs_launch_nonfinite(const void *x, int dtype, size_t n, unsigned long long *dcount,
                              cudaStream_t s) {
    if (n == 0) return HS_OK;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    const size_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < (size_t)sms * 8 ? want : (size_t)sms * 8);
    if (dtype == HS_F64)
        nonfinite_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double *>(x), n, dcount);
    else if (dtype == HS_F32)
        nonfinite_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(x), n, dcount);
    else
        return HS_ERR_INVALID_ARG;
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

extern "C" hs_status hs_check_finite(hs_plan_t P, const void *data, int dtype, size_t n,
                                     void *stream, unsigned long long *count) {
    if (!P || !count || (n > 0 && !data) || (dtype != HS_F64 && dtype != HS_F32))
        return HS_ERR_INVALID_ARG;
    if (n > 0 && !hs_is_device_ptr(data)) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *dc = reinterpret_cast<unsigned long long *>(P->d_red + 62);
    if (cudaMemsetAsync(dc, 0, sizeof(*dc), s) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    const hs_status st = hs_launch_nonfinite(data, dtype, n, dc, s);
    if (st != HS_OK) return st;
    if (cudaMemcpyAsync(count, dc, sizeof(*count), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    return HS_OK;
}
