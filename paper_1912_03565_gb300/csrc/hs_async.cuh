// Asynchronous global -> shared copies (cp.async, sm_80 and later) used to keep
// several z-planes of a stencil tile in flight without holding them in
// registers.  A copy whose element lies outside the array is issued with a
// source size of 0, which writes zeros and reads nothing.
#pragma once

#include <cuda_runtime.h>

namespace hs_tiles {

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 4- or 8-byte copy through L1 (.ca); valid = false fills the destination with zeros
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool valid) {
    static_assert(BYTES == 4 || BYTES == 8, "cp.async.ca size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst)),
                 "l"(src), "n"(BYTES), "r"(valid ? BYTES : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// wait until at most N of this thread's committed groups are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace hs_tiles
