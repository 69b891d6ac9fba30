// Persistent batch kernel (Section 3.6's solve per work item): register cap for 2 resident CTAs of 256 threads per
// SM, fused transform tiles.
#include "hs_batch.cuh"

namespace hs_batch {

__global__ void __launch_bounds__(256, 2) batch_kernel2f(BatchArgs A) {
    batch_body<true>(A);
}

const void *batch_kernel_v2f() { return reinterpret_cast<const void *>(&batch_kernel2f); }

}  // namespace hs_batch
