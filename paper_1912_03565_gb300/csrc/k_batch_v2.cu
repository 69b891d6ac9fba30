// Persistent batch kernel (Section 3.6's solve per work item): register cap for 2 resident CTAs of 256 threads per
// SM, staged transform tiles.
#include "hs_batch.cuh"

namespace hs_batch {

__global__ void __launch_bounds__(256, 2) batch_kernel2(BatchArgs A) {
    batch_body<false>(A);
}

const void *batch_kernel_v2() { return reinterpret_cast<const void *>(&batch_kernel2); }

}  // namespace hs_batch
