// Batched CG kernels instantiated for precision P_DF64.
#include "batched_kernels.cuh"

namespace stag {
template cudaError_t launch_batch_pbk<P_DF64, 128, 4>(int, const BatchArgs &, cudaStream_t);
template cudaError_t launch_batch_pbk<P_DF64, 256, 4>(int, const BatchArgs &, cudaStream_t);
}  // namespace stag
