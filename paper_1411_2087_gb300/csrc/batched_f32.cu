// Batched CG kernels instantiated for precision P_F32.
#include "batched_kernels.cuh"

namespace stag {
template cudaError_t launch_batch_pbk<P_F32, 128, 4>(int, const BatchArgs &, cudaStream_t);
template cudaError_t launch_batch_pbk<P_F32, 128, 8>(int, const BatchArgs &, cudaStream_t);
template cudaError_t launch_batch_pbk<P_F32, 256, 4>(int, const BatchArgs &, cudaStream_t);
template cudaError_t launch_batch_pbk<P_F32, 256, 8>(int, const BatchArgs &, cudaStream_t);
}  // namespace stag
