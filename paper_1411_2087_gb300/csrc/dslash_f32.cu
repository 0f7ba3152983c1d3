// Dslash kernels instantiated for precision P_F32.
#include "dslash_launch.cuh"

namespace stag {
template cudaError_t launch_dslash_p<P_F32>(int, const DslashArgs &, int, cudaStream_t);
}  // namespace stag
