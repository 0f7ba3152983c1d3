// Dslash kernels instantiated for precision P_F16.
#include "dslash_launch.cuh"

namespace stag {
template cudaError_t launch_dslash_p<P_F16>(int, const DslashArgs &, int, cudaStream_t);
}  // namespace stag
