// Dispatch of the Dslash launchers over precisions.
#include "dslash.cuh"
#include "kernels.h"

namespace stag {

template <int P> cudaError_t launch_dslash_p(int epi, const DslashArgs &a, int block, cudaStream_t s);
extern template cudaError_t launch_dslash_p<P_F64>(int, const DslashArgs &, int, cudaStream_t);
extern template cudaError_t launch_dslash_p<P_DF64>(int, const DslashArgs &, int, cudaStream_t);
extern template cudaError_t launch_dslash_p<P_F32>(int, const DslashArgs &, int, cudaStream_t);
extern template cudaError_t launch_dslash_p<P_F16>(int, const DslashArgs &, int, cudaStream_t);

int dslash_default_block(int prec) {
    (void)prec;
    return 128;
}

int dslash_grid(const Geom &g, int block) { return (g.Vh + block - 1) / block; }

cudaError_t launch_dslash(int prec, int epi, const DslashArgs &a, int block, cudaStream_t s) {
    if (block <= 0)
        block = dslash_default_block(prec);
    switch (prec) {
    case P_F64: return launch_dslash_p<P_F64>(epi, a, block, s);
    case P_DF64: return launch_dslash_p<P_DF64>(epi, a, block, s);
    case P_F32: return launch_dslash_p<P_F32>(epi, a, block, s);
    case P_F16: return launch_dslash_p<P_F16>(epi, a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stag
