// Instantiations and launcher of the Dslash kernels.
#include "dslash.cuh"
#include "kernels.h"

namespace stag {

int dslash_default_block(int prec) {
    (void)prec;
    return 128;
}

int dslash_grid(const Geom &g, int block) { return (g.Vh + block - 1) / block; }

template <int P, int BLOCK>
static cudaError_t launch_p_b(int epi, const DslashArgs &a, cudaStream_t s) {
    const int grid = dslash_grid(a.g, BLOCK);
    if (grid == 0)
        return cudaSuccess;
    switch (epi) {
    case EPI_NONE: dslash_kernel<P, EPI_NONE, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
    case EPI_M: dslash_kernel<P, EPI_M, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
    case EPI_M_PAP: dslash_kernel<P, EPI_M_PAP, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
    case EPI_RESID: dslash_kernel<P, EPI_RESID, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int P>
static cudaError_t launch_p(int epi, const DslashArgs &a, int block, cudaStream_t s) {
    switch (block) {
    case 64: return launch_p_b<P, 64>(epi, a, s);
    case 128: return launch_p_b<P, 128>(epi, a, s);
    case 256: return launch_p_b<P, 256>(epi, a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dslash(int prec, int epi, const DslashArgs &a, int block, cudaStream_t s) {
    if (block <= 0)
        block = dslash_default_block(prec);
    switch (prec) {
    case P_F64: return launch_p<P_F64>(epi, a, block, s);
    case P_DF64: return launch_p<P_DF64>(epi, a, block, s);
    case P_F32: return launch_p<P_F32>(epi, a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stag
