// Launcher template of the Dslash kernels; each precision is instantiated in
// its own translation unit (dslash_<prec>.cu) so that they compile in parallel.
#pragma once
#include "dslash.cuh"
#include "kernels.h"

namespace stag {

template <int P, int BLOCK, bool COMP>
static cudaError_t launch_p_b_c(int epi, const DslashArgs &a, cudaStream_t s) {
    const int n = a.cn ? a.cn : a.g.Vh;
    const int grid = (n + BLOCK - 1) / BLOCK;
    if (grid == 0)
        return cudaSuccess;
    if constexpr (P == P_F16 && COMP) {
        switch (epi) {
        case EPI_NONE: dslash_kernel_capped<P, EPI_NONE, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_M: dslash_kernel_capped<P, EPI_M, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_M_PAP: dslash_kernel_capped<P, EPI_M_PAP, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_RESID: dslash_kernel_capped<P, EPI_RESID, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_RESID_STORE: dslash_kernel_capped<P, EPI_RESID_STORE, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_M_PART: dslash_kernel_capped<P, EPI_M_PART, BLOCK><<<grid, BLOCK, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (epi) {
        case EPI_NONE: dslash_kernel<P, EPI_NONE, BLOCK, COMP><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_M: dslash_kernel<P, EPI_M, BLOCK, COMP><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_M_PAP: dslash_kernel<P, EPI_M_PAP, BLOCK, COMP><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_RESID: dslash_kernel<P, EPI_RESID, BLOCK, COMP><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_RESID_STORE: dslash_kernel<P, EPI_RESID_STORE, BLOCK, COMP><<<grid, BLOCK, 0, s>>>(a); break;
        case EPI_M_PART: dslash_kernel<P, EPI_M_PART, BLOCK, COMP><<<grid, BLOCK, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

// the 12-real layout exists for FP32 and 16-bit links only
template <int P, int BLOCK>
static cudaError_t launch_p_b(int epi, const DslashArgs &a, cudaStream_t s) {
    if constexpr (P == P_F32 || P == P_F16) {
        if (a.compressed)
            return launch_p_b_c<P, BLOCK, true>(epi, a, s);
    } else {
        if (a.compressed)
            return cudaErrorInvalidValue;
    }
    return launch_p_b_c<P, BLOCK, false>(epi, a, s);
}

template <int P> cudaError_t launch_dslash_p(int epi, const DslashArgs &a, int block, cudaStream_t s) {
    switch (block) {
    case 128: return launch_p_b<P, 128>(epi, a, s);
    case 256: return launch_p_b<P, 256>(epi, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stag
