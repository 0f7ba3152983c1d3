// Launcher template of the Dslash kernels; each precision is instantiated in
// its own translation unit (dslash_<prec>.cu) so that they compile in parallel.
#pragma once
#include "dslash.cuh"
#include "kernels.h"

namespace stag {

// Which kernels run under the register cap by default (before tuning), by
// measurement (48^3x96, kernel times inside the mixed solves).  Left free,
// the compiler gives these 32-44 registers and keeps too few stencil loads
// in flight:
//   FP32 uncompressed          D_oe 947 -> 901 us, M with partials 954 -> 913 us
//   16-bit, one site           M with <p, Mp> partials 635 -> 557 us (full links)
// FP32 on 12-real links (56-62 registers free) and the FP64 and double-float
// kernels (HBM-bound at their free choice) keep the compiler's choice.
template <int P, int EPI, int CM>
constexpr bool kCapped = P == P_F16 || (P == P_F32 && CM != 3);

// The plain stencil and the M stencil with <p, Mp> partials (the solvers'
// two kernels per iteration) are instantiated in both register variants, so
// that the autotuner can time them; the other epilogues use the default.
template <int P, int EPI, int BLOCK, int CM>
static void launch_one(int grid, const DslashArgs &a, cudaStream_t s) {
    constexpr bool tunable = EPI == EPI_NONE || EPI == EPI_M_PART;
    const bool capped = tunable && a.regs != REGS_DEFAULT && a.regs != REGS_PAIR ? a.regs == REGS_CAPPED
                                                                                 : kCapped<P, EPI, CM>;
    if constexpr (tunable) {
        if (capped)
            dslash_kernel_capped<P, EPI, BLOCK, CM><<<grid, BLOCK, 0, s>>>(a);
        else
            dslash_kernel<P, EPI, BLOCK, CM><<<grid, BLOCK, 0, s>>>(a);
    } else if constexpr (kCapped<P, EPI, CM>) {
        dslash_kernel_capped<P, EPI, BLOCK, CM><<<grid, BLOCK, 0, s>>>(a);
    } else {
        dslash_kernel<P, EPI, BLOCK, CM><<<grid, BLOCK, 0, s>>>(a);
    }
}

template <int P, int BLOCK, int CM>
static cudaError_t launch_p_b_c(int epi, const DslashArgs &a, cudaStream_t s) {
    if constexpr (P == P_F16 && pair16_ring<BLOCK, CM>() > 0) {
        if (pair16_used(P, epi, a)) {
            const int grid = dslash_pair16_grid(a.g, BLOCK);
            if (epi == EPI_NONE)
                dslash_pair16_kernel<EPI_NONE, BLOCK, CM><<<grid, BLOCK, 0, s>>>(a);
            else
                dslash_pair16_kernel<EPI_M_PART, BLOCK, CM><<<grid, BLOCK, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    const int n = (a.cn ? a.cn : a.g.Vh) + (a.cn ? a.cnb : 0);
    const int grid = (n + BLOCK - 1) / BLOCK;
    if (grid == 0)
        return cudaSuccess;
    switch (epi) {
    case EPI_NONE: launch_one<P, EPI_NONE, BLOCK, CM>(grid, a, s); break;
    case EPI_M: launch_one<P, EPI_M, BLOCK, CM>(grid, a, s); break;
    case EPI_M_PAP: launch_one<P, EPI_M_PAP, BLOCK, CM>(grid, a, s); break;
    case EPI_RESID: launch_one<P, EPI_RESID, BLOCK, CM>(grid, a, s); break;
    case EPI_RESID_STORE: launch_one<P, EPI_RESID_STORE, BLOCK, CM>(grid, a, s); break;
    case EPI_M_PART: launch_one<P, EPI_M_PART, BLOCK, CM>(grid, a, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// the 12-real layout exists for FP32 and 16-bit links only: every link
// 12-real (mask 3), or the three-link ones only (mask 2)
template <int P, int BLOCK>
static cudaError_t launch_p_b(int epi, const DslashArgs &a, cudaStream_t s) {
    if constexpr (P == P_F32 || P == P_F16) {
        switch (a.compressed) {
        case 0: return launch_p_b_c<P, BLOCK, 0>(epi, a, s);
        case 2: return launch_p_b_c<P, BLOCK, 2>(epi, a, s);
        case 3: return launch_p_b_c<P, BLOCK, 3>(epi, a, s);
        default: return cudaErrorInvalidValue;
        }
    } else {
        if (a.compressed)
            return cudaErrorInvalidValue;
        return launch_p_b_c<P, BLOCK, 0>(epi, a, s);
    }
}

template <int P> cudaError_t launch_dslash_p(int epi, const DslashArgs &a, int block, cudaStream_t s) {
    switch (block) {
    case 64: return launch_p_b<P, 64>(epi, a, s);
    case 128: return launch_p_b<P, 128>(epi, a, s);
    case 256: return launch_p_b<P, 256>(epi, a, s);
    case 512: return launch_p_b<P, 512>(epi, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stag
