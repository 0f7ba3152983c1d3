// Deterministic block and grid reductions in FP64.
//
// Each block reduces its threads' values with warp shuffles and shared
// memory in a fixed tree, writes one partial, and takes a ticket; the block
// that draws the last ticket sums all partials in a fixed order.  The result
// therefore does not depend on block scheduling.
#pragma once
#include "common.cuh"

namespace stag {

template <int BLOCK> STAG_D double block_sum(double v, double *smem) {
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        smem[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < BLOCK / 32 ? smem[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;  // valid in thread 0
}

// Grid-wide sum.  Every thread of every block must call it.  Returns true in
// all threads of the one block that finishes last; there `total` holds the
// grid sum (in every thread).  `ticket` must be zero on entry and is reset to
// zero by the last block.
template <int BLOCK>
STAG_D bool grid_sum(double v, double *partial, unsigned *ticket, double *smem, double &total) {
    __shared__ bool last;
    double s = block_sum<BLOCK>(v, smem);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s;
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last)
        return false;
    __threadfence();
    double acc = 0.0;
    const volatile double *vp = partial;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += BLOCK)
        acc += vp[i];
    acc = block_sum<BLOCK>(acc, smem);
    if (threadIdx.x == 0) {
        smem[0] = acc;
        *ticket = 0u;
    }
    __syncthreads();
    total = smem[0];
    __syncthreads();
    return true;
}

// Grid-wide sum of two values per thread (same protocol as grid_sum;
// partial must hold 2 * gridDim.x doubles).
template <int BLOCK>
STAG_D bool grid_sum2(double v0, double v1, double *partial, unsigned *ticket, double *smem,
                      double &t0, double &t1) {
    __shared__ bool last;
    const double s0 = block_sum<BLOCK>(v0, smem);
    const double s1 = block_sum<BLOCK>(v1, smem);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s0;
        partial[2 * blockIdx.x + 1] = s1;
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last)
        return false;
    __threadfence();
    const volatile double *vp = partial;
    double a0 = 0.0, a1 = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += BLOCK) {
        a0 += vp[2 * i];
        a1 += vp[2 * i + 1];
    }
    a0 = block_sum<BLOCK>(a0, smem);
    a1 = block_sum<BLOCK>(a1, smem);
    __shared__ double res[2];
    if (threadIdx.x == 0) {
        res[0] = a0;
        res[1] = a1;
        *ticket = 0u;
    }
    __syncthreads();
    t0 = res[0];
    t1 = res[1];
    __syncthreads();
    return true;
}

}  // namespace stag
