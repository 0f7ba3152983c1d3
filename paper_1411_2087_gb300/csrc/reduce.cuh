// Deterministic block and grid reductions.
//
// Each block reduces its threads' values with warp shuffles and shared
// memory in a fixed tree, writes one FP64 partial, and takes a ticket; the
// block that draws the last ticket sums all partials in a fixed order.  The
// result therefore does not depend on block scheduling.
//
// Inside a block the tree runs in the thread values' reduction type: FP64
// for the FP64 path, double-float (about 48 bits, FP32 pipe) for the others.
// GB300's FP64 pipe runs at 1/64 of the FP32 rate, and an FP64 shuffle tree
// in every thread of a 5M-site reduction costs tens of microseconds; in
// double-float it costs a few, and only thread 0 of each block converts its
// result to FP64.
#pragma once
#include "common.cuh"

namespace stag {

// reduction type of per-thread values computed in arithmetic type R
template <class R> struct RedType { using type = df; };
template <> struct RedType<double> { using type = double; };
template <class R> using red_t = typename RedType<R>::type;

template <class T> STAG_D T red_zero();
template <> STAG_D double red_zero<double>() { return 0.0; }
template <> STAG_D df red_zero<df>() { return df_zero(); }

STAG_D double red_add(double a, double b) { return a + b; }
STAG_D df red_add(df a, df b) { return df_add(a, b); }
STAG_D double red_to_double(double a) { return a; }
STAG_D double red_to_double(df a) { return df_to_double(a); }

STAG_D double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
STAG_D df shfl_down(df v, int o) {
    return df_make(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}

// Sum over the block; the FP64 result is valid in thread 0 only (0 elsewhere).
// smem: 32 doubles of shared memory.
template <int BLOCK, class T> STAG_D double block_sum(T v, double *smem) {
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
    static_assert(sizeof(T) <= sizeof(double), "reduction type");
    T *ts = reinterpret_cast<T *>(smem);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = red_add(v, shfl_down(v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        ts[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < BLOCK / 32 ? ts[lane] : red_zero<T>();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = red_add(v, shfl_down(v, o));
    }
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        r = red_to_double(v);
    return r;
}

// Grid-wide sum.  Every thread of every block must call it.  Returns true in
// all threads of the one block that finishes last; there `total` holds the
// grid sum (in every thread).  `ticket` must be zero on entry and is reset to
// zero by the last block.
template <int BLOCK, class T>
STAG_D bool grid_sum(T v, double *partial, unsigned *ticket, double *smem, double &total) {
    __shared__ bool last;
    const double s = block_sum<BLOCK>(v, smem);
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
template <int BLOCK, class T>
STAG_D bool grid_sum2(T v0, T v1, double *partial, unsigned *ticket, double *smem,
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
