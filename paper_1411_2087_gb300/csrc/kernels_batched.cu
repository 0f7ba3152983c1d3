// Dispatch of the batched CG kernels over precision, block size and group
// size (the kernels are in batched_kernels.cuh, instantiated in
// batched_<prec>.cu so that the precisions compile in parallel).
#include "batched.cuh"
#include "kernels.h"

namespace stag {

template <int P, int BLOCK, int K> cudaError_t launch_batch_pbk(int what, const BatchArgs &a, cudaStream_t s);
#define STAG_BATCH_EXTERN(P, B, K) \
    extern template cudaError_t launch_batch_pbk<P, B, K>(int, const BatchArgs &, cudaStream_t);
STAG_BATCH_EXTERN(P_F32, 128, 4)
STAG_BATCH_EXTERN(P_F32, 128, 8)
STAG_BATCH_EXTERN(P_F32, 256, 4)
STAG_BATCH_EXTERN(P_F32, 256, 8)
STAG_BATCH_EXTERN(P_DF64, 128, 4)
STAG_BATCH_EXTERN(P_DF64, 256, 4)
STAG_BATCH_EXTERN(P_F64, 128, 4)
STAG_BATCH_EXTERN(P_F64, 256, 4)
#undef STAG_BATCH_EXTERN

// right-hand sides per group: FP32 keeps K vectors per thread (kernels for
// K = 4 and 8), double float and FP64 map one thread to one (site, system)
// pair (K = 2 or 4 lanes share a link load; one kernel serves both)
int batch_max_k(int prec) { return prec == P_F32 ? 8 : 4; }
int batch_min_k(int prec) { return prec == P_F32 ? 4 : 2; }

cudaError_t launch_batch(int prec, int what, const BatchArgs &a, int block, cudaStream_t s) {
    if (block != 128 && block != 256)
        return cudaErrorInvalidValue;
    const bool b128 = block == 128;
    switch (prec) {
    case P_F32:
        if (a.kmax <= 4)
            return b128 ? launch_batch_pbk<P_F32, 128, 4>(what, a, s) : launch_batch_pbk<P_F32, 256, 4>(what, a, s);
        return b128 ? launch_batch_pbk<P_F32, 128, 8>(what, a, s) : launch_batch_pbk<P_F32, 256, 8>(what, a, s);
    case P_DF64:
        return b128 ? launch_batch_pbk<P_DF64, 128, 4>(what, a, s) : launch_batch_pbk<P_DF64, 256, 4>(what, a, s);
    case P_F64:
        return b128 ? launch_batch_pbk<P_F64, 128, 4>(what, a, s) : launch_batch_pbk<P_F64, 256, 4>(what, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stag
