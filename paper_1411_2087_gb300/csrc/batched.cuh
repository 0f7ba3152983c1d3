// Batched CG: many right-hand sides on one or several lattices iterate in
// lock step inside one graph.  Systems on the same lattice form a group that
// shares every link load: the multi-RHS Dslash streams each link matrix from
// HBM once and applies it to all K vectors of the group, so the link bytes
// per right-hand side drop by K.  In FP32 one thread holds a link and applies
// it to the K vectors.  In double-float and FP64 the arithmetic per site is
// K times that of a single Dslash and a thread holding K accumulators runs
// out of registers, so there one thread handles one (site, system) pair and
// the K lanes of a site load the same link in one coalesced request (the
// lane-mapped Dslash).  One grouped launch covers all groups
// (lattices of different sizes): block b belongs to the group whose block
// range contains it.  Each system keeps its own CG scalars and stops on its
// own; the loop ends when none is running.
#pragma once
#include "dslash.cuh"

namespace stag {

constexpr int BATCH_MAX_G = 8;   // groups (lattice, up to K right-hand sides)
constexpr int BATCH_KMAX = 8;    // right-hand sides per group

struct BatchGroup {
    Geom g;
    int K;            // right-hand sides in this group
    int block0;       // first block of this group in the grouped launch
    int nblocks;      // blocks of this group
    int sys0;         // index of the group's first system
    int dblock0;      // first block of this group in a lane-mapped Dslash launch
    int dnblocks;     // its blocks there: one thread per (site, system), K lanes per site
    const void *links[2];  // per parity [8][9][stride]
    float link_scale[2];
    void *x[BATCH_KMAX], *r[BATCH_KMAX], *p[BATCH_KMAX], *Ap[BATCH_KMAX], *t[BATCH_KMAX];
    const void *b[BATCH_KMAX];
    double *partial;  // this group's partial sums, [max(nblocks, dnblocks)][BATCH_KMAX]
};

struct BatchCtl {
    unsigned group_ticket;  // groups that finished their last block this kernel
    int running;            // systems still iterating
    cudaGraphConditionalHandle cond;
    int has_cond;
    int pad;
};

struct BatchArgs {
    int G;
    int kmax;     // the largest group: selects the kernels' K
    int nblocks;  // total blocks of the grouped launch
    int dnblocks; // total blocks of a lane-mapped Dslash launch
    BatchGroup grp[BATCH_MAX_G];
    CgScalars *sys;    // one per system
    unsigned *tickets; // one per group
    BatchCtl *ctl;
};

enum BatchKernel {
    BATCH_INIT = 0, BATCH_DSLASH_OE, BATCH_M_PAP, BATCH_UPDATE, BATCH_P, BATCH_DSLASH_X, BATCH_RESID
};

// the group that block `blk` belongs to
STAG_D int group_of(const BatchArgs &a, int blk) {
    int gi = 0;
#pragma unroll 1
    for (int k = 1; k < a.G; k++)
        if (blk >= a.grp[k].block0)
            gi = k;
    return gi;
}

// the same for a lane-mapped Dslash launch
STAG_D int group_of_lanes(const BatchArgs &a, int blk) {
    int gi = 0;
#pragma unroll 1
    for (int k = 1; k < a.G; k++)
        if (blk >= a.grp[k].dblock0)
            gi = k;
    return gi;
}

// Sum K values per thread over the blocks of one group.  Returns true in
// the group's last block; there tot[k] holds the sums (all threads).
template <int BLOCK, int K, class T>
STAG_D bool group_sum(const T (&v)[K], int Kact, double *partial, int lblk, int nblk, unsigned *ticket,
                      double *smem, double (&tot)[K]) {
    __shared__ bool last;
    __shared__ double res[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (k < Kact) {
            const double s = block_sum<BLOCK>(v[k], smem);
            if (threadIdx.x == 0)
                partial[(size_t)lblk * K + k] = s;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last)
        return false;
    __threadfence();
    const volatile double *vp = partial;
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (k < Kact) {
            double acc = 0.0;
            for (int i = threadIdx.x; i < nblk; i += BLOCK)
                acc += vp[(size_t)i * K + k];
            acc = block_sum<BLOCK>(acc, smem);
            if (threadIdx.x == 0)
                res[k] = acc;
        }
    }
    if (threadIdx.x == 0)
        *ticket = 0u;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++)
        tot[k] = k < Kact ? res[k] : 0.0;
    __syncthreads();
    return true;
}

// after a group's last block updated its systems: the last group to finish
// sets the loop condition from the count of running systems
STAG_D void batch_finish_group(const BatchArgs &a) {
    __threadfence();
    const unsigned t = atomicAdd(&a.ctl->group_ticket, 1u);
    if (t == (unsigned)a.G - 1) {
        __threadfence();
        a.ctl->group_ticket = 0u;
        const int running = atomicAdd(&a.ctl->running, 0);
        if (a.ctl->has_cond)
            cudaGraphSetConditional(a.ctl->cond, running > 0 ? 1u : 0u);
    }
}

}  // namespace stag
