// Internal declarations shared by the host-side translation units of
// libstag (stag_api.cu, solvers.cu, learned.cu): handle structs, error
// reporting, argument helpers.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/stag.h"
#include "batched.cuh"
#include "dslash.cuh"
#include "kernels.h"

using namespace stag;

namespace stag {
// the calling thread's last error message (stag_last_error_message)
void set_error_message(const char *msg);
}  // namespace stag

static inline int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    stag::set_error_message(buf);
    return code;
}

#define CUDA_TRY(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? STAG_ERR_NOMEM : STAG_ERR_CUDA,  \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                         \
    } while (0)

// NVTX range named after a C-ABI call, so that profiler timelines show the
// library's calls (a no-op unless a profiling tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define STAG_NVTX(name) NvtxRange nvtx_range_(name)

#define STAG_TRY(call)           \
    do {                         \
        int s_ = (call);         \
        if (s_ != STAG_OK)       \
            return s_;           \
    } while (0)

// make `dev` current for the scope of one API call, then restore
struct DeviceGuard {
    int prev = -1;
    int err = 0;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
            err = 1;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

#define DEVICE_SCOPE(dev)                                                        \
    DeviceGuard guard_(dev);                                                     \
    if (guard_.err)                                                              \
        return fail(STAG_ERR_CUDA, "cannot make CUDA device %d current", (dev));

static inline bool prec_valid(int p) {
    return p == STAG_F64 || p == STAG_DF64 || p == STAG_F32 || p == STAG_F16;
}
static inline const char *prec_name(int p) {
    switch (p) {
    case STAG_F64: return "F64";
    case STAG_DF64: return "DF64";
    case STAG_F32: return "F32";
    case STAG_F16: return "F16";
    default: return "?";
    }
}

// --------------------------------------------------------------------------
// handles
// --------------------------------------------------------------------------
struct CgWork {
    int prec = -1;
    void *r = nullptr, *p = nullptr, *Ap = nullptr, *t = nullptr, *bw = nullptr, *xw = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle cond = 0;
};

struct stag_lattice_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int dims[4];
    double bc[4];
    long long V = 0, Vh = 0;
    Geom geom;
    void *links[4] = {nullptr, nullptr, nullptr, nullptr};  // per precision [2][8][9][stride]
    void *links_c12[4] = {nullptr, nullptr, nullptr, nullptr};  // copies with 12-real kinds (FP32, 16-bit)
    int c12_mask[4] = {0, 0, 0, 0};  // their compression masks (link_kind_offset): 3 all, 2 three-link only
    bool has_gauge = false;
    double c1 = 0, c3 = 0;
    int live_fields = 0;
    // reduction scratch and scalars
    double *partial = nullptr;
    CgScalars *sc = nullptr;
    CgScalars *sc_host = nullptr;  // pinned mirror
    CgWork cg[4];
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double *staging = nullptr;             // canonical [Vh][3] complex128 for host import/export
    float link_scale[2] = {0.f, 0.f};      // 16-bit links: field max / 32767 (one-link, three-link)
    float *xs = nullptr;                   // F32 correction x_sloppy of the mixed solver
    unsigned *absmax = nullptr;            // scratch for the 16-bit link scales
    struct MixedGraph {
        cudaGraphExec_t exec = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphConditionalHandle cond = 0;      // WHILE: the iteration loop
        cudaGraphConditionalHandle rel_cond = 0;  // IF: the reliable update
    } mixed[4][4];
    // multi-shift CG
    ShiftState *ms_state = nullptr;        // device, MS_MAX entries
    cudaGraphConditionalHandle ms_rel_cond = 0;  // mixed multi-shift graph: the reliable-update branch
    ShiftState *ms_state_host = nullptr;   // pinned mirror
    double *ms_true = nullptr;             // device, |b - (M + sigma_s) x_s|^2 per shift
    double *ms_true_host = nullptr;        // pinned mirror
    void *ms_p[4][MS_MAX] = {};            // search directions per precision
    void *ms_xlo[MS_MAX] = {};             // FP32 solutions of the sloppy multi-shift phase
    void *ms_blo = nullptr;                // FP32 right-hand side of that phase
    void *ms_rhi[4] = {};                  // residual of one shift (high precision)
    void *ms_ehi[4] = {};                  // correction of one shift (high precision)
    // batched CG: per-system work vectors (r, p, Ap, t) by precision and slot
    void *bwork[4][BATCH_MAX_G * BATCH_KMAX][4] = {};
    void *bxlo[BATCH_MAX_G * BATCH_KMAX] = {};  // FP32 solutions of the sloppy batched phase
    void *bblo[BATCH_MAX_G * BATCH_KMAX] = {};  // FP32 right-hand sides of that phase
    int batch_block[4] = {128, 128, 128, 128};  // block size of the batched kernels (autotuned)
    int batch_k[4] = {0, 0, 0, 0};              // right-hand sides per batched group (0 = the largest)
    int dslash_block[4] = {0, 0, 0, 0};         // block size of the Dslash kernels (0 = default)
    int dslash_regs[4] = {0, 0, 0, 0};          // its register variant (REGS_*)
    int mdslash_block[4] = {0, 0, 0, 0};        // block size of the M Dslash with <p, Mp> partials (0 = as above)
    int mdslash_regs[4] = {0, 0, 0, 0};         // its register variant
    int cg_launch = STAG_CG_LAUNCH_GRAPH;  // how stag_cg_solve drives its iterations
    int cg_chunk = 32;                     // iterations between status polls (host mode)
};

struct stag_field_s {
    stag_lattice lat = nullptr;
    int parity = 0;
    int prec = 0;
    void *data = nullptr;
    size_t bytes = 0;
    bool owned = true;   // false: a view of caller memory (stag_field_wrap)
};

// lattice geometry of the kernels (dims even and >= 2; stride >= V/2)
static inline Geom geom_of(const int dims[4], long long stride) {
    Geom g;
    for (int k = 0; k < 4; k++)
        g.L[k] = dims[k];
    g.Lxh = dims[0] / 2;
    g.Vh = (int)((long long)dims[0] * dims[1] * dims[2] * dims[3] / 2);
    g.stride = (int)stride;
    g.plane[0] = 0;
    g.plane[1] = dims[0] / 2;
    g.plane[2] = dims[0] * dims[1] / 2;
    g.plane[3] = dims[0] * dims[1] * dims[2] / 2;
    geom_set_div(g);
    return g;
}

static inline size_t field_bytes(const stag_lattice lat, int prec) {
    return prec_vec_bytes(prec, (size_t)lat->geom.stride);
}
static inline size_t link_bytes(const stag_lattice lat, int prec) {
    return 2ull * 8 * 9 * lat->geom.stride * prec_link_elem_bytes(prec);
}
static inline const void *links_of(const stag_lattice lat, int prec, int parity) {
    const char *base = (const char *)lat->links[prec];
    return base + (size_t)parity * 8 * 9 * lat->geom.stride * prec_link_elem_bytes(prec);
}

static inline void free_cg(CgWork &w) {
    if (w.exec)
        cudaGraphExecDestroy(w.exec);
    if (w.graph)
        cudaGraphDestroy(w.graph);
    void *bufs[] = {w.r, w.p, w.Ap, w.t, w.bw, w.xw};
    for (void *b : bufs)
        if (b)
            cudaFree(b);
    w = CgWork();
}

static inline void drop_mixed_graphs(stag_lattice lat) {
    for (int h = 0; h < 4; h++)
        for (int l = 0; l < 4; l++) {
            auto &m = lat->mixed[h][l];
            if (m.exec)
                cudaGraphExecDestroy(m.exec);
            if (m.graph)
                cudaGraphDestroy(m.graph);
            m = stag_lattice_s::MixedGraph();
        }
}

static inline DslashArgs dslash_args(stag_lattice lat, int prec, int out_par, const void *in, void *out) {
    DslashArgs a;
    memset(&a, 0, sizeof a);
    a.g = lat->geom;
    a.out_par = out_par;
    a.links_out = links_of(lat, prec, out_par);
    a.links_in = links_of(lat, prec, 1 - out_par);
    a.in = in;
    a.out = out;
    a.partial = lat->partial;
    a.sc = lat->sc;
    a.regs = lat->dslash_regs[prec];
    if (prec == STAG_F16) {
        a.link_scale[0] = lat->link_scale[0];
        a.link_scale[1] = lat->link_scale[1];
    }
    if (lat->links_c12[prec]) {
        // the copy with 12-real kinds replaces the full one for this precision
        const size_t half = link_parity_bytes(prec, lat->c12_mask[prec], (size_t)lat->geom.stride);
        a.links_out = (const char *)lat->links_c12[prec] + (size_t)out_par * half;
        a.links_in = (const char *)lat->links_c12[prec] + (size_t)(1 - out_par) * half;
        a.compressed = lat->c12_mask[prec];
        a.inv_c[0] = (float)(1.0 / lat->c1);
        a.inv_c[1] = (float)(1.0 / lat->c3);
        for (int k = 0; k < 4; k++)
            a.bc_neg[k] = lat->bc[k] < 0 ? 1 : 0;
    }
    return a;
}

static inline int ensure_cg_work(stag_lattice lat, int prec) {
    CgWork &w = lat->cg[prec];
    if (w.r)
        return STAG_OK;
    w.prec = prec;
    const size_t b = field_bytes(lat, prec);
    void **bufs[] = {&w.r, &w.p, &w.Ap, &w.t, &w.bw, &w.xw};
    for (void **pp : bufs) {
        cudaError_t e = cudaMalloc(pp, b);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(*pp, 0, b, lat->stream);
        if (e != cudaSuccess) {
            free_cg(w);
            return fail(STAG_ERR_NOMEM, "CG workspace (%s): %s", prec_name(prec), cudaGetErrorString(e));
        }
    }
    return STAG_OK;
}

static inline int upload_scalars(stag_lattice lat, double mass, double tol, int max_iter, bool has_cond,
                          cudaGraphConditionalHandle cond, double delta = 0.0,
                          bool has_rel_cond = false, cudaGraphConditionalHandle rel_cond = 0) {
    // pageable source: the copy has read it when cudaMemcpyAsync returns
    CgScalars h;
    memset(&h, 0, sizeof h);
    h.m2 = make_dpair(mass * mass);
    h.tol2 = tol * tol;
    h.max_iter = max_iter;
    h.has_cond = has_cond ? 1 : 0;
    h.cond = cond;
    h.delta = delta;
    h.has_rel_cond = has_rel_cond ? 1 : 0;
    h.rel_cond = rel_cond;
    CUDA_TRY(cudaMemcpyAsync(lat->sc, &h, sizeof h, cudaMemcpyHostToDevice, lat->stream));
    return STAG_OK;
}

static inline int alloc_vec(stag_lattice lat, int prec, void **p) {
    if (*p)
        return STAG_OK;
    const size_t b = field_bytes(lat, prec);
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, b);
    if (e == cudaSuccess) {
        e = cudaMemsetAsync(q, 0, b, lat->stream);
        if (e != cudaSuccess)
            cudaFree(q);
    }
    if (e != cudaSuccess)
        return fail(STAG_ERR_NOMEM, "vector allocation (%s): %s", prec_name(prec), cudaGetErrorString(e));
    *p = q;
    return STAG_OK;
}


// block size of the M Dslash that writes <p, Mp> partials (EPI_M_PART)
static inline int m_block(const stag_lattice lat, int prec) {
    if (lat->mdslash_block[prec] > 0)
        return lat->mdslash_block[prec];
    return lat->dslash_block[prec] > 0 ? lat->dslash_block[prec] : dslash_default_block(prec);
}

// lattices up to this many sites per parity sum <p, Ap> in the M Dslash's
// last block (one launch less per iteration, which is what counts when the
// launches are short); larger ones write block partials and sum them in a
// one-block kernel, which lets the Dslash blocks retire without a ticket
constexpr int kSmallVh = 65536;

// Ap = m^2 p - D_eo t with <p, Ap>, alpha and the breakdown test in sc
// (skip_if_done: everything returns at once after the solve)
static inline cudaError_t enqueue_m_pap(stag_lattice lat, int prec, const void *t, void *Ap, const void *p,
                                        bool skip_if_done, cudaStream_t s, const int *gate = nullptr) {
    DslashArgs a = dslash_args(lat, prec, STAG_EVEN, t, Ap);
    a.p = p;
    a.skip_if_done = skip_if_done;
    a.gate = gate;
    a.regs = lat->mdslash_block[prec] > 0 ? lat->mdslash_regs[prec] : lat->dslash_regs[prec];
    const int block = m_block(lat, prec);
    if (lat->geom.Vh <= kSmallVh)
        return launch_dslash(prec, EPI_M_PAP, a, block, s);
    cudaError_t e = launch_dslash(prec, EPI_M_PART, a, block, s);
    if (e != cudaSuccess)
        return e;
    const int n = pair16_used(prec, EPI_M_PART, a) ? dslash_pair16_grid(lat->geom, block) : dslash_grid(lat->geom, block);
    return launch_pap_finish(lat->partial, n, lat->sc, skip_if_done, s, gate);
}

// Source normalisation (stag_api.cu): when the exponent k of b's largest
// entry is far from 0 (double-float and FP32 fields), `scaled` is a copy
// b 2^-k to solve with, and rhs_scale_end multiplies the n solutions by 2^k
// and frees it (call it on every path once begin succeeded).
struct RhsScale {
    int k = 0;
    stag_field scaled = nullptr;
};
int rhs_scale_begin(const stag_field b, RhsScale *rs);
int rhs_scale_end(RhsScale *rs, stag_field const *xs, int n);

// one plain CG iteration on the lattice stream (stag_api.cu)
cudaError_t enqueue_cg_body(stag_lattice lat, CgWork &w, cudaStream_t s, bool skip_if_done);

// A flexible preconditioner inside the mixed solver (learned.cu): enqueue
// z = N(r_s) in the low precision with the block partials of Re<z, r_s> and
// Re<z, Ap> (Ap NULL on the first call), then beta and rr = <r_s, z> into the
// scalars (first: beta = 0).  Kernels return at once unless the solve runs.
struct MixedPrecond {
    cudaError_t (*enqueue)(void *ctx, int lo, const void *rs, void *z, const void *Ap, int first, cudaStream_t s);
    void *ctx = nullptr;
    void *z = nullptr;  // low-precision buffer for z
};

// shared between the solver translation units
int mixed_solve_raw(stag_lattice lat, int hi, int lo, void *x_data, const void *b_data, size_t bytes,
                    double mass, double rel_tol, int max_iter, double delta, stag_solve_info *info,
                    const MixedPrecond *pc = nullptr);
int shifted_residual(stag_lattice lat, int hi, const void *x, const void *b, double mk, void *r_out,
                     double *rr);
