// libstag solvers beyond the plain CG: mixed precision with reliable
// updates, multi-shift, batched multi-right-hand-side CG, and the block-size
// autotuner.  Documentation in include/stag.h.
#include "api_internal.h"

#include <algorithm>
#include <map>
#include <mutex>
#include <string>

// --------------------------------------------------------------------------
// mixed-precision CG with reliable updates (kernels_mixed.cu has the method)
// --------------------------------------------------------------------------
static const int *reliable_flag(stag_lattice lat) {
    return (const int *)((const char *)lat->sc + offsetof(CgScalars, reliable));
}

// the four kernels of a reliable update; each returns at once unless it is due
static cudaError_t enqueue_reliable_update(stag_lattice lat, int hi, int lo, cudaStream_t s) {
    CgWork &H = lat->cg[hi];
    CgWork &L = lat->cg[lo];
    const Geom &g = lat->geom;
    cudaError_t e;
    if ((e = launch_mixed_accum(hi, g, H.xw, lat->xs, lat->sc, s)) != cudaSuccess)
        return e;
    DslashArgs a3 = dslash_args(lat, hi, STAG_ODD, H.xw, H.t);
    a3.gate = reliable_flag(lat);
    if ((e = launch_dslash(hi, EPI_NONE, a3, lat->dslash_block[hi], s)) != cudaSuccess)
        return e;
    DslashArgs a4 = dslash_args(lat, hi, STAG_EVEN, H.t, H.r);
    a4.p = H.xw;
    a4.b = H.bw;
    a4.gate = reliable_flag(lat);
    if ((e = launch_dslash(hi, EPI_RESID_STORE, a4, lat->dslash_block[hi], s)) != cudaSuccess)
        return e;
    return launch_mixed_restart(hi, lo, g, H.r, L.r, lat->sc, s);
}

// One iteration.  Host mode: all kernels launched on the lattice stream.
// Graph capture (side != nullptr): the reliable update goes into a
// conditional IF node whose handle (*rel_cond, created on the loop-body
// graph) mixed_update sets, captured on the second stream `side`.
static cudaError_t enqueue_mixed_body(stag_lattice lat, int hi, int lo, bool host_mode, cudaStream_t side = nullptr,
                                      cudaGraphConditionalHandle *rel_cond = nullptr,
                                      const MixedPrecond *pc = nullptr) {
    CgWork &L = lat->cg[lo];
    cudaStream_t s = lat->stream;
    const Geom &g = lat->geom;
    cudaError_t e;
    // low precision: t_s = D_oe p; Ap = m^2 p - D_eo t_s, alpha
    DslashArgs a1 = dslash_args(lat, lo, STAG_ODD, L.p, L.t);
    a1.skip_if_done = host_mode;
    if ((e = launch_dslash(lo, EPI_NONE, a1, lat->dslash_block[lo], s)) != cudaSuccess)
        return e;
    if ((e = enqueue_m_pap(lat, lo, L.t, L.Ap, L.p, host_mode, s)) != cudaSuccess)
        return e;
    if ((e = launch_mixed_update(lo, g, lat->xs, L.r, L.p, L.Ap, lat->partial, lat->sc, s)) != cudaSuccess)
        return e;
    if (!side) {
        if ((e = enqueue_reliable_update(lat, hi, lo, s)) != cudaSuccess)
            return e;
    } else {
        cudaStreamCaptureStatus st;
        cudaGraph_t body = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        if ((e = cudaStreamGetCaptureInfo(s, &st, nullptr, &body, &deps, nullptr, &ndeps)) != cudaSuccess)
            return e;
        if ((e = cudaGraphConditionalHandleCreate(rel_cond, body, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
            return e;
        cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
        ip.conditional.handle = *rel_cond;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t branch;
        if ((e = cudaGraphAddNode(&branch, body, deps, nullptr, ndeps, &ip)) != cudaSuccess)
            return e;
        if ((e = cudaStreamUpdateCaptureDependencies(s, &branch, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamBeginCaptureToGraph(side, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return e;
        cudaError_t e2 = enqueue_reliable_update(lat, hi, lo, side);
        cudaGraph_t branch_out = nullptr;
        e = cudaStreamEndCapture(side, &branch_out);
        if (e2 != cudaSuccess)
            return e2;
        if (e != cudaSuccess)
            return e;
    }
    if (pc) {
        // flexible: z = N(r_s), beta, p = z + beta p
        if ((e = pc->enqueue(pc->ctx, lo, L.r, pc->z, L.Ap, 0, s)) != cudaSuccess)
            return e;
        return launch_cg_p_update(lo, g, pc->z, L.p, lat->sc, s);
    }
    return launch_cg_p_update(lo, g, L.r, L.p, lat->sc, s);
}

static cudaError_t enqueue_mixed_init(stag_lattice lat, int hi, int lo, const MixedPrecond *pc = nullptr) {
    CgWork &H = lat->cg[hi];
    CgWork &L = lat->cg[lo];
    cudaError_t e = launch_mixed_init(hi, lo, lat->geom, H.xw, H.r, H.bw, lat->xs, L.r, L.p, lat->partial,
                                      lat->sc, lat->stream);
    if (e != cudaSuccess || !pc)
        return e;
    // flexible: p = z = N(b), rr = <b, z>
    if ((e = pc->enqueue(pc->ctx, lo, L.r, pc->z, nullptr, 1, lat->stream)) != cudaSuccess)
        return e;
    return cudaMemcpyAsync(L.p, pc->z, field_bytes(lat, lo), cudaMemcpyDeviceToDevice, lat->stream);
}

// the mixed solver's graph: init, then WHILE(body) with the reliable update
// in an IF node.  Without a preconditioner it is kept per (hi, lo) on the
// lattice (mg); with one the caller runs and destroys it.
static int build_mixed_graph(stag_lattice lat, int hi, int lo, const MixedPrecond *pc = nullptr,
                             stag_lattice_s::MixedGraph *out = nullptr) {
    auto &mg = out ? *out : lat->mixed[hi][lo];
    cudaStream_t s = lat->stream;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 0, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(STAG_ERR_CUDA, "cudaGraphConditionalHandleCreate: %s", cudaGetErrorString(e));
    }
    auto bail = [&](const char *what, cudaError_t err) {
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(s, &junk);
        }
        cudaGetLastError();
        cudaGraphDestroy(graph);
        return fail(STAG_ERR_CUDA, "mixed CG graph (%s): %s", what, cudaGetErrorString(err));
    };
    if ((e = cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail("begin capture", e);
    if ((e = enqueue_mixed_init(lat, hi, lo, pc)) != cudaSuccess)
        return bail("init", e);
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if ((e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &ndeps)) != cudaSuccess)
        return bail("capture info", e);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((e = cudaGraphAddNode(&loop, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess)
        return bail("add loop node", e);
    if ((e = cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return bail("update deps", e);
    cudaGraph_t captured = nullptr;
    if ((e = cudaStreamEndCapture(s, &captured)) != cudaSuccess)
        return bail("end capture", e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t side = nullptr;
    if ((e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking)) != cudaSuccess)
        return bail("side stream", e);
    if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        cudaStreamDestroy(side);
        return bail("begin body capture", e);
    }
    cudaGraphConditionalHandle rel_cond = 0;
    e = enqueue_mixed_body(lat, hi, lo, false, side, &rel_cond, pc);
    cudaStreamDestroy(side);
    if (e != cudaSuccess)
        return bail("body", e);
    cudaGraph_t body_out = nullptr;
    if ((e = cudaStreamEndCapture(s, &body_out)) != cudaSuccess)
        return bail("end body capture", e);
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
        return bail("instantiate", e);
    mg.graph = graph;
    mg.exec = exec;
    mg.cond = cond;
    mg.rel_cond = rel_cond;
    return STAG_OK;
}

// the mixed solver on raw buffers of precision hi (x_data, b_data: bytes each);
// arguments already checked
int mixed_solve_raw(stag_lattice lat, int hi, int lo, void *x_data, const void *b_data,
                           size_t bytes, double mass, double rel_tol, int max_iter, double delta,
                           stag_solve_info *info, const MixedPrecond *pc) {
    STAG_TRY(ensure_cg_work(lat, hi));
    STAG_TRY(ensure_cg_work(lat, lo));
    if (!lat->xs) {
        // the init kernel of every solve zeroes x_s
        float *xs = nullptr;
        CUDA_TRY(cudaMalloc(&xs, prec_vec_bytes(STAG_F32, lat->geom.stride)));
        lat->xs = xs;
    }
    CgWork &H = lat->cg[hi];
    cudaStream_t s = lat->stream;
    CUDA_TRY(cudaMemcpyAsync(H.bw, b_data, bytes, cudaMemcpyDeviceToDevice, s));
    // flexible mode flag, after the scalars are uploaded (pageable source:
    // read when cudaMemcpyAsync returns)
    const int fcg_flag = pc ? 1 : 0;
    auto set_fcg = [&]() {
        return cudaMemcpyAsync((char *)lat->sc + offsetof(CgScalars, fcg), &fcg_flag, sizeof fcg_flag,
                               cudaMemcpyHostToDevice, s);
    };
    if (lat->cg_launch == STAG_CG_LAUNCH_GRAPH) {
        stag_lattice_s::MixedGraph once;
        auto &mg = pc ? once : lat->mixed[hi][lo];
        if (!mg.exec)
            STAG_TRY(build_mixed_graph(lat, hi, lo, pc, &mg));
        STAG_TRY(upload_scalars(lat, mass, rel_tol, max_iter, true, mg.cond, delta, true, mg.rel_cond));
        cudaError_t e = set_fcg();
        if (e == cudaSuccess)
            e = cudaEventRecord(lat->ev0, s);
        if (e == cudaSuccess)
            e = cudaGraphLaunch(mg.exec, s);
        if (e == cudaSuccess)
            e = cudaEventRecord(lat->ev1, s);
        if (pc) {
            cudaStreamSynchronize(s);
            cudaGraphExecDestroy(once.exec);
            cudaGraphDestroy(once.graph);
        }
        CUDA_TRY(e);
    } else {
        STAG_TRY(upload_scalars(lat, mass, rel_tol, max_iter, false, 0, delta));
        CUDA_TRY(set_fcg());
        CUDA_TRY(cudaEventRecord(lat->ev0, s));
        CUDA_TRY(enqueue_mixed_init(lat, hi, lo, pc));
        const int chunk = lat->cg_chunk;
        const long long max_chunks = (long long)max_iter / chunk + 2;
        for (long long k = 0; k < max_chunks; k++) {
            CUDA_TRY(cudaMemcpyAsync(&lat->sc_host->status, &lat->sc->status, sizeof(int),
                                     cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            if (lat->sc_host->status != CG_RUNNING)
                break;
            for (int j = 0; j < chunk; j++)
                CUDA_TRY(enqueue_mixed_body(lat, hi, lo, true, nullptr, nullptr, pc));
        }
        CUDA_TRY(cudaEventRecord(lat->ev1, s));
    }
    CUDA_TRY(cudaMemcpyAsync(x_data, H.xw, bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, lat->ev0, lat->ev1));
    const CgScalars &h = *lat->sc_host;
    stag_solve_info local;
    memset(&local, 0, sizeof local);
    local.iters = h.iter;
    local.restarts = h.restarts;
    local.status = h.status == CG_CONVERGED ? STAG_OK
                   : h.status == CG_BREAKDOWN ? STAG_ERR_BREAKDOWN
                                              : STAG_ERR_NOT_CONVERGED;
    local.true_rel_resid = h.bb > 0 ? std::sqrt(h.true_rr / h.bb) : 0.0;
    local.iter_rel_resid = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
    local.seconds = ms * 1e-3;
    // model: low-precision iterations plus one high-precision M per update
    const double lo_real = lo == STAG_F16 ? 2.0 : 4.0;
    const double Vh = (double)lat->Vh;
    const double model_bytes = h.iter * ((2.0 * 300 + 60) * lo_real + (lo == STAG_F16 ? 2 * 2 * 4 : 0) + 48) * Vh +
                         h.restarts * (2.0 * 2400 + 4 * 48) * Vh;
    const double flops = h.iter * (2.0 * 1146 + 72) * Vh + h.restarts * (2.0 * 1146 + 24) * Vh;
    if (ms > 0) {
        local.gflops = flops / (ms * 1e-3) / 1e9;
        local.gbs = model_bytes / (ms * 1e-3) / 1e9;
    }
    if (info)
        *info = local;
    if (local.status != STAG_OK)
        return fail(local.status, "stag_cg_solve_mixed: %s after %d iterations (true |r|/|b| = %.3e)",
                    local.status == STAG_ERR_BREAKDOWN ? "breakdown" : "not converged", local.iters,
                    local.true_rel_resid);
    return STAG_OK;
}

extern "C" int stag_cg_solve_mixed(stag_lattice lat, stag_field x, const stag_field b, double mass,
                                   double rel_tol, int max_iter, int inner_prec, double delta,
                                   stag_solve_info *info) {
    STAG_NVTX("stag_cg_solve_mixed");
    if (info)
        memset(info, 0, sizeof *info);
    if (!lat || !x || !b)
        return fail(STAG_ERR_ARG, "stag_cg_solve_mixed: NULL argument");
    if (x->lat != lat || b->lat != lat)
        return fail(STAG_ERR_ARG, "stag_cg_solve_mixed: field belongs to another lattice");
    if (x->parity != STAG_EVEN || b->parity != STAG_EVEN)
        return fail(STAG_ERR_STATE, "stag_cg_solve_mixed: x and b must be even fields");
    if (x->prec != b->prec || (x->prec != STAG_F64 && x->prec != STAG_DF64))
        return fail(STAG_ERR_STATE, "stag_cg_solve_mixed: x and b must both be F64 or both DF64");
    if (x == b)
        return fail(STAG_ERR_ARG, "stag_cg_solve_mixed: x and b must differ");
    if (inner_prec != STAG_F32 && inner_prec != STAG_F16)
        return fail(STAG_ERR_ARG, "stag_cg_solve_mixed: inner precision must be F32 or F16");
    if (!(mass > 0) || !std::isfinite(mass))
        return fail(STAG_ERR_ARG, "stag_cg_solve_mixed: mass must be positive and finite");
    if (!(rel_tol >= 0) || !std::isfinite(rel_tol))
        return fail(STAG_ERR_ARG, "stag_cg_solve_mixed: rel_tol must be >= 0");
    if (max_iter < 0)
        return fail(STAG_ERR_ARG, "stag_cg_solve_mixed: max_iter must be >= 0");
    if (!(delta > 0 && delta < 1))
        return fail(STAG_ERR_ARG, "stag_cg_solve_mixed: delta must be in (0, 1)");
    const int hi = x->prec, lo = inner_prec;
    if (!lat->has_gauge || !lat->links[hi] || !lat->links[lo])
        return fail(STAG_ERR_STATE, "stag_cg_solve_mixed: needs %s and %s gauge copies", prec_name(hi),
                    prec_name(lo));
    DEVICE_SCOPE(lat->device);
    RhsScale rs;
    STAG_TRY(rhs_scale_begin(b, &rs));
    const stag_field bs = rs.scaled ? rs.scaled : b;
    const int st = mixed_solve_raw(lat, hi, lo, x->data, bs->data, bs->bytes, mass, rel_tol, max_iter, delta, info);
    STAG_TRY(rhs_scale_end(&rs, &x, 1));
    return st;
}


// --------------------------------------------------------------------------
// multi-shift CG (kernels_multishift.cu has the recurrences)
// --------------------------------------------------------------------------
static int ensure_ms_state(stag_lattice lat) {
    // each buffer on its own: an allocation that failed in an earlier call
    // is retried here instead of leaving the others in use without it
    if (!lat->ms_state)
        CUDA_TRY(cudaMalloc(&lat->ms_state, sizeof(ShiftState) * MS_MAX));
    if (!lat->ms_state_host)
        CUDA_TRY(cudaMallocHost(&lat->ms_state_host, sizeof(ShiftState) * MS_MAX));
    if (!lat->ms_true)
        CUDA_TRY(cudaMalloc(&lat->ms_true, sizeof(double) * MS_MAX));
    if (!lat->ms_true_host)
        CUDA_TRY(cudaMallocHost(&lat->ms_true_host, sizeof(double) * MS_MAX));
    return STAG_OK;
}

// the base residual recomputed in the vectors' precision (mixed multi-shift:
// gated on sc->reliable), then the restart of the base scalars
static cudaError_t enqueue_ms_reliable(stag_lattice lat, int prec, const MsArgs &a, cudaStream_t s) {
    CgWork &w = lat->cg[prec];
    cudaError_t e;
    DslashArgs a3 = dslash_args(lat, prec, STAG_ODD, a.x[a.base], w.t);
    a3.gate = reliable_flag(lat);
    if ((e = launch_dslash(prec, EPI_NONE, a3, lat->dslash_block[prec], s)) != cudaSuccess)
        return e;
    DslashArgs a4 = dslash_args(lat, prec, STAG_EVEN, w.t, a.r);
    a4.p = a.x[a.base];
    a4.b = a.b;
    a4.gate = reliable_flag(lat);
    if ((e = launch_dslash(prec, EPI_RESID_STORE, a4, lat->dslash_block[prec], s)) != cudaSuccess)
        return e;
    return launch_ms_restart(a, lat->sc, lat->ms_state, s);
}

// one iteration; lo >= 0: the Dslash pair in FP32 on a.p_lo (mixed), with
// the reliable update in an IF node when captured (side != nullptr, as in
// the mixed solver) or gated kernels otherwise
static const int *scalar_flag(stag_lattice lat, size_t off) { return (const int *)((const char *)lat->sc + off); }

// the Dslash pair M p_base of one iteration in precision op, with the
// <p, M p> partials and alpha; gate: run only while *gate != 0
static cudaError_t enqueue_ms_op(stag_lattice lat, int op, const void *pb, bool host_mode, const int *gate,
                                 cudaStream_t s) {
    CgWork &w = lat->cg[op];
    DslashArgs a1 = dslash_args(lat, op, STAG_ODD, pb, w.t);
    a1.skip_if_done = host_mode;
    a1.gate = gate;
    cudaError_t e = launch_dslash(op, EPI_NONE, a1, lat->dslash_block[op], s);
    if (e != cudaSuccess)
        return e;
    return enqueue_m_pap(lat, op, w.t, w.Ap, pb, host_mode, s, gate);
}

static cudaError_t enqueue_ms_body(stag_lattice lat, int prec, const MsArgs &a, bool host_mode, int lo = -1,
                                   cudaStream_t side = nullptr) {
    cudaStream_t s = lat->stream;
    cudaError_t e;
    if (lo < 0) {
        if ((e = enqueue_ms_op(lat, prec, a.p[a.base], host_mode, nullptr, s)) != cudaSuccess)
            return e;
    } else {
        // the exact operator while |r| is large, the FP32 one afterwards
        if ((e = enqueue_ms_op(lat, prec, a.p[a.base], host_mode, scalar_flag(lat, offsetof(CgScalars, ms_hi_op)),
                               s)) != cudaSuccess ||
            (e = enqueue_ms_op(lat, lo, a.p_lo, host_mode, scalar_flag(lat, offsetof(CgScalars, ms_lo_op)), s)) !=
                cudaSuccess)
            return e;
    }
    const void *Ap = lat->cg[lo >= 0 ? lo : prec].Ap;
    if ((e = launch_ms_update(prec, lat->geom, a, Ap, lat->partial, lat->sc, lat->ms_state, s, lo)) !=
        cudaSuccess)
        return e;
    if ((e = launch_ms_p(prec, lat->geom, a, lat->sc, lat->ms_state, s, lo)) != cudaSuccess)
        return e;
    if (lo < 0)
        return cudaSuccess;
    if (!side)
        return enqueue_ms_reliable(lat, prec, a, s);
    cudaStreamCaptureStatus st;
    cudaGraph_t body = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if ((e = cudaStreamGetCaptureInfo(s, &st, nullptr, &body, &deps, nullptr, &ndeps)) != cudaSuccess)
        return e;
    cudaGraphConditionalHandle rel_cond;
    if ((e = cudaGraphConditionalHandleCreate(&rel_cond, body, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return e;
    // the kernels set the IF condition through the handle in the scalars
    lat->ms_rel_cond = rel_cond;
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    ip.conditional.handle = rel_cond;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t branch;
    if ((e = cudaGraphAddNode(&branch, body, deps, nullptr, ndeps, &ip)) != cudaSuccess)
        return e;
    if ((e = cudaStreamUpdateCaptureDependencies(s, &branch, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return e;
    if ((e = cudaStreamBeginCaptureToGraph(side, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return e;
    cudaError_t e2 = enqueue_ms_reliable(lat, prec, a, side);
    cudaGraph_t branch_out = nullptr;
    e = cudaStreamEndCapture(side, &branch_out);
    return e2 != cudaSuccess ? e2 : e;
}

// one graph: init, WHILE(body); built per call (the solution buffers are
// the caller's) and destroyed after it
static int run_ms_graph(stag_lattice lat, int prec, const MsArgs &a, double mass_base, double tol,
                        int max_iter, int lo, double delta) {
    cudaStream_t s = lat->stream;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 0, 0);
    auto bail = [&](const char *what, cudaError_t err) {
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(s, &junk);
        }
        cudaGetLastError();
        if (exec)
            cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(STAG_ERR_CUDA, "multi-shift graph (%s): %s", what, cudaGetErrorString(err));
    };
    if (e != cudaSuccess)
        return bail("conditional handle", e);
    if ((e = cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail("begin capture", e);
    if ((e = launch_ms_init(prec, lat->geom, a, lat->partial, lat->sc, lat->ms_state, s, lo)) != cudaSuccess)
        return bail("init", e);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if ((e = cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &ndeps)) != cudaSuccess)
        return bail("capture info", e);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((e = cudaGraphAddNode(&loop, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess)
        return bail("add loop node", e);
    if ((e = cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return bail("update deps", e);
    cudaGraph_t captured = nullptr;
    if ((e = cudaStreamEndCapture(s, &captured)) != cudaSuccess)
        return bail("end capture", e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t side = nullptr;
    if (lo >= 0 && (e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking)) != cudaSuccess)
        return bail("side stream", e);
    if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        if (side)
            cudaStreamDestroy(side);
        return bail("begin body capture", e);
    }
    e = enqueue_ms_body(lat, prec, a, false, lo, side);
    if (side)
        cudaStreamDestroy(side);
    if (e != cudaSuccess)
        return bail("body", e);
    cudaGraph_t body_out = nullptr;
    if ((e = cudaStreamEndCapture(s, &body_out)) != cudaSuccess)
        return bail("end body capture", e);
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
        return bail("instantiate", e);
    STAG_TRY(upload_scalars(lat, mass_base, tol, max_iter, true, cond, lo >= 0 ? delta : 0.0, lo >= 0,
                            lo >= 0 ? lat->ms_rel_cond : 0));
    if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess)
        return bail("launch", e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
        return bail("run", e);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return STAG_OK;
}

// multi-shift CG on raw buffers of precision prec; infos[s] per shift
// lo >= 0: the Dslash pair in FP32 with reliable updates of the base
// residual at delta (vectors in prec: F64 or DF64)
static int ms_solve_raw(stag_lattice lat, int prec, void *const *x_data, const double *shifts, int n,
                        const void *b_data, size_t bytes, double mass, double tol, int max_iter,
                        stag_solve_info *infos, double *seconds, int lo = -1, double delta = 0.0) {
    STAG_TRY(ensure_cg_work(lat, prec));
    if (lo >= 0)
        STAG_TRY(ensure_cg_work(lat, lo));
    STAG_TRY(ensure_ms_state(lat));
    for (int k = 0; k < n; k++)
        STAG_TRY(alloc_vec(lat, prec, &lat->ms_p[prec][k]));
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    MsArgs a;
    memset(&a, 0, sizeof a);
    a.n = n;
    a.base = 0;
    for (int k = 1; k < n; k++)
        if (shifts[k] < shifts[a.base])
            a.base = k;
    for (int k = 0; k < n; k++) {
        a.delta[k] = shifts[k] - shifts[a.base];
        a.x[k] = x_data[k];
        a.p[k] = lat->ms_p[prec][k];
    }
    a.b = w.bw;
    a.r = w.r;
    a.p_lo = lo >= 0 ? lat->cg[lo].p : nullptr;
    a.Ap_hi = w.Ap;
    // FP32 operator: its rounding (about 6e-8 relative) enters the shifted
    // solutions in proportion to |r|, so it takes over once |r| < theta |b|,
    // theta = tol / (16 * 6e-8)
    const double theta = lo >= 0 ? std::min(1.0, tol / (16 * 6e-8)) : 0.0;
    a.theta2 = theta * theta;
    const double mass_base = std::sqrt(mass * mass + shifts[a.base]);
    CUDA_TRY(cudaMemcpyAsync(w.bw, b_data, bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaEventRecord(lat->ev0, s));
    if (lat->cg_launch == STAG_CG_LAUNCH_GRAPH) {
        STAG_TRY(run_ms_graph(lat, prec, a, mass_base, tol, max_iter, lo, delta));
    } else {
        STAG_TRY(upload_scalars(lat, mass_base, tol, max_iter, false, 0, lo >= 0 ? delta : 0.0));
        CUDA_TRY(launch_ms_init(prec, lat->geom, a, lat->partial, lat->sc, lat->ms_state, s, lo));
        const int chunk = lat->cg_chunk;
        const long long max_chunks = (long long)max_iter / chunk + 2;
        for (long long k = 0; k < max_chunks; k++) {
            CUDA_TRY(cudaMemcpyAsync(&lat->sc_host->status, &lat->sc->status, sizeof(int),
                                     cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            if (lat->sc_host->status != CG_RUNNING)
                break;
            for (int j = 0; j < chunk; j++)
                CUDA_TRY(enqueue_ms_body(lat, prec, a, true, lo));
        }
    }
    CUDA_TRY(cudaEventRecord(lat->ev1, s));
    // true residual of every shift, |b - (M + sigma_s) x_s|^2
    for (int k = 0; k < n; k++) {
        DslashArgs a1 = dslash_args(lat, prec, STAG_ODD, x_data[k], w.t);
        CUDA_TRY(launch_dslash(prec, EPI_NONE, a1, lat->dslash_block[prec], s));
        DslashArgs a2 = dslash_args(lat, prec, STAG_EVEN, w.t, nullptr);
        a2.p = x_data[k];
        a2.b = w.bw;
        a2.m2 = make_dpair(mass * mass + shifts[k]);
        a2.m2_in_args = 1;
        CUDA_TRY(launch_dslash(prec, EPI_RESID, a2, lat->dslash_block[prec], s));
        CUDA_TRY(cudaMemcpyAsync(lat->ms_true + k, (const char *)lat->sc + offsetof(CgScalars, true_rr),
                                 sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CUDA_TRY(cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(lat->ms_state_host, lat->ms_state, sizeof(ShiftState) * n,
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(lat->ms_true_host, lat->ms_true, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, lat->ev0, lat->ev1));
    if (seconds)
        *seconds = ms * 1e-3;
    const CgScalars &h = *lat->sc_host;
    int worst = STAG_OK;
    for (int k = 0; k < n; k++) {
        const ShiftState &st = lat->ms_state_host[k];
        stag_solve_info &inf = infos[k];
        memset(&inf, 0, sizeof inf);
        inf.iters = h.bb > 0 && st.iters == 0 && h.status != CG_CONVERGED ? h.iter : st.iters;
        inf.status = h.status == CG_BREAKDOWN ? STAG_ERR_BREAKDOWN
                     : (st.active == 0 ? STAG_OK : STAG_ERR_NOT_CONVERGED);
        inf.true_rel_resid = h.bb > 0 ? std::sqrt(lat->ms_true_host[k] / h.bb) : 0.0;
        inf.iter_rel_resid = h.bb > 0 ? std::sqrt(st.zeta * st.zeta * h.rr / h.bb) : 0.0;
        inf.seconds = ms * 1e-3;
        if (inf.status != STAG_OK && worst == STAG_OK)
            worst = inf.status;
    }
    // model rates on the first entry: base CG plus the per-shift vector passes
    const double rb = prec == STAG_F32 ? 4.0 : 8.0;
    const double Vh = (double)lat->Vh;
    const double bytes_it = ((2.0 * 300 + 60) * rb + n * 4 * 6 * rb) * Vh;
    const double flops_it = (2.0 * 1146 + 72 + n * 24.0) * Vh;
    if (ms > 0) {
        infos[0].gbs = bytes_it * h.iter / (ms * 1e-3) / 1e9;
        infos[0].gflops = flops_it * h.iter / (ms * 1e-3) / 1e9;
    }
    return worst;
}

static int check_ms_args(stag_lattice lat, stag_field *xs, const double *shifts, int n, const stag_field b,
                         double mass, double rel_tol, int max_iter, const char *who) {
    if (!lat || !xs || !shifts || !b)
        return fail(STAG_ERR_ARG, "%s: NULL argument", who);
    if (n < 1 || n > MS_MAX)
        return fail(STAG_ERR_ARG, "%s: number of shifts %d not in [1, %d]", who, n, MS_MAX);
    if (b->lat != lat || b->parity != STAG_EVEN)
        return fail(STAG_ERR_ARG, "%s: b must be an even field of this lattice", who);
    for (int k = 0; k < n; k++) {
        if (!xs[k] || xs[k]->lat != lat || xs[k]->parity != STAG_EVEN || xs[k]->prec != b->prec)
            return fail(STAG_ERR_ARG, "%s: xs[%d] must be an even field of b's precision", who, k);
        if (xs[k] == b)
            return fail(STAG_ERR_ARG, "%s: xs[%d] aliases b", who, k);
        for (int j = 0; j < k; j++)
            if (xs[j] == xs[k])
                return fail(STAG_ERR_ARG, "%s: xs[%d] and xs[%d] are the same field", who, j, k);
        if (!(shifts[k] >= 0) || !std::isfinite(shifts[k]))
            return fail(STAG_ERR_ARG, "%s: shift %d must be finite and >= 0", who, k);
    }
    if (!(mass > 0) || !std::isfinite(mass))
        return fail(STAG_ERR_ARG, "%s: mass must be positive and finite", who);
    if (!(rel_tol >= 0) || !std::isfinite(rel_tol))
        return fail(STAG_ERR_ARG, "%s: rel_tol must be >= 0", who);
    if (max_iter < 0)
        return fail(STAG_ERR_ARG, "%s: max_iter must be >= 0", who);
    return STAG_OK;
}

extern "C" int stag_cg_multishift(stag_lattice lat, stag_field *xs, const double *shifts, int n,
                                  const stag_field b, double mass, double rel_tol, int max_iter,
                                  stag_solve_info *infos) {
    STAG_NVTX("stag_cg_multishift");
    STAG_TRY(check_ms_args(lat, xs, shifts, n, b, mass, rel_tol, max_iter, "stag_cg_multishift"));
    const int prec = b->prec;
    if (prec != STAG_F64 && prec != STAG_DF64 && prec != STAG_F32)
        return fail(STAG_ERR_STATE, "stag_cg_multishift: fields must be F64, DF64 or F32");
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_cg_multishift: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    void *xd[MS_MAX];
    for (int k = 0; k < n; k++)
        xd[k] = xs[k]->data;
    stag_solve_info local[MS_MAX];
    RhsScale rs;
    STAG_TRY(rhs_scale_begin(b, &rs));
    const stag_field bs = rs.scaled ? rs.scaled : b;
    const int st = ms_solve_raw(lat, prec, xd, shifts, n, bs->data, bs->bytes, mass, rel_tol, max_iter,
                                local, nullptr);
    STAG_TRY(rhs_scale_end(&rs, xs, n));
    if (infos)
        memcpy(infos, local, sizeof(stag_solve_info) * n);
    if (st != STAG_OK && st != STAG_ERR_NOT_CONVERGED && st != STAG_ERR_BREAKDOWN)
        return st;
    if (st != STAG_OK)
        return fail(st, "stag_cg_multishift: %s", st == STAG_ERR_BREAKDOWN ? "breakdown" : "not converged");
    return STAG_OK;
}

// |b - (M + m_k^2 - m^2) x|^2 into the host, r stored to r_out (precision hi)
int shifted_residual(stag_lattice lat, int hi, const void *x, const void *b, double mk, void *r_out,
                            double *rr) {
    CgWork &H = lat->cg[hi];
    cudaStream_t s = lat->stream;
    DslashArgs a1 = dslash_args(lat, hi, STAG_ODD, x, H.t);
    CUDA_TRY(launch_dslash(hi, EPI_NONE, a1, lat->dslash_block[hi], s));
    DslashArgs a2 = dslash_args(lat, hi, STAG_EVEN, H.t, r_out);
    a2.p = x;
    a2.b = b;
    a2.m2 = make_dpair(mk * mk);
    a2.m2_in_args = 1;
    CUDA_TRY(launch_dslash(hi, r_out ? EPI_RESID_STORE : EPI_RESID, a2, lat->dslash_block[hi], s));
    CUDA_TRY(cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *rr = lat->sc_host->true_rr;
    return STAG_OK;
}

static int multishift_mixed_impl(stag_lattice lat, stag_field *xs, const double *shifts, int n,
                                 const stag_field b, double mass, double rel_tol, int max_iter,
                                 int inner_prec, double delta, stag_solve_info *infos);

extern "C" int stag_cg_multishift_mixed(stag_lattice lat, stag_field *xs, const double *shifts, int n,
                                        const stag_field b, double mass, double rel_tol, int max_iter,
                                        int inner_prec, double delta, stag_solve_info *infos) {
    STAG_NVTX("stag_cg_multishift_mixed");
    STAG_TRY(check_ms_args(lat, xs, shifts, n, b, mass, rel_tol, max_iter, "stag_cg_multishift_mixed"));
    RhsScale rs;
    STAG_TRY(rhs_scale_begin(b, &rs));
    const int st = multishift_mixed_impl(lat, xs, shifts, n, rs.scaled ? rs.scaled : b, mass, rel_tol, max_iter,
                                         inner_prec, delta, infos);
    STAG_TRY(rhs_scale_end(&rs, xs, n));
    return st;
}

static int multishift_mixed_impl(stag_lattice lat, stag_field *xs, const double *shifts, int n,
                                 const stag_field b, double mass, double rel_tol, int max_iter,
                                 int inner_prec, double delta, stag_solve_info *infos) {
    const int hi = b->prec;
    if (hi != STAG_F64 && hi != STAG_DF64)
        return fail(STAG_ERR_STATE, "stag_cg_multishift_mixed: fields must be F64 or DF64");
    if (inner_prec != STAG_F32 && inner_prec != STAG_F16)
        return fail(STAG_ERR_ARG, "stag_cg_multishift_mixed: inner precision must be F32 or F16");
    if (!(delta > 0 && delta < 1))
        return fail(STAG_ERR_ARG, "stag_cg_multishift_mixed: delta must be in (0, 1)");
    if (!lat->has_gauge || !lat->links[hi] || !lat->links[STAG_F32] || !lat->links[inner_prec])
        return fail(STAG_ERR_STATE, "stag_cg_multishift_mixed: needs %s, F32 and %s gauge copies",
                    prec_name(hi), prec_name(inner_prec));
    DEVICE_SCOPE(lat->device);
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = lat->stream;
    const Geom &g = lat->geom;
    STAG_TRY(ensure_cg_work(lat, hi));
    STAG_TRY(alloc_vec(lat, hi, &lat->ms_rhi[hi]));
    STAG_TRY(alloc_vec(lat, hi, &lat->ms_ehi[hi]));
    // |b|^2 in the high precision: the residual of x = 0
    CUDA_TRY(cudaMemsetAsync(lat->ms_ehi[hi], 0, field_bytes(lat, hi), s));
    double bb = 0;
    STAG_TRY(shifted_residual(lat, hi, lat->ms_ehi[hi], b->data, mass, nullptr, &bb));
    // phase 1: all shifts in one Krylov space, vectors in the high precision,
    // the Dslash pair in FP32, reliable updates of the base residual
    void *xd[MS_MAX];
    for (int k = 0; k < n; k++)
        xd[k] = xs[k]->data;
    stag_solve_info lo_info[MS_MAX];
    int st = ms_solve_raw(lat, hi, xd, shifts, n, b->data, b->bytes, mass, rel_tol, max_iter, lo_info, nullptr,
                          STAG_F32, delta);
    if (st != STAG_OK && st != STAG_ERR_NOT_CONVERGED)
        return st;
    // phase 2: a shift whose recomputed residual misses the tolerance (the
    // shifted systems cannot take reliable updates inside the shared space)
    // is refined by the mixed solver on its own residual
    int worst = STAG_OK;
    stag_solve_info out[MS_MAX];
    for (int k = 0; k < n; k++) {
        memset(&out[k], 0, sizeof out[k]);
        const double mk = std::sqrt(mass * mass + shifts[k]);
        double rr0 = 0;
        STAG_TRY(shifted_residual(lat, hi, xs[k]->data, b->data, mk, lat->ms_rhi[hi], &rr0));
        const double rel0 = bb > 0 ? std::sqrt(rr0 / bb) : 0.0;
        stag_solve_info ri;
        memset(&ri, 0, sizeof ri);
        if (rel0 > rel_tol) {
            const int rs = mixed_solve_raw(lat, hi, inner_prec, lat->ms_ehi[hi], lat->ms_rhi[hi],
                                           field_bytes(lat, hi), mk, rel_tol / rel0, max_iter, delta, &ri);
            if (rs != STAG_OK && rs != STAG_ERR_NOT_CONVERGED && rs != STAG_ERR_BREAKDOWN)
                return rs;
            CUDA_TRY(launch_axpy1(hi, g, lat->ms_ehi[hi], xs[k]->data, s));
        }
        double rr1 = 0;
        STAG_TRY(shifted_residual(lat, hi, xs[k]->data, b->data, mk, nullptr, &rr1));
        out[k].iters = lo_info[k].iters;
        out[k].restarts = ri.iters;  // refinement iterations (inner precision)
        out[k].true_rel_resid = bb > 0 ? std::sqrt(rr1 / bb) : 0.0;
        out[k].iter_rel_resid = rel0;
        out[k].status = out[k].true_rel_resid <= rel_tol * 1.05 || bb == 0 ? STAG_OK
                        : ri.status != STAG_OK ? ri.status : STAG_ERR_NOT_CONVERGED;
        if (out[k].status != STAG_OK && worst == STAG_OK)
            worst = out[k].status;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < n; k++)
        out[k].seconds = secs;
    if (infos)
        memcpy(infos, out, sizeof(stag_solve_info) * n);
    if (worst != STAG_OK)
        return fail(worst, "stag_cg_multishift_mixed: a shift did not reach the tolerance");
    return STAG_OK;
}

// --------------------------------------------------------------------------
// batched CG over many (lattice, right-hand side) systems, one graph
// --------------------------------------------------------------------------
struct BatchPlan {
    BatchArgs a;
    int nsys = 0;
    int prec = 0;
    cudaStream_t stream = nullptr;
    int block = 128;
    // device buffers owned by one call
    CgScalars *sys = nullptr;
    unsigned *tickets = nullptr;
    BatchCtl *ctl = nullptr;
    double *partial = nullptr;
    void release() {
        if (sys) cudaFree(sys);
        if (tickets) cudaFree(tickets);
        if (ctl) cudaFree(ctl);
        if (partial) cudaFree(partial);
        sys = nullptr;
        tickets = nullptr;
        ctl = nullptr;
        partial = nullptr;
    }
};

// group systems by lattice (consecutive, at most batch_max_k per group) and
// allocate work vectors and reduction buffers; x/b are raw buffers
static int plan_batch(BatchPlan &P, int n, stag_lattice *lats, void *const *x, const void *const *b,
                      int prec) {
    // systems per group: the lattice's tuned group size, else the largest
    auto group_k = [&](stag_lattice L) { return L->batch_k[prec] > 0 ? L->batch_k[prec] : batch_max_k(prec); };
    memset(&P.a, 0, sizeof P.a);
    P.nsys = n;
    P.prec = prec;
    P.stream = lats[0]->stream;
    P.block = lats[0]->batch_block[prec];
    int slot_of_lat[BATCH_MAX_G * BATCH_KMAX];
    int G = 0, blocks = 0;
    size_t partial_total = 0;
    for (int i = 0; i < n; i++) {
        // slot = index of this system among the earlier systems of its lattice
        int slot = 0;
        for (int j = 0; j < i; j++)
            if (lats[j] == lats[i])
                slot++;
        slot_of_lat[i] = slot;
        const int K = group_k(lats[i]);
        const bool new_group = G == 0 || lats[i] != lats[i - 1] || P.a.grp[G - 1].K == K;
        if (new_group) {
            if (G == BATCH_MAX_G)
                return fail(STAG_ERR_ARG, "stag_cg_solve_batched: more than %d groups (at most %d "
                            "systems of one lattice per group; keep systems of a lattice together)",
                            BATCH_MAX_G, K);
            BatchGroup &gr = P.a.grp[G];
            gr.g = lats[i]->geom;
            gr.K = 0;
            gr.block0 = blocks;
            gr.nblocks = (gr.g.Vh + P.block - 1) / P.block;
            gr.sys0 = i;
            gr.links[0] = links_of(lats[i], prec, 0);
            gr.links[1] = links_of(lats[i], prec, 1);
            gr.link_scale[0] = gr.link_scale[1] = 0.f;
            blocks += gr.nblocks;
            G++;
        }
        BatchGroup &gr = P.a.grp[G - 1];
        const int k = gr.K++;
        stag_lattice L = lats[i];
        for (int v = 0; v < 4; v++)
            STAG_TRY(alloc_vec(L, prec, &L->bwork[prec][slot_of_lat[i]][v]));
        gr.x[k] = x[i];
        gr.b[k] = b[i];
        gr.r[k] = L->bwork[prec][slot_of_lat[i]][0];
        gr.p[k] = L->bwork[prec][slot_of_lat[i]][1];
        gr.Ap[k] = L->bwork[prec][slot_of_lat[i]][2];
        gr.t[k] = L->bwork[prec][slot_of_lat[i]][3];
    }
    P.a.G = G;
    P.a.nblocks = blocks;
    P.a.kmax = 0;
    for (int gi = 0; gi < G; gi++)
        P.a.kmax = std::max(P.a.kmax, P.a.grp[gi].K);
    // lane-mapped Dslash (double-float, FP64): one thread per (site, system)
    int dblocks = 0;
    for (int gi = 0; gi < G; gi++) {
        BatchGroup &gr = P.a.grp[gi];
        gr.dblock0 = dblocks;
        gr.dnblocks = (int)(((long long)gr.g.Vh * gr.K + P.block - 1) / P.block);
        dblocks += gr.dnblocks;
        partial_total += (size_t)std::max(gr.nblocks, gr.dnblocks) * BATCH_KMAX;
    }
    P.a.dnblocks = dblocks;
    cudaError_t e;
    if ((e = cudaMalloc(&P.sys, sizeof(CgScalars) * n)) != cudaSuccess ||
        (e = cudaMalloc(&P.tickets, sizeof(unsigned) * G)) != cudaSuccess ||
        (e = cudaMalloc(&P.ctl, sizeof(BatchCtl))) != cudaSuccess ||
        (e = cudaMalloc(&P.partial, sizeof(double) * partial_total)) != cudaSuccess) {
        P.release();
        return fail(STAG_ERR_NOMEM, "stag_cg_solve_batched: %s", cudaGetErrorString(e));
    }
    // every system starts as CG_RUNNING (0) until the init kernel decides
    if ((e = cudaMemsetAsync(P.sys, 0, sizeof(CgScalars) * n, P.stream)) != cudaSuccess) {
        P.release();
        return fail(STAG_ERR_CUDA, "stag_cg_solve_batched: %s", cudaGetErrorString(e));
    }
    size_t off = 0;
    for (int gi = 0; gi < G; gi++) {
        P.a.grp[gi].partial = P.partial + off;
        off += (size_t)std::max(P.a.grp[gi].nblocks, P.a.grp[gi].dnblocks) * BATCH_KMAX;
    }
    P.a.sys = P.sys;
    P.a.tickets = P.tickets;
    P.a.ctl = P.ctl;
    return STAG_OK;
}

static cudaError_t enqueue_batch_body(const BatchPlan &P) {
    cudaError_t e;
    const int w[4] = {BATCH_DSLASH_OE, BATCH_M_PAP, BATCH_UPDATE, BATCH_P};
    for (int k = 0; k < 4; k++)
        if ((e = launch_batch(P.prec, w[k], P.a, P.block, P.stream)) != cudaSuccess)
            return e;
    return cudaSuccess;
}

// run the batched CG to completion: init, WHILE(body), true residuals
static int run_batch(BatchPlan &P, const double *masses, double tol, int max_iter, float *ms_out) {
    cudaStream_t s = P.stream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 0, 0);
    auto bail = [&](const char *what, cudaError_t err) {
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(s, &junk);
        }
        cudaGetLastError();
        if (exec)
            cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(STAG_ERR_CUDA, "batched CG graph (%s): %s", what, cudaGetErrorString(err));
    };
    if (e != cudaSuccess)
        return bail("conditional handle", e);
    // scalars: per system m^2, tol^2, max_iter; control block
    {
        std::vector<CgScalars> h(P.nsys);
        memset(h.data(), 0, sizeof(CgScalars) * P.nsys);
        for (int i = 0; i < P.nsys; i++) {
            h[i].m2 = make_dpair(masses[i] * masses[i]);
            h[i].tol2 = tol * tol;
            h[i].max_iter = max_iter;
        }
        BatchCtl c;
        memset(&c, 0, sizeof c);
        c.cond = cond;
        c.has_cond = 1;
        if ((e = cudaMemcpyAsync(P.sys, h.data(), sizeof(CgScalars) * P.nsys, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(P.ctl, &c, sizeof c, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(P.tickets, 0, sizeof(unsigned) * P.a.G, s)) != cudaSuccess)
            return bail("scalars", e);
    }
    if ((e = cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail("begin capture", e);
    if ((e = launch_batch(P.prec, BATCH_INIT, P.a, P.block, s)) != cudaSuccess)
        return bail("init", e);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if ((e = cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &ndeps)) != cudaSuccess)
        return bail("capture info", e);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((e = cudaGraphAddNode(&loop, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess)
        return bail("add loop node", e);
    if ((e = cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return bail("update deps", e);
    if ((e = launch_batch(P.prec, BATCH_DSLASH_X, P.a, P.block, s)) != cudaSuccess ||
        (e = launch_batch(P.prec, BATCH_RESID, P.a, P.block, s)) != cudaSuccess)
        return bail("true residual", e);
    cudaGraph_t captured = nullptr;
    if ((e = cudaStreamEndCapture(s, &captured)) != cudaSuccess)
        return bail("end capture", e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail("begin body capture", e);
    if ((e = enqueue_batch_body(P)) != cudaSuccess)
        return bail("body", e);
    cudaGraph_t body_out = nullptr;
    if ((e = cudaStreamEndCapture(s, &body_out)) != cudaSuccess)
        return bail("end body capture", e);
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
        return bail("instantiate", e);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    e = cudaGraphLaunch(exec, s);
    cudaEventRecord(e1, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return bail("run", e != cudaSuccess ? e : e2);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (ms_out)
        *ms_out = ms;
    return STAG_OK;
}

static int check_batch(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs, const double *masses,
                       double rel_tol, int max_iter, const char *who) {
    if (!lats || !xs || !bs || !masses)
        return fail(STAG_ERR_ARG, "%s: NULL argument", who);
    if (n < 1 || n > BATCH_MAX_G * BATCH_KMAX)
        return fail(STAG_ERR_ARG, "%s: number of systems %d not in [1, %d]", who, n, BATCH_MAX_G * BATCH_KMAX);
    for (int i = 0; i < n; i++) {
        if (!lats[i] || !xs[i] || !bs[i])
            return fail(STAG_ERR_ARG, "%s: NULL lattice or field for system %d", who, i);
        if (lats[i]->device != lats[0]->device)
            return fail(STAG_ERR_ARG, "%s: all lattices must be on one device", who);
        if (xs[i]->lat != lats[i] || bs[i]->lat != lats[i] || xs[i]->parity != STAG_EVEN ||
            bs[i]->parity != STAG_EVEN)
            return fail(STAG_ERR_ARG, "%s: system %d needs even fields of its lattice", who, i);
        if (xs[i]->prec != bs[0]->prec || bs[i]->prec != bs[0]->prec)
            return fail(STAG_ERR_ARG, "%s: all fields must have one precision", who);
        if (xs[i] == bs[i])
            return fail(STAG_ERR_ARG, "%s: x and b of system %d alias", who, i);
        for (int j = 0; j < i; j++)
            if (xs[j] == xs[i])
                return fail(STAG_ERR_ARG, "%s: systems %d and %d share a solution field", who, j, i);
        if (!(masses[i] > 0) || !std::isfinite(masses[i]))
            return fail(STAG_ERR_ARG, "%s: mass %d must be positive and finite", who, i);
        // systems of one lattice must be consecutive
        for (int j = 0; j + 1 < i; j++)
            if (lats[j] == lats[i] && lats[j + 1] != lats[i])
                return fail(STAG_ERR_ARG, "%s: systems of one lattice must be consecutive", who);
    }
    if (!(rel_tol >= 0) || !std::isfinite(rel_tol))
        return fail(STAG_ERR_ARG, "%s: rel_tol must be >= 0", who);
    if (max_iter < 0)
        return fail(STAG_ERR_ARG, "%s: max_iter must be >= 0", who);
    return STAG_OK;
}

static int batch_solve_raw(int n, stag_lattice *lats, void *const *x, const void *const *b, const double *masses,
                           int prec, double rel_tol, int max_iter, stag_solve_info *infos) {
    for (int i = 0; i < n; i++)
        if (!lats[i]->has_gauge || !lats[i]->links[prec])
            return fail(STAG_ERR_STATE, "stag_cg_solve_batched: lattice of system %d has no %s gauge copy",
                        i, prec_name(prec));
    // work of the other lattices' streams must be done before the batch
    // runs on the first lattice's stream
    for (int i = 1; i < n; i++)
        if (lats[i]->stream != lats[0]->stream)
            CUDA_TRY(cudaStreamSynchronize(lats[i]->stream));
    BatchPlan P;
    STAG_TRY(plan_batch(P, n, lats, x, b, prec));
    float ms = 0.f;
    int st = run_batch(P, masses, rel_tol, max_iter, &ms);
    if (st != STAG_OK) {
        P.release();
        return st;
    }
    std::vector<CgScalars> h(n);
    cudaError_t e = cudaMemcpy(h.data(), P.sys, sizeof(CgScalars) * n, cudaMemcpyDeviceToHost);
    P.release();
    if (e != cudaSuccess)
        return fail(STAG_ERR_CUDA, "stag_cg_solve_batched: %s", cudaGetErrorString(e));
    int worst = STAG_OK;
    double total_bytes = 0, total_flops = 0;
    const double rb = prec == STAG_F32 ? 4.0 : 8.0;
    for (int i = 0; i < n; i++) {
        stag_solve_info &inf = infos[i];
        memset(&inf, 0, sizeof inf);
        inf.iters = h[i].iter;
        inf.status = h[i].status == CG_CONVERGED ? STAG_OK
                     : h[i].status == CG_BREAKDOWN ? STAG_ERR_BREAKDOWN
                                                   : STAG_ERR_NOT_CONVERGED;
        inf.true_rel_resid = h[i].bb > 0 ? std::sqrt(h[i].true_rr / h[i].bb) : 0.0;
        inf.iter_rel_resid = h[i].bb > 0 ? std::sqrt(h[i].rr / h[i].bb) : 0.0;
        inf.seconds = ms * 1e-3;
        if (inf.status != STAG_OK && worst == STAG_OK)
            worst = inf.status;
        total_bytes += (2.0 * 300 + 60) * rb * (double)lats[i]->Vh * h[i].iter;
        total_flops += (2.0 * 1146 + 72) * (double)lats[i]->Vh * h[i].iter;
    }
    if (ms > 0) {
        // per-system-equivalent rates of the whole batch (links counted once
        // per system, as if solved alone)
        infos[0].gbs = total_bytes / (ms * 1e-3) / 1e9;
        infos[0].gflops = total_flops / (ms * 1e-3) / 1e9;
    }
    return worst;
}

// per-system source normalisation around a batched solve
struct BatchRhsScale {
    std::vector<RhsScale> rs;
    std::vector<stag_field> b;
    int begin(int n, const stag_field *bs) {
        rs.assign(n, RhsScale());
        b.assign(bs, bs + n);
        for (int i = 0; i < n; i++) {
            const int st = rhs_scale_begin(bs[i], &rs[i]);
            if (st != STAG_OK) {
                end(i, nullptr);
                return st;
            }
            if (rs[i].scaled)
                b[i] = rs[i].scaled;
        }
        return STAG_OK;
    }
    // xs NULL: only free the copies of the first n systems
    int end(int n, stag_field *xs) {
        int worst = STAG_OK;
        for (int i = 0; i < n; i++) {
            const int st = xs ? rhs_scale_end(&rs[i], &xs[i], 1) : rhs_scale_end(&rs[i], nullptr, 0);
            if (st != STAG_OK && worst == STAG_OK)
                worst = st;
        }
        return worst;
    }
};

static int batched_impl(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs, const double *masses,
                        double rel_tol, int max_iter, stag_solve_info *infos);
static int batched_mixed_impl(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs,
                              const double *masses, double rel_tol, int max_iter, int inner_prec, double delta,
                              stag_solve_info *infos);

extern "C" int stag_cg_solve_batched(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs,
                                     const double *masses, double rel_tol, int max_iter,
                                     stag_solve_info *infos) {
    STAG_NVTX("stag_cg_solve_batched");
    STAG_TRY(check_batch(n, lats, xs, bs, masses, rel_tol, max_iter, "stag_cg_solve_batched"));
    BatchRhsScale sc;
    STAG_TRY(sc.begin(n, bs));
    const int st = batched_impl(n, lats, xs, sc.b.data(), masses, rel_tol, max_iter, infos);
    STAG_TRY(sc.end(n, xs));
    return st;
}

static int batched_impl(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs, const double *masses,
                        double rel_tol, int max_iter, stag_solve_info *infos) {
    const int prec = bs[0]->prec;
    if (prec != STAG_F64 && prec != STAG_DF64 && prec != STAG_F32)
        return fail(STAG_ERR_STATE, "stag_cg_solve_batched: fields must be F64, DF64 or F32");
    DEVICE_SCOPE(lats[0]->device);
    std::vector<void *> x(n);
    std::vector<const void *> b(n);
    for (int i = 0; i < n; i++) {
        x[i] = xs[i]->data;
        b[i] = bs[i]->data;
    }
    std::vector<stag_solve_info> loc(n);
    const int st = batch_solve_raw(n, lats, x.data(), b.data(), masses, prec, rel_tol, max_iter, loc.data());
    if (infos)
        memcpy(infos, loc.data(), sizeof(stag_solve_info) * n);
    if (st != STAG_OK && st != STAG_ERR_NOT_CONVERGED && st != STAG_ERR_BREAKDOWN)
        return st;
    if (st != STAG_OK)
        return fail(st, "stag_cg_solve_batched: a system %s", st == STAG_ERR_BREAKDOWN ? "broke down"
                                                                                      : "did not converge");
    return STAG_OK;
}

extern "C" int stag_cg_solve_batched_mixed(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs,
                                           const double *masses, double rel_tol, int max_iter, int inner_prec,
                                           double delta, stag_solve_info *infos) {
    STAG_NVTX("stag_cg_solve_batched_mixed");
    STAG_TRY(check_batch(n, lats, xs, bs, masses, rel_tol, max_iter, "stag_cg_solve_batched_mixed"));
    BatchRhsScale sc;
    STAG_TRY(sc.begin(n, bs));
    const int st = batched_mixed_impl(n, lats, xs, sc.b.data(), masses, rel_tol, max_iter, inner_prec, delta,
                                      infos);
    STAG_TRY(sc.end(n, xs));
    return st;
}

static int batched_mixed_impl(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs,
                              const double *masses, double rel_tol, int max_iter, int inner_prec, double delta,
                              stag_solve_info *infos) {
    const int hi = bs[0]->prec;
    if (hi != STAG_F64 && hi != STAG_DF64)
        return fail(STAG_ERR_STATE, "stag_cg_solve_batched_mixed: fields must be F64 or DF64");
    if (inner_prec != STAG_F32 && inner_prec != STAG_F16)
        return fail(STAG_ERR_ARG, "stag_cg_solve_batched_mixed: inner precision must be F32 or F16");
    if (!(delta > 0 && delta < 1))
        return fail(STAG_ERR_ARG, "stag_cg_solve_batched_mixed: delta must be in (0, 1)");
    for (int i = 0; i < n; i++)
        if (!lats[i]->has_gauge || !lats[i]->links[hi] || !lats[i]->links[STAG_F32] ||
            !lats[i]->links[inner_prec])
            return fail(STAG_ERR_STATE, "stag_cg_solve_batched_mixed: every lattice needs %s, F32 and %s "
                        "gauge copies", prec_name(hi), prec_name(inner_prec));
    DEVICE_SCOPE(lats[0]->device);
    const auto t0 = std::chrono::steady_clock::now();
    // phase 1: every system in FP32 in one batched graph, to max(rel_tol, 1e-5)
    std::vector<void *> xl(n);
    std::vector<const void *> bl(n);
    for (int i = 0; i < n; i++) {
        int slot = 0;
        for (int j = 0; j < i; j++)
            slot += lats[j] == lats[i];
        STAG_TRY(alloc_vec(lats[i], STAG_F32, &lats[i]->bxlo[slot]));
        STAG_TRY(alloc_vec(lats[i], STAG_F32, &lats[i]->bblo[slot]));
        CUDA_TRY(launch_convert(STAG_F32, hi, lats[i]->geom, bs[i]->data, lats[i]->bblo[slot], lats[i]->stream));
        xl[i] = lats[i]->bxlo[slot];
        bl[i] = lats[i]->bblo[slot];
    }
    const double sloppy = rel_tol > 1e-5 ? rel_tol : 1e-5;
    std::vector<stag_solve_info> lo(n);
    int st = batch_solve_raw(n, lats, xl.data(), bl.data(), masses, STAG_F32, sloppy, max_iter, lo.data());
    if (st != STAG_OK && st != STAG_ERR_NOT_CONVERGED)
        return st;
    // phase 2: per system, x = x_lo, then reliable-update CG on its residual
    int worst = STAG_OK;
    std::vector<stag_solve_info> out(n);
    for (int i = 0; i < n; i++) {
        stag_lattice L = lats[i];
        const Geom &g = L->geom;
        memset(&out[i], 0, sizeof out[i]);
        STAG_TRY(ensure_cg_work(L, hi));
        STAG_TRY(alloc_vec(L, hi, &L->ms_rhi[hi]));
        STAG_TRY(alloc_vec(L, hi, &L->ms_ehi[hi]));
        CUDA_TRY(launch_convert(hi, STAG_F32, g, xl[i], xs[i]->data, L->stream));
        CUDA_TRY(cudaMemsetAsync(L->ms_ehi[hi], 0, field_bytes(L, hi), L->stream));
        double bb = 0, rr0 = 0, rr1 = 0;
        STAG_TRY(shifted_residual(L, hi, L->ms_ehi[hi], bs[i]->data, masses[i], nullptr, &bb));
        STAG_TRY(shifted_residual(L, hi, xs[i]->data, bs[i]->data, masses[i], L->ms_rhi[hi], &rr0));
        const double rel0 = bb > 0 ? std::sqrt(rr0 / bb) : 0.0;
        stag_solve_info ri;
        memset(&ri, 0, sizeof ri);
        if (rel0 > rel_tol) {
            const int rs = mixed_solve_raw(L, hi, inner_prec, L->ms_ehi[hi], L->ms_rhi[hi], field_bytes(L, hi),
                                           masses[i], rel_tol / rel0, max_iter, delta, &ri);
            if (rs != STAG_OK && rs != STAG_ERR_NOT_CONVERGED && rs != STAG_ERR_BREAKDOWN)
                return rs;
            CUDA_TRY(launch_axpy1(hi, g, L->ms_ehi[hi], xs[i]->data, L->stream));
        }
        STAG_TRY(shifted_residual(L, hi, xs[i]->data, bs[i]->data, masses[i], nullptr, &rr1));
        out[i].iters = lo[i].iters;
        out[i].restarts = ri.iters;
        out[i].iter_rel_resid = rel0;
        out[i].true_rel_resid = bb > 0 ? std::sqrt(rr1 / bb) : 0.0;
        out[i].status = out[i].true_rel_resid <= rel_tol * 1.05 || bb == 0 ? STAG_OK
                        : ri.status != STAG_OK ? ri.status : STAG_ERR_NOT_CONVERGED;
        if (out[i].status != STAG_OK && worst == STAG_OK)
            worst = out[i].status;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < n; i++)
        out[i].seconds = secs;
    if (infos)
        memcpy(infos, out.data(), sizeof(stag_solve_info) * n);
    if (worst != STAG_OK)
        return fail(worst, "stag_cg_solve_batched_mixed: a system did not reach the tolerance");
    return STAG_OK;
}

// --------------------------------------------------------------------------
// autotuner: time the candidate block sizes, keep the fastest per lattice
// and precision
// --------------------------------------------------------------------------
// --------------------------------------------------------------------------
// autotuner
// --------------------------------------------------------------------------
// The choices of one (lattice shape, precision, link layout, device): block
// size and register variant of the Dslash and of the M Dslash with partials,
// block size and group size of the batched Dslash.
struct TuneChoice {
    int dblock = 0, dregs = 0, mblock = 0, mregs = 0, bblock = 0, bk = 0;
};

static std::mutex g_tune_mutex;
static std::map<std::string, TuneChoice> g_tune_cache;
static bool g_tune_file_read = false;

static std::string tune_key(const stag_lattice lat, int prec) {
    cudaDeviceProp prop;
    std::string dev = "unknown";
    if (cudaGetDeviceProperties(&prop, lat->device) == cudaSuccess) {
        dev = prop.name;
        for (char &c : dev)
            if (c == ' ')
                c = '_';
    }
    char buf[256];
    snprintf(buf, sizeof buf, "%d %d %d %d %d %d %s", lat->dims[0], lat->dims[1], lat->dims[2], lat->dims[3], prec,
             lat->links_c12[prec] ? lat->c12_mask[prec] : 0, dev.c_str());
    return buf;
}

// the optional file cache: one line per key, "stag-tune2 <key> <six ints>"
// (lines of other formats, such as those of earlier candidate sets, are ignored)
static const char *tune_file() { return getenv("STAG_TUNE_CACHE"); }

// a choice read from the file is applied only if stag_lattice_set_tuning
// would accept each of its parts (a batched group beyond the kernels' size
// would overrun the per-group arrays)
static bool tune_choice_valid(int prec, const TuneChoice &c) {
    auto block_ok = [](int b) { return b == 64 || b == 128 || b == 256 || b == 512; };
    auto regs_ok = [](int r) { return r >= REGS_DEFAULT && r <= REGS_PAIR; };
    if (!prec_valid(prec) || !block_ok(c.dblock) || !block_ok(c.mblock) || !regs_ok(c.dregs) ||
        !regs_ok(c.mregs))
        return false;
    if (c.bblock == 0)
        return c.bk == 0;
    if (prec == STAG_F16 || (c.bblock != 128 && c.bblock != 256))
        return false;
    return c.bk == 0 || (c.bk >= batch_min_k(prec) && c.bk <= batch_max_k(prec) && (c.bk & (c.bk - 1)) == 0);
}

static void tune_file_read_locked() {
    if (g_tune_file_read)
        return;
    g_tune_file_read = true;
    const char *path = tune_file();
    if (!path)
        return;
    FILE *f = fopen(path, "r");
    if (!f)
        return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        int d[4], prec, comp;
        char dev[200];
        TuneChoice c;
        if (sscanf(line, "stag-tune2 %d %d %d %d %d %d %199s %d %d %d %d %d %d", &d[0], &d[1], &d[2], &d[3], &prec,
                   &comp, dev, &c.dblock, &c.dregs, &c.mblock, &c.mregs, &c.bblock, &c.bk) == 13 &&
            tune_choice_valid(prec, c)) {
            char key[256];
            snprintf(key, sizeof key, "%d %d %d %d %d %d %s", d[0], d[1], d[2], d[3], prec, comp, dev);
            g_tune_cache[key] = c;
        }
    }
    fclose(f);
}

static void tune_file_append(const std::string &key, const TuneChoice &c) {
    const char *path = tune_file();
    if (!path)
        return;
    FILE *f = fopen(path, "a");
    if (!f)
        return;
    fprintf(f, "stag-tune2 %s %d %d %d %d %d %d\n", key.c_str(), c.dblock, c.dregs, c.mblock, c.mregs, c.bblock, c.bk);
    fclose(f);
}

static void apply_choice(stag_lattice lat, int prec, const TuneChoice &c) {
    lat->dslash_block[prec] = c.dblock;
    lat->dslash_regs[prec] = c.dregs;
    lat->mdslash_block[prec] = c.mblock;
    lat->mdslash_regs[prec] = c.mregs;
    if (c.bblock > 0) {
        lat->batch_block[prec] = c.bblock;
        lat->batch_k[prec] = c.bk;
    }
}

// microseconds per launch of `launch` (2 warm-ups, `reps` timed launches,
// CUDA events on the lattice stream)
template <class F>
static int time_launch(stag_lattice lat, F launch, int reps, double *us) {
    cudaStream_t s = lat->stream;
    for (int i = 0; i < 2; i++)
        CUDA_TRY(launch());
    CUDA_TRY(cudaEventRecord(lat->ev0, s));
    for (int i = 0; i < reps; i++)
        CUDA_TRY(launch());
    CUDA_TRY(cudaEventRecord(lat->ev1, s));
    CUDA_TRY(cudaEventSynchronize(lat->ev1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, lat->ev0, lat->ev1));
    *us = 1e3 * ms / reps;
    return STAG_OK;
}

static const int kTuneBlocks[4] = {64, 128, 256, 512};

static int tune_all(stag_lattice lat, int prec, std::vector<stag_tune_result> &res, TuneChoice &c) {
    STAG_TRY(ensure_cg_work(lat, prec));
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    const int reps = 10;
    // the Dslash and the M Dslash with partials: block x register variant
    for (int kind = 0; kind < 2; kind++) {
        double best = 1e300;
        for (int bi = 0; bi < 4; bi++)
            for (int regs = REGS_FREE; regs <= REGS_PAIR; regs++) {
                const int block = kTuneBlocks[bi];
                DslashArgs a = kind == 0 ? dslash_args(lat, prec, STAG_ODD, w.p, w.t)
                                         : dslash_args(lat, prec, STAG_EVEN, w.t, w.Ap);
                a.p = w.p;
                a.regs = regs;
                if (regs == REGS_PAIR && !pair16_used(prec, EPI_NONE, a))
                    continue;  // the pair form exists for the compressed 16-bit stencil only
                const int epi = kind == 0 ? EPI_NONE : EPI_M_PART;
                double us = 0;
                STAG_TRY(time_launch(lat, [&]() { return launch_dslash(prec, epi, a, block, s); }, reps, &us));
                stag_tune_result r = {kind == 0 ? STAG_TUNE_DSLASH : STAG_TUNE_M, block, regs, 0, us, 0};
                res.push_back(r);
                if (us < best) {
                    best = us;
                    (kind == 0 ? c.dblock : c.mblock) = block;
                    (kind == 0 ? c.dregs : c.mregs) = regs;
                }
            }
    }
    if (prec == STAG_F16)
        return STAG_OK;  // no batched kernels in 16-bit storage
    // the batched Dslash: block x systems per group, one group of K systems;
    // the time per right-hand side decides
    const int kmax = batch_max_k(prec);
    for (int i = 0; i < kmax; i++)
        STAG_TRY(alloc_vec(lat, prec, &lat->bwork[prec][BATCH_MAX_G * BATCH_KMAX - 1 - i][0]));
    double best = 1e300;
    const int saved_block = lat->batch_block[prec], saved_k = lat->batch_k[prec];
    for (int K = batch_min_k(prec); K <= kmax; K *= 2)
        for (int block = 128; block <= 256; block *= 2) {
            std::vector<stag_lattice> lats(K, lat);
            std::vector<void *> x(K);
            std::vector<const void *> b(K);
            for (int i = 0; i < K; i++) {
                x[i] = lat->bwork[prec][BATCH_MAX_G * BATCH_KMAX - 1 - i][0];
                b[i] = w.p;
            }
            lat->batch_block[prec] = block;
            lat->batch_k[prec] = K;
            BatchPlan P;
            int st = plan_batch(P, K, lats.data(), x.data(), b.data(), prec);
            double us = 0;
            if (st == STAG_OK)
                st = time_launch(lat, [&]() { return launch_batch(prec, BATCH_DSLASH_X, P.a, block, s); }, reps, &us);
            P.release();
            if (st != STAG_OK) {
                lat->batch_block[prec] = saved_block;
                lat->batch_k[prec] = saved_k;
                return st;
            }
            stag_tune_result r = {STAG_TUNE_BATCH, block, 0, K, us, 0};
            res.push_back(r);
            // a smaller group must win clearly: systems that do not fill
            // whole groups leave partly empty ones, which a single-group
            // timing does not see
            const double per_rhs = us / K * (K < kmax ? 1.15 : 1.0);
            if (per_rhs < best) {
                best = per_rhs;
                c.bblock = block;
                c.bk = K;
            }
        }
    return STAG_OK;
}

static int check_tune_args(stag_lattice lat, int prec, const char *who) {
    if (!lat)
        return fail(STAG_ERR_ARG, "%s: lattice is NULL", who);
    if (!prec_valid(prec))
        return fail(STAG_ERR_ARG, "%s: bad precision %d", who, prec);
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "%s: no %s gauge copy uploaded", who, prec_name(prec));
    return STAG_OK;
}

extern "C" int stag_lattice_autotune_all(stag_lattice lat, int prec, unsigned flags, stag_tune_result *out,
                                         int cap, int *n, int *cached) {
    STAG_NVTX("stag_lattice_autotune_all");
    if (n)
        *n = 0;
    if (cached)
        *cached = 0;
    STAG_TRY(check_tune_args(lat, prec, "stag_lattice_autotune_all"));
    if (cap < 0 || (cap > 0 && !out) || (flags & ~STAG_TUNE_FORCE))
        return fail(STAG_ERR_ARG, "stag_lattice_autotune_all: bad output buffer or flags");
    DEVICE_SCOPE(lat->device);
    const std::string key = tune_key(lat, prec);
    TuneChoice c;
    bool hit = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        tune_file_read_locked();
        auto it = g_tune_cache.find(key);
        if (!(flags & STAG_TUNE_FORCE) && it != g_tune_cache.end()) {
            c = it->second;
            hit = true;
        }
    }
    std::vector<stag_tune_result> res;
    if (hit) {
        // the cached choices, untimed
        res.push_back({STAG_TUNE_DSLASH, c.dblock, c.dregs, 0, 0.0, 1});
        res.push_back({STAG_TUNE_M, c.mblock, c.mregs, 0, 0.0, 1});
        if (c.bblock > 0)
            res.push_back({STAG_TUNE_BATCH, c.bblock, 0, c.bk, 0.0, 1});
    } else {
        STAG_TRY(tune_all(lat, prec, res, c));
        for (auto &r : res)
            r.chosen = (r.kernel == STAG_TUNE_DSLASH && r.block == c.dblock && r.regs == c.dregs) ||
                       (r.kernel == STAG_TUNE_M && r.block == c.mblock && r.regs == c.mregs) ||
                       (r.kernel == STAG_TUNE_BATCH && r.block == c.bblock && r.group == c.bk);
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = c;
        tune_file_append(key, c);
    }
    apply_choice(lat, prec, c);
    const int m = (int)res.size() < cap ? (int)res.size() : cap;
    for (int k = 0; k < m; k++)
        out[k] = res[k];
    if (n)
        *n = m;
    if (cached)
        *cached = hit ? 1 : 0;
    return STAG_OK;
}

extern "C" int stag_lattice_set_tuning(stag_lattice lat, int prec, int kernel, int block, int regs, int group) {
    STAG_TRY(check_tune_args(lat, prec, "stag_lattice_set_tuning"));
    switch (kernel) {
    case STAG_TUNE_DSLASH:
    case STAG_TUNE_M:
        if ((block != 64 && block != 128 && block != 256 && block != 512) || regs < REGS_DEFAULT || regs > REGS_PAIR)
            return fail(STAG_ERR_ARG, "stag_lattice_set_tuning: block 64/128/256/512, regs 0..3");
        (kernel == STAG_TUNE_DSLASH ? lat->dslash_block : lat->mdslash_block)[prec] = block;
        (kernel == STAG_TUNE_DSLASH ? lat->dslash_regs : lat->mdslash_regs)[prec] = regs;
        return STAG_OK;
    case STAG_TUNE_BATCH:
        if (prec == STAG_F16 || (block != 128 && block != 256) ||
            (group != 0 && (group < batch_min_k(prec) || group > batch_max_k(prec) || (group & (group - 1)))))
            return fail(STAG_ERR_ARG, "stag_lattice_set_tuning: batched block 128/256, group 0 or a power of two "
                        "in [%d, %d] (no batched kernels in 16-bit storage)", batch_min_k(prec), batch_max_k(prec));
        lat->batch_block[prec] = block;
        lat->batch_k[prec] = group;
        return STAG_OK;
    default:
        return fail(STAG_ERR_ARG, "stag_lattice_set_tuning: unknown kernel %d", kernel);
    }
}

extern "C" int stag_lattice_autotune(stag_lattice lat, int prec, double *dslash_us, double *batch_us) {
    STAG_NVTX("stag_lattice_autotune");
    STAG_TRY(check_tune_args(lat, prec, "stag_lattice_autotune"));
    stag_tune_result r[64];
    int n = 0;
    STAG_TRY(stag_lattice_autotune_all(lat, prec, STAG_TUNE_FORCE, r, 64, &n, nullptr));
    // per block size of 128 and 256: the fastest register variant / group size
    for (int q = 0; q < 2; q++) {
        const int block = q ? 256 : 128;
        double bd = 0, per_rhs = 0;
        for (int k = 0; k < n; k++) {
            if (r[k].block != block)
                continue;
            if (r[k].kernel == STAG_TUNE_DSLASH && (bd == 0 || r[k].us < bd))
                bd = r[k].us;
            if (r[k].kernel == STAG_TUNE_BATCH && (per_rhs == 0 || r[k].us / r[k].group < per_rhs))
                per_rhs = r[k].us / r[k].group;
        }
        if (dslash_us)
            dslash_us[q] = bd;
        if (batch_us)  // one launch over the largest group
            batch_us[q] = per_rhs * (prec == STAG_F16 ? 0 : batch_max_k(prec));
    }
    return STAG_OK;
}

