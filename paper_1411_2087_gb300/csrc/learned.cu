// Learned gauge-covariant preconditioner (host side): the net object,
// training-pair collection from CG, training with the project's own forward
// and backward kernels and Adam, and the flexible CG that applies the net.
// Documentation in include/stag.h; the kernels are in kernels_learned.cu.
#include <algorithm>
#include <random>

#include "api_internal.h"
#include "learned.cuh"

struct stag_net_s {
    stag_lattice lat = nullptr;
    int C = 8;        // hidden channels: layers 1 -> C -> C -> 1
    NetGeom ng;
    float2 *NL = nullptr;         // net links [4][9][V]
    int nw = 0;                   // complex weights in all layers
    int off[3] = {0, 0, 0};       // complex offset of each layer's weights
    double *w = nullptr;          // master weights (re, im), device
    float *w32 = nullptr;         // FP32 copy used by the kernels
    float2 *wt = nullptr;         // adjoint weights of layers 2 and 3 (backward pass)
    double *grad = nullptr, *m = nullptr, *v = nullptr;
    int adam_t = 0;
    float2 *a0 = nullptr, *a1 = nullptr, *a2 = nullptr, *y = nullptr;  // activations
    float2 *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;                 // output gradients
    double2 *wpartial = nullptr;
    double *scal = nullptr;       // [0] loss accumulator
    // training pairs: even FP32 [3][Vh] residuals and errors, |e|^2 on the device
    std::vector<float2 *> pr, pe;
    std::vector<float2 *> slabs;
    double *enorm2 = nullptr;  // |e_k|^2 per pair
    double *rnorm2 = nullptr;  // |r_k|^2 per pair
    int enorm_cap = 0;
    int loss_kind = STAG_NET_LOSS_ERROR;
    double mass = 0;           // mass of the collected pairs (residual loss)
    // FP32 solver-layout work vectors of the residual loss: z, Mz / Mq, t (odd)
    void *fz = nullptr, *fmz = nullptr, *ft = nullptr;
    // flexible CG work vectors per precision
    void *r_old[4] = {};
    void *z[4] = {};
};

static void net_free(stag_net n) {
    void *bufs[] = {n->NL, n->w, n->w32, n->wt, n->grad, n->m, n->v, n->a0, n->a1, n->a2, n->y,
                    n->g1, n->g2, n->g3, n->wpartial, n->scal, n->enorm2, n->rnorm2,
                    n->fz, n->fmz, n->ft};
    for (void *b : bufs)
        if (b)
            cudaFree(b);
    for (float2 *p : n->slabs)
        cudaFree(p);
    for (int q = 0; q < 4; q++) {
        if (n->r_old[q])
            cudaFree(n->r_old[q]);
        if (n->z[q])
            cudaFree(n->z[q]);
    }
}

extern "C" int stag_net_create(stag_lattice lat, const double *fat, int ptr_kind, int channels, unsigned seed,
                               stag_net *out) {
    if (!out)
        return fail(STAG_ERR_ARG, "stag_net_create: out is NULL");
    *out = nullptr;
    if (!lat || !fat)
        return fail(STAG_ERR_ARG, "stag_net_create: NULL argument");
    if (channels != 1 && channels != 2 && channels != 4 && channels != 8)
        return fail(STAG_ERR_ARG, "stag_net_create: channels must be 1, 2, 4 or 8");
    if (ptr_kind != STAG_PTR_HOST && ptr_kind != STAG_PTR_DEVICE)
        return fail(STAG_ERR_ARG, "stag_net_create: bad ptr_kind %d", ptr_kind);
    DEVICE_SCOPE(lat->device);
    stag_net n = new (std::nothrow) stag_net_s();
    if (!n)
        return fail(STAG_ERR_NOMEM, "stag_net_create: host allocation failed");
    n->lat = lat;
    n->C = channels;
    for (int k = 0; k < 4; k++)
        n->ng.L[k] = lat->dims[k];
    n->ng.V = (int)lat->V;
    n->ng.step[0] = 1;
    n->ng.step[1] = lat->dims[0];
    n->ng.step[2] = lat->dims[0] * lat->dims[1];
    n->ng.step[3] = lat->dims[0] * lat->dims[1] * lat->dims[2];
    const int C = channels;
    n->off[0] = 0;
    n->off[1] = 9 * C;
    n->off[2] = 9 * C + 9 * C * C;
    n->nw = 9 * C + 9 * C * C + 9 * C;
    const size_t V = (size_t)lat->V;
    cudaStream_t s = lat->stream;
    auto bail = [&](cudaError_t e) {
        cudaStreamSynchronize(s);
        net_free(n);
        delete n;
        return fail(e == cudaErrorMemoryAllocation ? STAG_ERR_NOMEM : STAG_ERR_CUDA, "stag_net_create: %s",
                    cudaGetErrorString(e));
    };
    cudaError_t e;
    if (ptr_kind == STAG_PTR_DEVICE && (e = cudaDeviceSynchronize()) != cudaSuccess)
        return bail(e);
    const size_t nr = 2 * (size_t)n->nw;
    if ((e = cudaMalloc(&n->NL, sizeof(float2) * 36 * V)) != cudaSuccess ||
        (e = cudaMalloc(&n->w, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->w32, sizeof(float) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->wt, sizeof(float2) * n->nw)) != cudaSuccess ||
        (e = cudaMalloc(&n->grad, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->m, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->v, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->a0, sizeof(float2) * 3 * V)) != cudaSuccess ||
        (e = cudaMalloc(&n->a1, sizeof(float2) * 3 * V * C)) != cudaSuccess ||
        (e = cudaMalloc(&n->a2, sizeof(float2) * 3 * V * C)) != cudaSuccess ||
        (e = cudaMalloc(&n->y, sizeof(float2) * 3 * V)) != cudaSuccess ||
        (e = cudaMalloc(&n->g1, sizeof(float2) * 3 * V * C)) != cudaSuccess ||
        (e = cudaMalloc(&n->g2, sizeof(float2) * 3 * V * C)) != cudaSuccess ||
        (e = cudaMalloc(&n->g3, sizeof(float2) * 3 * V)) != cudaSuccess ||
        (e = cudaMalloc(&n->wpartial, sizeof(double2) * wgrad_partial_blocks() * 9 * C * C)) != cudaSuccess ||
        (e = cudaMalloc(&n->scal, sizeof(double) * 4)) != cudaSuccess)
        return bail(e);
    // net links from the raw fat links
    double *fat_d = (double *)fat;
    bool owned = false;
    if (ptr_kind == STAG_PTR_HOST) {
        const size_t bytes = 4 * V * 18 * sizeof(double);
        if ((e = cudaMalloc(&fat_d, bytes)) != cudaSuccess)
            return bail(e);
        owned = true;
        if ((e = cudaMemcpyAsync(fat_d, fat, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
            cudaFree(fat_d);
            return bail(e);
        }
    }
    e = launch_net_links(n->ng, lat->bc, fat_d, n->NL, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (owned)
        cudaFree(fat_d);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return bail(e != cudaSuccess ? e : e2);
    // initial weights: the identity map plus seeded noise of 1e-2
    std::vector<double> w(nr, 0.0);
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1e-2);
    for (auto &v : w)
        v = nd(rng);
    auto W = [&](int layer, int d, int o, int i) -> double & {
        const int cin = layer == 0 ? 1 : C, cout = layer == 2 ? 1 : C;
        return w[2 * (size_t)(n->off[layer] + (d * cout + o) * cin + i)];
    };
    for (int o = 0; o < C; o++) {
        W(0, 0, o, 0) += 1.0;
        W(1, 0, o, o) += 1.0;
        W(2, 0, 0, o) += 1.0 / C;
    }
    std::vector<float> w32(w.begin(), w.end());
    if ((e = cudaMemcpy(n->w, w.data(), sizeof(double) * nr, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(n->w32, w32.data(), sizeof(float) * nr, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(n->m, 0, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMemset(n->v, 0, sizeof(double) * nr)) != cudaSuccess)
        return bail(e);
    lat->live_fields++;  // the lattice outlives its nets
    *out = n;
    return STAG_OK;
}

extern "C" int stag_net_destroy(stag_net n) {
    if (!n)
        return STAG_OK;
    DEVICE_SCOPE(n->lat->device);
    cudaStreamSynchronize(n->lat->stream);
    net_free(n);
    n->lat->live_fields--;
    delete n;
    return STAG_OK;
}

extern "C" int stag_net_num_weights(const stag_net n, int *count) {
    if (!n || !count)
        return fail(STAG_ERR_ARG, "stag_net_num_weights: NULL argument");
    *count = n->nw;
    return STAG_OK;
}

extern "C" int stag_net_set_weights(stag_net n, const double *w) {
    if (!n)
        return fail(STAG_ERR_ARG, "stag_net_set_weights: NULL net");
    if (!w)
        return STAG_OK;
    DEVICE_SCOPE(n->lat->device);
    const size_t nr = 2 * (size_t)n->nw;
    for (size_t k = 0; k < nr; k++)
        if (!std::isfinite(w[k]))
            return fail(STAG_ERR_ARG, "stag_net_set_weights: weight %zu is not finite", k);
    std::vector<float> w32(w, w + nr);
    CUDA_TRY(cudaMemcpy(n->w, w, sizeof(double) * nr, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(n->w32, w32.data(), sizeof(float) * nr, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(n->m, 0, sizeof(double) * nr));
    CUDA_TRY(cudaMemset(n->v, 0, sizeof(double) * nr));
    n->adam_t = 0;
    return STAG_OK;
}

extern "C" int stag_net_get_weights(const stag_net n, double *w) {
    if (!n || !w)
        return fail(STAG_ERR_ARG, "stag_net_get_weights: NULL argument");
    DEVICE_SCOPE(n->lat->device);
    CUDA_TRY(cudaMemcpy(w, n->w, sizeof(double) * 2 * n->nw, cudaMemcpyDeviceToHost));
    return STAG_OK;
}

static const float2 *wl(const stag_net n, int layer) { return (const float2 *)n->w32 + n->off[layer]; }

// y = net(a0) through the three layers (a0 must already hold the input,
// zero on odd sites).  even_out: only the even sites of y are computed (all
// a preconditioner needs).
static cudaError_t net_forward(stag_net n, int round_half, const int *gate, cudaStream_t s, bool even_out = false) {
    cudaError_t e;
    const int C = n->C;
    if ((e = launch_covconv(1, C, n->ng, n->NL, wl(n, 0), round_half, n->a0, n->a1, gate, s, 0, -1)) != cudaSuccess)
        return e;
    if ((e = launch_covconv(C, C, n->ng, n->NL, wl(n, 1), round_half, n->a1, n->a2, gate, s)) != cudaSuccess)
        return e;
    return launch_covconv(C, 1, n->ng, n->NL, wl(n, 2), round_half, n->a2, n->y, gate, s, -1, even_out ? 0 : -1);
}

// dL/dW* += gradient of the loss of one pair whose output gradient is in g3
static cudaError_t net_backward(stag_net n, cudaStream_t s) {
    cudaError_t e;
    const int C = n->C;
    double2 *gr = (double2 *)n->grad;
    // adjoint weights of layers 3 and 2
    float2 *wt3 = n->wt + n->off[2];
    float2 *wt2 = n->wt + n->off[1];
    if ((e = launch_net_adjoint(C, 1, wl(n, 2), wt3, s)) != cudaSuccess ||
        (e = launch_net_adjoint(C, C, wl(n, 1), wt2, s)) != cudaSuccess)
        return e;
    if ((e = launch_covconv_wgrad(C, 1, n->ng, n->NL, n->a2, n->g3, n->wpartial, gr + n->off[2], s)) != cudaSuccess)
        return e;
    if ((e = launch_covconv(1, C, n->ng, n->NL, wt3, 0, n->g3, n->g2, nullptr, s)) != cudaSuccess)
        return e;
    if ((e = launch_covconv_wgrad(C, C, n->ng, n->NL, n->a1, n->g2, n->wpartial, gr + n->off[1], s)) != cudaSuccess)
        return e;
    if ((e = launch_covconv(C, C, n->ng, n->NL, wt2, 0, n->g2, n->g1, nullptr, s)) != cudaSuccess)
        return e;
    return launch_covconv_wgrad(1, C, n->ng, n->NL, n->a0, n->g1, n->wpartial, gr + n->off[0], s);
}

// ---- applying the net to solver fields --------------------------------
static int check_net_field(const stag_net n, const stag_field f, const char *who) {
    if (!f || f->lat != n->lat || f->parity != STAG_EVEN)
        return fail(STAG_ERR_ARG, "%s: fields must be even fields of the net's lattice", who);
    if (f->prec != STAG_F64 && f->prec != STAG_DF64 && f->prec != STAG_F32)
        return fail(STAG_ERR_ARG, "%s: fields must be F64, DF64 or F32", who);
    return STAG_OK;
}

static cudaError_t net_apply_raw(stag_net n, int prec, const void *in, void *out, int round_half, const int *gate,
                                 cudaStream_t s) {
    cudaError_t e;
    if ((e = launch_solver_to_full(prec, n->ng, n->lat->geom, in, n->a0, gate, s)) != cudaSuccess)
        return e;
    if ((e = net_forward(n, round_half, gate, s, true)) != cudaSuccess)
        return e;
    return launch_full_to_solver(prec, n->ng, n->lat->geom, n->y, out, gate, s);
}

extern "C" int stag_net_apply(stag_net n, stag_field out_even, const stag_field in_even, int fp16_weights) {
    STAG_NVTX("stag_net_apply");
    if (!n)
        return fail(STAG_ERR_ARG, "stag_net_apply: NULL net");
    STAG_TRY(check_net_field(n, out_even, "stag_net_apply"));
    STAG_TRY(check_net_field(n, in_even, "stag_net_apply"));
    if (out_even->prec != in_even->prec)
        return fail(STAG_ERR_ARG, "stag_net_apply: precision mismatch");
    DEVICE_SCOPE(n->lat->device);
    CUDA_TRY(net_apply_raw(n, in_even->prec, in_even->data, out_even->data, fp16_weights ? 1 : 0, nullptr,
                           n->lat->stream));
    return STAG_OK;
}

// ---- training pairs -----------------------------------------------------
static int add_pair_slab(stag_net n, int count) {
    const size_t Vh = (size_t)n->lat->Vh;
    float2 *slab = nullptr;
    CUDA_TRY(cudaMalloc(&slab, sizeof(float2) * 3 * Vh * 2 * (size_t)count));
    n->slabs.push_back(slab);
    for (int k = 0; k < count; k++) {
        n->pr.push_back(slab + (size_t)(2 * k) * 3 * Vh);
        n->pe.push_back(slab + (size_t)(2 * k + 1) * 3 * Vh);
    }
    return STAG_OK;
}

static int refresh_enorms(stag_net n) {
    const int np = (int)n->pe.size();
    if (np > n->enorm_cap) {
        if (n->enorm2)
            cudaFree(n->enorm2);
        if (n->rnorm2)
            cudaFree(n->rnorm2);
        n->enorm2 = n->rnorm2 = nullptr;
        CUDA_TRY(cudaMalloc(&n->enorm2, sizeof(double) * np));
        CUDA_TRY(cudaMalloc(&n->rnorm2, sizeof(double) * np));
        n->enorm_cap = np;
    }
    cudaStream_t s = n->lat->stream;
    CUDA_TRY(cudaMemsetAsync(n->enorm2, 0, sizeof(double) * np, s));
    CUDA_TRY(cudaMemsetAsync(n->rnorm2, 0, sizeof(double) * np, s));
    for (int k = 0; k < np; k++) {
        CUDA_TRY(launch_pair_norm2((int)(3 * n->lat->Vh), n->pe[k], n->enorm2 + k, s));
        CUDA_TRY(launch_pair_norm2((int)(3 * n->lat->Vh), n->pr[k], n->rnorm2 + k, s));
    }
    return STAG_OK;
}

// y holds N(r) (full); g3 <- gradient of |M z - r|^2 / |r|^2 with respect to
// conj(y), z = y on even sites: M (M z - r) / |r|^2 (M Hermitian), FP32
static int resid_loss_grad(stag_net n, int p, cudaStream_t s) {
    stag_lattice lat = n->lat;
    const int P = STAG_F32;
    const Geom &g = lat->geom;
    CUDA_TRY(launch_full_to_solver(P, n->ng, g, n->y, n->fz, nullptr, s));
    // Mz
    DslashArgs a1 = dslash_args(lat, P, STAG_ODD, n->fz, n->ft);
    CUDA_TRY(launch_dslash(P, EPI_NONE, a1, lat->dslash_block[P], s));
    DslashArgs a2 = dslash_args(lat, P, STAG_EVEN, n->ft, n->fmz);
    a2.p = n->fz;
    a2.m2 = make_dpair(n->mass * n->mass);
    a2.m2_in_args = 1;
    CUDA_TRY(launch_dslash(P, EPI_M, a2, lat->dslash_block[P], s));
    CUDA_TRY(launch_solver_to_full(P, n->ng, g, n->fmz, n->g3, nullptr, s));
    // q = Mz - r (into g3), loss
    CUDA_TRY(launch_resid_loss(n->ng, n->g3, n->a0, n->rnorm2 + p, n->scal, s));
    // M q / |r|^2
    CUDA_TRY(launch_full_to_solver(P, n->ng, g, n->g3, n->fz, nullptr, s));
    DslashArgs a3 = dslash_args(lat, P, STAG_ODD, n->fz, n->ft);
    CUDA_TRY(launch_dslash(P, EPI_NONE, a3, lat->dslash_block[P], s));
    DslashArgs a4 = dslash_args(lat, P, STAG_EVEN, n->ft, n->fmz);
    a4.p = n->fz;
    a4.m2 = make_dpair(n->mass * n->mass);
    a4.m2_in_args = 1;
    CUDA_TRY(launch_dslash(P, EPI_M, a4, lat->dslash_block[P], s));
    CUDA_TRY(launch_solver_to_full(P, n->ng, g, n->fmz, n->g3, nullptr, s));
    CUDA_TRY(launch_scale_full(n->ng, n->g3, n->rnorm2 + p, s));
    return STAG_OK;
}

// CG iterates of a run from x = 0 become training pairs (r_k, e_k = x* - x_k):
// the solve to rel_tol gives x*, a second run, driven from the host, stops
// every `stride` iterations to record the pair.
extern "C" int stag_net_collect_pairs(stag_net n, const stag_field b, double mass, double rel_tol, int stride,
                                      int max_pairs, int *collected) {
    STAG_NVTX("stag_net_collect_pairs");
    if (collected)
        *collected = 0;
    if (!n || !b)
        return fail(STAG_ERR_ARG, "stag_net_collect_pairs: NULL argument");
    STAG_TRY(check_net_field(n, b, "stag_net_collect_pairs"));
    if (!(mass > 0) || !(rel_tol > 0) || stride < 1 || max_pairs < 1)
        return fail(STAG_ERR_ARG, "stag_net_collect_pairs: need mass > 0, rel_tol > 0, stride >= 1, max_pairs >= 1");
    stag_lattice lat = n->lat;
    const int prec = b->prec;
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_net_collect_pairs: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    // x* by the plain CG
    stag_field xs = nullptr;
    STAG_TRY(stag_field_create(lat, STAG_EVEN, prec, &xs));
    stag_solve_info info;
    int st = stag_cg_solve(lat, xs, b, mass, rel_tol, 100000, &info);
    if (st != STAG_OK) {
        stag_field_destroy(xs);
        return st;
    }
    const int total_iters = info.iters;
    // snapshots strictly before convergence (e_k = 0 at the last iterate)
    int want = (total_iters - 1) / stride;
    if (want > max_pairs)
        want = max_pairs;
    if (want < 1) {
        stag_field_destroy(xs);
        return fail(STAG_ERR_ARG, "stag_net_collect_pairs: stride %d exceeds the %d iterations of the solve",
                    stride, total_iters);
    }
    st = add_pair_slab(n, want);
    if (st != STAG_OK) {
        stag_field_destroy(xs);
        return st;
    }
    const int first = (int)n->pr.size() - want;
    n->mass = mass;
    // the second run: same kernels, same order, so the same iterates
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    cudaError_t e = cudaMemcpyAsync(w.bw, b->data, b->bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        st = upload_scalars(lat, mass, rel_tol, 100000, false, 0);
    if (e == cudaSuccess && st == STAG_OK)
        e = launch_cg_init(prec, lat->geom, w.xw, w.r, w.p, w.bw, lat->partial, lat->sc, s);
    int got = 0;
    for (int k = 0; e == cudaSuccess && st == STAG_OK && got < want; k++) {
        for (int j = 0; j < stride && e == cudaSuccess; j++)
            e = enqueue_cg_body(lat, w, s, true);
        if (e != cudaSuccess)
            break;
        // pair: r_k (the iterated residual) and e_k = x* - x_k
        e = launch_solver_to_pair(prec, lat->geom, w.r, nullptr, n->pr[first + got], s);
        if (e == cudaSuccess)
            e = launch_solver_to_pair(prec, lat->geom, xs->data, w.xw, n->pe[first + got], s);
        got++;
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    stag_field_destroy(xs);
    if (e == cudaSuccess)
        e = e2;
    if (e != cudaSuccess)
        return fail(STAG_ERR_CUDA, "stag_net_collect_pairs: %s", cudaGetErrorString(e));
    if (st != STAG_OK)
        return st;
    STAG_TRY(refresh_enorms(n));
    if (collected)
        *collected = got;
    return STAG_OK;
}

extern "C" int stag_net_get_pair(const stag_net n, int k, double *r, double *e) {
    if (!n || !r || !e)
        return fail(STAG_ERR_ARG, "stag_net_get_pair: NULL argument");
    if (k < 0 || k >= (int)n->pr.size())
        return fail(STAG_ERR_ARG, "stag_net_get_pair: pair %d of %zu", k, n->pr.size());
    DEVICE_SCOPE(n->lat->device);
    const size_t Vh = (size_t)n->lat->Vh;
    std::vector<float2> h(3 * Vh);
    for (int which = 0; which < 2; which++) {
        CUDA_TRY(cudaMemcpy(h.data(), which ? n->pe[k] : n->pr[k], sizeof(float2) * 3 * Vh, cudaMemcpyDeviceToHost));
        double *dst = which ? e : r;
        for (size_t c = 0; c < Vh; c++)
            for (int a = 0; a < 3; a++) {
                dst[(3 * c + a) * 2] = h[a * Vh + c].x;
                dst[(3 * c + a) * 2 + 1] = h[a * Vh + c].y;
            }
    }
    return STAG_OK;
}

extern "C" int stag_net_set_loss(stag_net n, int kind) {
    if (!n)
        return fail(STAG_ERR_ARG, "stag_net_set_loss: NULL net");
    if (kind != STAG_NET_LOSS_ERROR && kind != STAG_NET_LOSS_RESIDUAL)
        return fail(STAG_ERR_ARG, "stag_net_set_loss: unknown loss %d", kind);
    if (kind == STAG_NET_LOSS_RESIDUAL) {
        stag_lattice lat = n->lat;
        if (!lat->has_gauge || !lat->links[STAG_F32])
            return fail(STAG_ERR_STATE, "stag_net_set_loss: the residual loss needs an F32 gauge copy");
        DEVICE_SCOPE(lat->device);
        STAG_TRY(alloc_vec(lat, STAG_F32, &n->fz));
        STAG_TRY(alloc_vec(lat, STAG_F32, &n->fmz));
        STAG_TRY(alloc_vec(lat, STAG_F32, &n->ft));
    }
    n->loss_kind = kind;
    return STAG_OK;
}

extern "C" int stag_net_num_pairs(const stag_net n, int *count) {
    if (!n || !count)
        return fail(STAG_ERR_ARG, "stag_net_num_pairs: NULL argument");
    *count = (int)n->pr.size();
    return STAG_OK;
}

// ---- training -------------------------------------------------------------
// loss and dL/dW* summed over pairs [first, first + count)
static int loss_grad_range(stag_net n, const int *idx, int count, double *loss) {
    cudaStream_t s = n->lat->stream;
    CUDA_TRY(cudaMemsetAsync(n->grad, 0, sizeof(double) * 2 * n->nw, s));
    CUDA_TRY(cudaMemsetAsync(n->scal, 0, sizeof(double), s));
    for (int k = 0; k < count; k++) {
        const int p = idx[k];
        CUDA_TRY(launch_pair_to_full(n->ng, n->pr[p], n->a0, s));
        CUDA_TRY(net_forward(n, 0, nullptr, s));
        if (n->loss_kind == STAG_NET_LOSS_RESIDUAL)
            STAG_TRY(resid_loss_grad(n, p, s));
        else
            CUDA_TRY(launch_pair_loss(n->ng, n->y, n->pe[p], n->enorm2 + p, n->g3, n->scal, s));
        CUDA_TRY(net_backward(n, s));
    }
    if (loss) {
        CUDA_TRY(cudaMemcpyAsync(loss, n->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    return STAG_OK;
}

extern "C" int stag_net_loss_grad(stag_net n, int first, int count, double *loss, double *grad) {
    if (!n)
        return fail(STAG_ERR_ARG, "stag_net_loss_grad: NULL net");
    if (first < 0 || count < 1 || first + count > (int)n->pr.size())
        return fail(STAG_ERR_ARG, "stag_net_loss_grad: pair range [%d, %d) outside the %zu collected pairs", first,
                    first + count, n->pr.size());
    DEVICE_SCOPE(n->lat->device);
    std::vector<int> idx(count);
    for (int k = 0; k < count; k++)
        idx[k] = first + k;
    double l = 0;
    STAG_TRY(loss_grad_range(n, idx.data(), count, &l));
    if (loss)
        *loss = l;
    if (grad)
        CUDA_TRY(cudaMemcpy(grad, n->grad, sizeof(double) * 2 * n->nw, cudaMemcpyDeviceToHost));
    return STAG_OK;
}

// Warm start of the residual loss: the scale s minimising sum |s M N(r) - r|^2
// over the pairs, s = sum Re<M N r, r> / sum |M N r|^2, folded into the last
// layer's weights
static int residual_warm_start(stag_net n) {
    stag_lattice lat = n->lat;
    cudaStream_t s = lat->stream;
    const int P = STAG_F32;
    const Geom &g = lat->geom;
    CUDA_TRY(cudaMemsetAsync(n->scal + 1, 0, 2 * sizeof(double), s));
    for (size_t p = 0; p < n->pr.size(); p++) {
        CUDA_TRY(launch_pair_to_full(n->ng, n->pr[p], n->a0, s));
        CUDA_TRY(net_forward(n, 0, nullptr, s));
        CUDA_TRY(launch_full_to_solver(P, n->ng, g, n->y, n->fz, nullptr, s));
        DslashArgs a1 = dslash_args(lat, P, STAG_ODD, n->fz, n->ft);
        CUDA_TRY(launch_dslash(P, EPI_NONE, a1, lat->dslash_block[P], s));
        DslashArgs a2 = dslash_args(lat, P, STAG_EVEN, n->ft, n->fmz);
        a2.p = n->fz;
        a2.m2 = make_dpair(n->mass * n->mass);
        a2.m2_in_args = 1;
        CUDA_TRY(launch_dslash(P, EPI_M, a2, lat->dslash_block[P], s));
        CUDA_TRY(launch_solver_to_full(P, n->ng, g, n->fmz, n->g3, nullptr, s));
        CUDA_TRY(launch_dot2_full(3 * n->ng.V, n->g3, n->a0, n->scal + 1, s));
    }
    double h[2];
    CUDA_TRY(cudaMemcpyAsync(h, n->scal + 1, sizeof h, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (!(h[1] > 0) || !std::isfinite(h[0]))
        return STAG_OK;
    const double scale = h[0] / h[1];
    std::vector<double> w(2 * (size_t)n->nw);
    STAG_TRY(stag_net_get_weights(n, w.data()));
    for (int k = 2 * n->off[2]; k < 2 * n->nw; k++)
        w[k] *= scale;
    return stag_net_set_weights(n, w.data());
}

extern "C" int stag_net_train(stag_net n, int epochs, int batch, double lr, unsigned seed, double *epoch_loss) {
    STAG_NVTX("stag_net_train");
    if (!n)
        return fail(STAG_ERR_ARG, "stag_net_train: NULL net");
    const int np = (int)n->pr.size();
    if (np < 1)
        return fail(STAG_ERR_STATE, "stag_net_train: no training pairs collected");
    if (epochs < 1 || batch < 1 || !(lr > 0))
        return fail(STAG_ERR_ARG, "stag_net_train: need epochs >= 1, batch >= 1, lr > 0");
    DEVICE_SCOPE(n->lat->device);
    std::mt19937_64 rng(seed);
    std::vector<int> order(np);
    for (int k = 0; k < np; k++)
        order[k] = k;
    cudaStream_t s = n->lat->stream;
    if (n->loss_kind == STAG_NET_LOSS_RESIDUAL && n->adam_t == 0)
        STAG_TRY(residual_warm_start(n));
    for (int ep = 0; ep < epochs; ep++) {
        std::shuffle(order.begin(), order.end(), rng);
        // cosine decay of the step size from lr to lr / 10
        const double lr_ep = lr * (0.1 + 0.45 * (1.0 + std::cos(M_PI * ep / epochs)));
        double tot = 0;
        for (int b0 = 0; b0 < np; b0 += batch) {
            const int cnt = std::min(batch, np - b0);
            double l = 0;
            STAG_TRY(loss_grad_range(n, order.data() + b0, cnt, &l));
            tot += l;
            n->adam_t++;
            CUDA_TRY(launch_adam(2 * n->nw, n->w, n->grad, n->m, n->v, lr_ep / cnt, n->adam_t, n->w32, s));
        }
        if (epoch_loss)
            epoch_loss[ep] = tot / np;
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    return STAG_OK;
}

// ---- flexible CG with the net as preconditioner -------------------------
static const int *status_flag(stag_lattice lat) {
    return (const int *)((const char *)lat->sc + offsetof(CgScalars, status));
}

// enqueue z = N(r) (or z = r without the net)
static cudaError_t precondition(stag_net n, int prec, bool use_net, const void *r, void *z, const int *gate,
                                cudaStream_t s) {
    if (use_net)
        return net_apply_raw(n, prec, r, z, 1, gate, s);
    return cudaMemcpyAsync(z, r, field_bytes(n->lat, prec), cudaMemcpyDeviceToDevice, s);
}

// one run of flexible CG from the current x (r = b - M x recomputed):
// returns the CG status code of the run
static int fcg_run(stag_net n, int prec, bool use_net, double mass, double tol2bb, int max_iter, int chunk,
                   int *iters, double *rr_out) {
    stag_lattice lat = n->lat;
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    const Geom &g = lat->geom;
    const int *gate = status_flag(lat);
    // scalars: m^2, rr_stop, status RUNNING, iter 0
    {
        CgScalars h;
        memset(&h, 0, sizeof h);
        h.m2 = make_dpair(mass * mass);
        h.max_iter = max_iter;
        h.rr_stop = tol2bb;
        h.tol2 = 0;
        CUDA_TRY(cudaMemcpyAsync(lat->sc, &h, sizeof h, cudaMemcpyHostToDevice, s));
    }
    // r = b - M x (true residual) and |r|^2 into true_rr
    DslashArgs a1 = dslash_args(lat, prec, STAG_ODD, w.xw, w.t);
    CUDA_TRY(launch_dslash(prec, EPI_NONE, a1, lat->dslash_block[prec], s));
    DslashArgs a2 = dslash_args(lat, prec, STAG_EVEN, w.t, w.r);
    a2.p = w.xw;
    a2.b = w.bw;
    CUDA_TRY(launch_dslash(prec, EPI_RESID_STORE, a2, lat->dslash_block[prec], s));
    // z = N(r); rr = <z, r>; p = z
    CUDA_TRY(precondition(n, prec, use_net, w.r, n->z[prec], gate, s));
    CUDA_TRY(launch_fcg_beta(prec, g, n->z[prec], w.r, nullptr, lat->partial, lat->sc, 1, s));
    CUDA_TRY(cudaMemcpyAsync(w.p, n->z[prec], field_bytes(lat, prec), cudaMemcpyDeviceToDevice, s));
    const long long max_chunks = (long long)max_iter / chunk + 2;
    for (long long k = 0; k < max_chunks; k++) {
        CUDA_TRY(cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (lat->sc_host->status != CG_RUNNING || lat->sc_host->true_rr <= tol2bb)
            break;
        for (int j = 0; j < chunk; j++) {
            // Ap = M p, alpha = <r, z> / <p, Ap>
            DslashArgs b1 = dslash_args(lat, prec, STAG_ODD, w.p, w.t);
            b1.skip_if_done = 1;
            CUDA_TRY(launch_dslash(prec, EPI_NONE, b1, lat->dslash_block[prec], s));
            CUDA_TRY(enqueue_m_pap(lat, prec, w.t, w.Ap, w.p, true, s));
            CUDA_TRY(launch_fcg_update(prec, g, w.xw, w.r, n->r_old[prec], w.p, w.Ap, lat->partial, lat->sc, s));
            CUDA_TRY(precondition(n, prec, use_net, w.r, n->z[prec], gate, s));
            CUDA_TRY(launch_fcg_beta(prec, g, n->z[prec], w.r, n->r_old[prec], lat->partial, lat->sc, 0, s));
            CUDA_TRY(launch_cg_p_update(prec, g, n->z[prec], w.p, lat->sc, s));
        }
    }
    CUDA_TRY(cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *iters = lat->sc_host->iter;
    *rr_out = lat->sc_host->fcg_rr;
    if (lat->sc_host->true_rr <= tol2bb)
        return CG_CONVERGED;
    return lat->sc_host->status;
}

extern "C" int stag_cg_solve_learned(stag_net n, stag_field x, const stag_field b, double mass, double rel_tol,
                                     int max_iter, stag_solve_info *info) {
    STAG_NVTX("stag_cg_solve_learned");
    if (info)
        memset(info, 0, sizeof *info);
    if (!n || !x || !b)
        return fail(STAG_ERR_ARG, "stag_cg_solve_learned: NULL argument");
    STAG_TRY(check_net_field(n, x, "stag_cg_solve_learned"));
    STAG_TRY(check_net_field(n, b, "stag_cg_solve_learned"));
    if (x->prec != b->prec || x == b)
        return fail(STAG_ERR_ARG, "stag_cg_solve_learned: x and b must be distinct fields of one precision");
    if (!(mass > 0) || !std::isfinite(mass) || !(rel_tol >= 0) || max_iter < 0)
        return fail(STAG_ERR_ARG, "stag_cg_solve_learned: need mass > 0, rel_tol >= 0, max_iter >= 0");
    stag_lattice lat = n->lat;
    const int prec = x->prec;
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_cg_solve_learned: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    const auto t0 = std::chrono::steady_clock::now();
    STAG_TRY(ensure_cg_work(lat, prec));
    STAG_TRY(alloc_vec(lat, prec, &n->r_old[prec]));
    STAG_TRY(alloc_vec(lat, prec, &n->z[prec]));
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    CUDA_TRY(cudaMemcpyAsync(w.bw, b->data, b->bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemsetAsync(w.xw, 0, field_bytes(lat, prec), s));
    // |b|^2: the residual of x = 0
    double bb = 0;
    STAG_TRY(shifted_residual(lat, prec, w.xw, w.bw, mass, nullptr, &bb));
    const double tol2bb = rel_tol * rel_tol * bb;
    int iters = 0, fallbacks = 0, status = CG_CONVERGED;
    double rr = 0;
    double rr_true = bb;
    if (bb > 0) {
        // flexible CG with the net.  A run that claims convergence on its
        // iterated residual is checked against the recomputed one and
        // restarted (with the net) if the two drifted apart; after a
        // breakdown, a stall or the iteration limit, plain CG (z = r)
        // continues from the current x.
        int it = 0;
        bool use_net = true;
        for (int attempt = 0; attempt < 4 && iters <= max_iter; attempt++) {
            status = fcg_run(n, prec, use_net, mass, tol2bb, max_iter - iters, use_net ? 8 : 32, &it, &rr);
            if (status < 0)
                return status;
            iters += it;
            STAG_TRY(shifted_residual(lat, prec, w.xw, w.bw, mass, nullptr, &rr_true));
            if (rr_true <= tol2bb)
                break;
            if (status != CG_CONVERGED) {
                if (use_net)
                    fallbacks++;
                use_net = false;
            }
        }
    }
    CUDA_TRY(cudaMemcpyAsync(x->data, w.xw, x->bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    stag_solve_info local;
    memset(&local, 0, sizeof local);
    local.iters = iters;
    local.restarts = fallbacks;
    local.true_rel_resid = bb > 0 ? std::sqrt(rr_true / bb) : 0.0;
    local.iter_rel_resid = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    local.status = (bb == 0 || local.true_rel_resid <= rel_tol * 1.0000001) ? STAG_OK
                   : status == CG_BREAKDOWN ? STAG_ERR_BREAKDOWN
                                            : STAG_ERR_NOT_CONVERGED;
    if (info)
        *info = local;
    if (local.status != STAG_OK)
        return fail(local.status, "stag_cg_solve_learned: true |r|/|b| = %.3e after %d iterations",
                    local.true_rel_resid, iters);
    return STAG_OK;
}
