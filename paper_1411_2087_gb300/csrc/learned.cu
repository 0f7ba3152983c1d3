// Learned gauge-covariant preconditioner (host side): the net object,
// training-pair collection from CG, training with the project's own forward
// and backward kernels and Adam, and the flexible CG that applies the net.
// Documentation in include/stag.h.  The net is evaluated and differentiated
// in its path form (kernels_netpath.cu): its weights are the three layers',
// and every forward pass first turns them into the 65 coefficients of the
// two-hop path sum that the layers compose to on even fields.
#include <algorithm>
#include <random>

#include "api_internal.h"
#include "learned.cuh"

struct stag_net_s {
    stag_lattice lat = nullptr;
    int C = 8;                    // hidden channels: layers 1 -> C -> C -> 1
    float2 *NL32 = nullptr;       // net links, FP32 [2][4][9][stride]
    short2 *NL16 = nullptr;       // the same in 16-bit fixed point
    void *NL12 = nullptr;         // 16-bit rows 0 and 1 (special unitary fat links only)
    float scale16 = 0.f;          // 16-bit value = q * scale16
    int bcneg = 0;                // bit mu: boundary sign of direction mu is -1
    int nw = 0;                   // complex weights in all layers
    int off[3] = {0, 0, 0};       // complex offset of each layer's weights
    double *w = nullptr;          // master weights (re, im), device
    float *w32 = nullptr;         // FP32 copy used by the kernels
    double *grad = nullptr, *m = nullptr, *v = nullptr;
    int adam_t = 0;
    NetPath *path = nullptr;      // path coefficients of the current weights
    float2 *chi = nullptr;        // odd-site intermediate [8][3][stride]
    double2 *G = nullptr;         // dL/dC* (64) and dL/dc0* (1), summed over pairs
    double2 *gpartial = nullptr;  // per-block partials of G
    double *scal = nullptr;       // [0] loss accumulator, [1..2] warm-start sums
    // training pairs: even FP32 [3][Vh] residuals and errors
    std::vector<float2 *> pr, pe;
    std::vector<float2 *> slabs;
    double *enorm2 = nullptr;  // |e_k|^2 per pair
    double *rnorm2 = nullptr;  // |r_k|^2 per pair
    int enorm_cap = 0;
    int loss_kind = STAG_NET_LOSS_ERROR;
    double mass = 0;           // mass of the collected pairs (residual loss)
    // FP32 solver-layout work vectors of the losses: z, Mz / g, t (odd)
    void *fz = nullptr, *fmz = nullptr, *ft = nullptr;
    // flexible CG: preconditioned residual per precision
    void *z[4] = {};
};

static void net_free(stag_net n) {
    void *bufs[] = {n->NL32, n->NL16, n->NL12, n->w, n->w32, n->grad, n->m, n->v, n->path, n->chi, n->G, n->gpartial,
                    n->scal, n->enorm2, n->rnorm2, n->fz, n->fmz, n->ft};
    for (void *b : bufs)
        if (b)
            cudaFree(b);
    for (float2 *p : n->slabs)
        cudaFree(p);
    for (int q = 0; q < 4; q++)
        if (n->z[q])
            cudaFree(n->z[q]);
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
    const int C = channels;
    n->off[0] = 0;
    n->off[1] = 9 * C;
    n->off[2] = 9 * C + 9 * C * C;
    n->nw = 9 * C + 9 * C * C + 9 * C;
    const size_t V = (size_t)lat->V;
    const size_t S = (size_t)lat->geom.stride;
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
    if ((e = cudaMalloc(&n->NL32, sizeof(float2) * 2 * 4 * 9 * S)) != cudaSuccess ||
        (e = cudaMalloc(&n->NL16, sizeof(short2) * 2 * 4 * 9 * S)) != cudaSuccess ||
        (e = cudaMalloc(&n->w, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->w32, sizeof(float) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->grad, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->m, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->v, sizeof(double) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&n->path, sizeof(NetPath))) != cudaSuccess ||
        (e = cudaMalloc(&n->chi, sizeof(float2) * 8 * 3 * S)) != cudaSuccess ||
        (e = cudaMalloc(&n->G, sizeof(double2) * 65)) != cudaSuccess ||
        (e = cudaMalloc(&n->gpartial, sizeof(double2) * 65 * net_grad_blocks(lat->geom))) != cudaSuccess ||
        (e = cudaMalloc(&n->scal, sizeof(double) * 4)) != cudaSuccess)
        return bail(e);
    // the padding sites of the link planes are never read; zero them anyway
    if ((e = cudaMemsetAsync(n->NL32, 0, sizeof(float2) * 2 * 4 * 9 * S, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(n->NL16, 0, sizeof(short2) * 2 * 4 * 9 * S, s)) != cudaSuccess)
        return bail(e);
    {
        int st = alloc_vec(lat, STAG_F32, &n->fz);
        if (st == STAG_OK)
            st = alloc_vec(lat, STAG_F32, &n->fmz);
        if (st != STAG_OK) {
            cudaStreamSynchronize(s);
            net_free(n);
            delete n;
            return st;
        }
    }
    // net links from the raw fat links (phases and boundary sign folded in)
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
    // the 16-bit copy's scale: the largest |re| or |im| of the field
    unsigned *amax_d = (unsigned *)(n->scal + 3);
    e = launch_absmax(fat_d, (long long)(4 * V * 18), amax_d, s);
    float amax = 0.f;
    if (e == cudaSuccess) {
        unsigned bits = 0;
        e = cudaMemcpyAsync(&bits, amax_d, sizeof bits, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        memcpy(&amax, &bits, sizeof amax);
    }
    if (e == cudaSuccess && !(amax < INFINITY)) {
        if (owned)
            cudaFree(fat_d);
        cudaStreamSynchronize(s);
        net_free(n);
        delete n;
        return fail(STAG_ERR_ARG, "stag_net_create: links hold a NaN, an infinity or an entry beyond FP32");
    }
    n->scale16 = amax > 0.f ? amax / kQ16 : 1.f;
    for (int k = 0; k < 4; k++)
        n->bcneg |= lat->bc[k] < 0 ? 1 << k : 0;
    if (e == cudaSuccess)
        e = launch_net_links_cb(lat->geom, lat->bc, fat_d, n->NL32, n->NL16, amax > 0.f ? kQ16 / amax : 0.f, s);
    // special unitary fat links (within 1e-6): the solver's 16-bit net links
    // keep rows 0 and 1 only and the kernels rebuild row 2 (two thirds of
    // the link bytes of the net's two stencil passes)
    if (e == cudaSuccess)
        e = launch_su3_deviation(fat_d, (long long)(4 * V), amax_d, s);
    if (e == cudaSuccess) {
        unsigned bits = 0;
        e = cudaMemcpyAsync(&bits, amax_d, sizeof bits, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        float dev = 1.f;
        memcpy(&dev, &bits, sizeof dev);
        if (e == cudaSuccess && dev <= 1e-6f) {
            e = cudaMalloc(&n->NL12, net_links12_bytes(lat->geom));
            if (e == cudaSuccess)
                e = cudaMemsetAsync(n->NL12, 0, net_links12_bytes(lat->geom), s);
            if (e == cudaSuccess)
                e = launch_net_links12(lat->geom, lat->bc, fat_d, n->NL12, amax > 0.f ? kQ16 / amax : 0.f, s);
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (owned)
        cudaFree(fat_d);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return bail(e != cudaSuccess ? e : e2);
    // initial weights: the identity map plus seeded noise.  With eight
    // channels each hop of layer 1 goes into a channel of its own (and r
    // into channel 0 as well), layer 2 is the identity and layer 3 reads
    // channel 0: the net starts as the identity, and the hop weights of
    // layer 3 set every two-hop path C[a][b] linearly, so the loss starts
    // at plain CG's preconditioner with no saddle at the start (noise 1e-3).
    // Fewer channels: the identity through every channel, noise 1e-2 (a
    // net of that form with eight channels took CG from 413 to 2360
    // iterations at 32^3x64 before training had moved it far).
    std::vector<double> w(nr, 0.0);
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, C == 8 ? 1e-3 : 1e-2);
    for (auto &v : w)
        v = nd(rng);
    auto W = [&](int layer, int d, int o, int i) -> double & {
        const int cin = layer == 0 ? 1 : C, cout = layer == 2 ? 1 : C;
        return w[2 * (size_t)(n->off[layer] + (d * cout + o) * cin + i)];
    };
    if (C == 8) {
        W(0, 0, 0, 0) += 1.0;
        for (int d = 1; d < 9; d++)
            W(0, d, d - 1, 0) += 1.0;
        for (int o = 0; o < C; o++)
            W(1, 0, o, o) += 1.0;
        W(2, 0, 0, 0) += 1.0;
    } else {
        for (int o = 0; o < C; o++) {
            W(0, 0, o, 0) += 1.0;
            W(1, 0, o, o) += 1.0;
            W(2, 0, 0, o) += 1.0 / C;
        }
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
    CUDA_TRY(cudaStreamSynchronize(n->lat->stream));
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
    CUDA_TRY(cudaStreamSynchronize(n->lat->stream));
    CUDA_TRY(cudaMemcpy(w, n->w, sizeof(double) * 2 * n->nw, cudaMemcpyDeviceToHost));
    return STAG_OK;
}

// ---- applying the net ------------------------------------------------------
static NetLinkSet net_links(const stag_net n, bool links16) {
    NetLinkSet s;
    s.l32 = n->NL32;
    s.bcneg = n->bcneg;
    if (links16) {
        s.l16 = n->NL16;
        s.l12 = n->NL12;
        s.scale16 = n->scale16;
    }
    return s;
}

// the path coefficients of the current weights (round_half: binary16
// weights; hermitian: of the net's Hermitian part)
static cudaError_t net_coefficients(stag_net n, int round_half, cudaStream_t s, int hermitian = 0) {
    return launch_net_path_coef(n->C, n->w32, n->off, round_half, n->path, s, hermitian);
}

// z = N(r) on even vectors with the coefficients in n->path: r of precision
// prec_in and component stride rs, z of prec_out and stride zs; dots: the
// partials of Re<z, r>, Re<z, Ap> for the flexible CG
static cudaError_t net_apply_path(stag_net n, int prec, const void *r, int rs, void *z, int zs, bool links16,
                                  bool dots, const void *Ap, const int *gate, cudaStream_t s) {
    stag_lattice lat = n->lat;
    const NetLinkSet nl = net_links(n, links16);
    cudaError_t e = launch_net_mid(prec, lat->geom, nl, n->path, r, rs, n->chi, gate, s);
    if (e != cudaSuccess)
        return e;
    return launch_net_out(prec, prec, lat->geom, nl, n->path, n->chi, r, rs, z, zs, dots, Ap, lat->partial, gate, s);
}

static int check_net_field(const stag_net n, const stag_field f, const char *who) {
    if (!f || f->lat != n->lat || f->parity != STAG_EVEN)
        return fail(STAG_ERR_ARG, "%s: fields must be even fields of the net's lattice", who);
    if (f->prec != STAG_F64 && f->prec != STAG_DF64 && f->prec != STAG_F32)
        return fail(STAG_ERR_ARG, "%s: fields must be F64, DF64 or F32", who);
    return STAG_OK;
}

extern "C" int stag_net_apply(stag_net n, stag_field out_even, const stag_field in_even, int flags) {
    STAG_NVTX("stag_net_apply");
    if (!n)
        return fail(STAG_ERR_ARG, "stag_net_apply: NULL net");
    STAG_TRY(check_net_field(n, out_even, "stag_net_apply"));
    STAG_TRY(check_net_field(n, in_even, "stag_net_apply"));
    if (out_even->prec != in_even->prec)
        return fail(STAG_ERR_ARG, "stag_net_apply: precision mismatch");
    if (out_even == in_even)
        return fail(STAG_ERR_ARG, "stag_net_apply: in and out must differ");
    if (flags & ~(STAG_NET_FP16_WEIGHTS | STAG_NET_LINKS16 | STAG_NET_HERMITIAN))
        return fail(STAG_ERR_ARG, "stag_net_apply: unknown flags 0x%x", flags);
    DEVICE_SCOPE(n->lat->device);
    cudaStream_t s = n->lat->stream;
    const int S = n->lat->geom.stride;
    CUDA_TRY(net_coefficients(n, (flags & STAG_NET_FP16_WEIGHTS) ? 1 : 0, s, (flags & STAG_NET_HERMITIAN) ? 1 : 0));
    CUDA_TRY(net_apply_path(n, in_even->prec, in_even->data, S, out_even->data, S, (flags & STAG_NET_LINKS16) != 0,
                            false, nullptr, nullptr, s));
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
        n->enorm_cap = 0;
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
    CUDA_TRY(cudaStreamSynchronize(n->lat->stream));
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
// out = M in = m^2 in - D_eo D_oe in on FP32 solver-layout vectors (t: odd)
static int apply_M_f32(stag_net n, const void *in, void *t, void *out, cudaStream_t s) {
    stag_lattice lat = n->lat;
    const int P = STAG_F32;
    DslashArgs a1 = dslash_args(lat, P, STAG_ODD, in, t);
    CUDA_TRY(launch_dslash(P, EPI_NONE, a1, lat->dslash_block[P], s));
    DslashArgs a2 = dslash_args(lat, P, STAG_EVEN, t, out);
    a2.p = in;
    a2.m2 = make_dpair(n->mass * n->mass);
    a2.m2_in_args = 1;
    CUDA_TRY(launch_dslash(P, EPI_M, a2, lat->dslash_block[P], s));
    return STAG_OK;
}

// loss of pair p added to scal[0] and its dL/dC*, dL/dc0* to G; the path
// coefficients must be current.  z = N(r) -> fz; then the output gradient g:
//   error loss:    g = (z - e) / |e|^2                  -> fmz
//   residual loss: q = (M z - r) / |r|^2 -> fmz, g = M q -> fz (M Hermitian)
static int pair_loss_grad(stag_net n, int p, cudaStream_t s) {
    stag_lattice lat = n->lat;
    const Geom &g = lat->geom;
    const int S = g.stride, Vh = g.Vh;
    CUDA_TRY(net_apply_path(n, STAG_F32, n->pr[p], Vh, n->fz, S, false, false, nullptr, nullptr, s));
    const float2 *gv;
    if (n->loss_kind == STAG_NET_LOSS_RESIDUAL) {
        STAG_TRY(apply_M_f32(n, n->fz, n->ft, n->fmz, s));
        CUDA_TRY(launch_net_resid_loss(Vh, (float2 *)n->fmz, S, n->pr[p], Vh, n->rnorm2 + p, n->scal, s));
        STAG_TRY(apply_M_f32(n, n->fmz, n->ft, n->fz, s));
        gv = (const float2 *)n->fz;
    } else {
        CUDA_TRY(launch_net_error_loss(Vh, (const float2 *)n->fz, S, n->pe[p], Vh, n->enorm2 + p, (float2 *)n->fmz,
                                       n->scal, s));
        gv = (const float2 *)n->fmz;
    }
    CUDA_TRY(launch_net_grad(g, n->NL32, n->pr[p], Vh, gv, S, n->gpartial, n->G, s));
    return STAG_OK;
}

// loss and dL/dW* summed over the pairs idx[0..count)
static int loss_grad_range(stag_net n, const int *idx, int count, double *loss) {
    cudaStream_t s = n->lat->stream;
    CUDA_TRY(cudaMemsetAsync(n->grad, 0, sizeof(double) * 2 * n->nw, s));
    CUDA_TRY(cudaMemsetAsync(n->G, 0, sizeof(double2) * 65, s));
    CUDA_TRY(cudaMemsetAsync(n->scal, 0, sizeof(double), s));
    CUDA_TRY(net_coefficients(n, 0, s));
    for (int k = 0; k < count; k++)
        STAG_TRY(pair_loss_grad(n, idx[k], s));
    CUDA_TRY(launch_net_path_chain(n->C, n->w32, n->off, n->G, (double2 *)n->grad, s));
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
    const int S = lat->geom.stride, Vh = lat->geom.Vh;
    CUDA_TRY(cudaMemsetAsync(n->scal + 1, 0, 2 * sizeof(double), s));
    CUDA_TRY(net_coefficients(n, 0, s));
    for (size_t p = 0; p < n->pr.size(); p++) {
        CUDA_TRY(net_apply_path(n, STAG_F32, n->pr[p], Vh, n->fz, S, false, false, nullptr, nullptr, s));
        STAG_TRY(apply_M_f32(n, n->fz, n->ft, n->fmz, s));
        CUDA_TRY(launch_net_dot2(Vh, (const float2 *)n->fmz, S, n->pr[p], Vh, n->scal + 1, s));
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

constexpr int kAdamWarmup = 100;

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
            // warm-up: the step size ramps up linearly over the net's first
            // kAdamWarmup steps.  Adam's first steps move every weight by about
            // the step size whatever its gradient; at full size from the start,
            // 32 steps (256 pairs, one epoch) left a net that took CG from 413
            // to 699 iterations (32^3x64)
            const double ramp = std::min(1.0, (double)n->adam_t / kAdamWarmup);
            CUDA_TRY(launch_adam(2 * n->nw, n->w, n->grad, n->m, n->v, lr_ep * ramp / cnt, n->adam_t, n->w32, s));
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

// z = N(r) (or z = r without the net) with the partials of Re<z, r> and
// Re<z, Ap> (Ap may be NULL), then beta and <z, r> in the scalars
static cudaError_t precondition(stag_net n, int prec, bool use_net, const void *r, void *z, const void *Ap,
                                int first, const int *gate, cudaStream_t s) {
    stag_lattice lat = n->lat;
    const int S = lat->geom.stride;
    cudaError_t e = use_net ? net_apply_path(n, prec, r, S, z, S, true, true, Ap, gate, s)
                            : launch_fcg_copy_dots(prec, lat->geom, r, z, Ap, lat->partial, gate, s);
    if (e != cudaSuccess)
        return e;
    return launch_fcg_finish(lat->partial, net_grid(lat->geom), lat->sc, first, s);
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
    CUDA_TRY(precondition(n, prec, use_net, w.r, n->z[prec], nullptr, 1, gate, s));
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
            // x += alpha p, r -= alpha Ap, |r|^2 and the stopping test
            CUDA_TRY(launch_fcg_update(prec, g, w.xw, w.r, w.p, w.Ap, lat->partial, lat->sc, s));
            // z = N(r), beta = -alpha <z, Ap> / <z_old, r_old>, p = z + beta p
            CUDA_TRY(precondition(n, prec, use_net, w.r, n->z[prec], w.Ap, 0, gate, s));
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

static int learned_impl(stag_net n, stag_field x, const stag_field b, double mass, double rel_tol, int max_iter,
                        stag_solve_info *info);

extern "C" int stag_cg_solve_learned(stag_net n, stag_field x, const stag_field b, double mass, double rel_tol,
                                     int max_iter, stag_solve_info *info) {
    STAG_NVTX("stag_cg_solve_learned");
    if (!n || !x || !b || x == b || check_net_field(n, b, "stag_cg_solve_learned") != STAG_OK)
        return learned_impl(n, x, b, mass, rel_tol, max_iter, info);  // reports the error
    RhsScale rs;
    STAG_TRY(rhs_scale_begin(b, &rs));
    const int st = learned_impl(n, x, rs.scaled ? rs.scaled : b, mass, rel_tol, max_iter, info);
    STAG_TRY(rhs_scale_end(&rs, &x, 1));
    return st;
}

static int learned_impl(stag_net n, stag_field x, const stag_field b, double mass, double rel_tol, int max_iter,
                        stag_solve_info *info) {
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
    STAG_TRY(alloc_vec(lat, prec, &n->z[prec]));
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    CUDA_TRY(cudaMemcpyAsync(w.bw, b->data, b->bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemsetAsync(w.xw, 0, field_bytes(lat, prec), s));
    // the deployed preconditioner: binary16 weights, 16-bit links, the net's
    // Hermitian part (CG's recurrences assume a Hermitian preconditioner)
    CUDA_TRY(net_coefficients(n, 1, s, 1));
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
            status = fcg_run(n, prec, use_net, mass, tol2bb, max_iter - iters, use_net ? 16 : 32, &it, &rr);
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

// ---- mixed-precision flexible CG with the net ---------------------------
static cudaError_t learned_precond_enqueue(void *ctx, int lo, const void *rs, void *z, const void *Ap, int first,
                                           cudaStream_t s) {
    stag_net n = (stag_net)ctx;
    stag_lattice lat = n->lat;
    const int S = lat->geom.stride;
    cudaError_t e = net_apply_path(n, lo, rs, S, z, S, true, true, Ap, status_flag(lat), s);
    if (e != cudaSuccess)
        return e;
    return launch_fcg_finish(lat->partial, net_grid(lat->geom), lat->sc, first, s);
}

extern "C" int stag_cg_solve_learned_mixed(stag_net n, stag_field x, const stag_field b, double mass,
                                           double rel_tol, int max_iter, int inner_prec, double delta,
                                           stag_solve_info *info) {
    STAG_NVTX("stag_cg_solve_learned_mixed");
    if (info)
        memset(info, 0, sizeof *info);
    if (!n || !x || !b)
        return fail(STAG_ERR_ARG, "stag_cg_solve_learned_mixed: NULL argument");
    STAG_TRY(check_net_field(n, x, "stag_cg_solve_learned_mixed"));
    STAG_TRY(check_net_field(n, b, "stag_cg_solve_learned_mixed"));
    if (x->prec != b->prec || x == b || (x->prec != STAG_F64 && x->prec != STAG_DF64))
        return fail(STAG_ERR_ARG, "stag_cg_solve_learned_mixed: x and b must be distinct F64 or DF64 fields");
    if (inner_prec != STAG_F32 && inner_prec != STAG_F16)
        return fail(STAG_ERR_ARG, "stag_cg_solve_learned_mixed: inner precision must be F32 or F16");
    if (!(mass > 0) || !std::isfinite(mass) || !(rel_tol >= 0) || !std::isfinite(rel_tol) || max_iter < 0)
        return fail(STAG_ERR_ARG, "stag_cg_solve_learned_mixed: need mass > 0, rel_tol >= 0, max_iter >= 0");
    if (!(delta > 0 && delta < 1))
        return fail(STAG_ERR_ARG, "stag_cg_solve_learned_mixed: delta must be in (0, 1)");
    stag_lattice lat = n->lat;
    const int hi = x->prec, lo = inner_prec;
    if (!lat->has_gauge || !lat->links[hi] || !lat->links[lo])
        return fail(STAG_ERR_STATE, "stag_cg_solve_learned_mixed: needs %s and %s gauge copies", prec_name(hi),
                    prec_name(lo));
    DEVICE_SCOPE(lat->device);
    const auto t0 = std::chrono::steady_clock::now();
    STAG_TRY(alloc_vec(lat, lo, &n->z[lo]));
    // the deployed preconditioner: binary16 weights, 16-bit links, the net's
    // Hermitian part
    CUDA_TRY(net_coefficients(n, 1, lat->stream, 1));
    MixedPrecond pc;
    pc.enqueue = learned_precond_enqueue;
    pc.ctx = n;
    pc.z = n->z[lo];
    RhsScale rs;
    STAG_TRY(rhs_scale_begin(b, &rs));
    const stag_field bs = rs.scaled ? rs.scaled : b;
    stag_solve_info first;
    int st = mixed_solve_raw(lat, hi, lo, x->data, bs->data, bs->bytes, mass, rel_tol, max_iter, delta, &first, &pc);
    if (st == STAG_ERR_BREAKDOWN || st == STAG_ERR_NOT_CONVERGED) {
        // the plain mixed solver from x = 0
        stag_solve_info second;
        st = mixed_solve_raw(lat, hi, lo, x->data, bs->data, bs->bytes, mass, rel_tol, max_iter, delta, &second);
        second.iters += first.iters;
        second.restarts += first.restarts;
        first = second;
    }
    STAG_TRY(rhs_scale_end(&rs, &x, 1));
    first.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info)
        *info = first;
    return st;
}
