// Domain decomposition in t, emulated on one GPU: the data movement of a
// lattice split over k ranks (Sec. 2: each rank owns a slab of time slices
// and exchanges the boundary slices of the vector it applies Dslash to).
//
// Domain d owns slices [t0, t0 + nt).  Before each Dslash it assembles its
// input in a private buffer from its own slab and the three slices on either
// side (the Naik term reaches three slices), which on a multi-GPU system its
// two neighbours would send; here they are device-to-device copies of the
// owners' slices.  The Dslash kernel then writes the outputs of the slab only
// and reads nothing of the input outside slab + halo (the rest of the private
// buffer stays zero, so a deeper reach would change the result).  Links are
// static: a rank holds those of its slab and of the three slices below it,
// and each domain here gets a private copy of exactly those (zero
// elsewhere), filled once per call as the exchange at upload would be.  The
// CG's global sums are per-domain partial sums added on the host in domain
// order, the allreduce of a multi-GPU run.
#include "api_internal.h"

#include <algorithm>
#include <climits>

namespace {

struct Domain {
    int t0 = 0, nt = 0;            // owned slices [t0, t0 + nt)
    void *buf = nullptr;           // assembled input (slab + halo, zero elsewhere)
    void *links = nullptr;         // links of slices [t0 - 3, t0 + nt), zero elsewhere
    CgScalars *sc = nullptr;       // this domain's scalars (partial sums)
};

constexpr int kHalo = 3;  // Naik reach in slices

struct Domains {
    stag_lattice lat;
    int prec;
    std::vector<Domain> d;
    ~Domains() {
        for (auto &x : d) {
            if (x.buf)
                cudaFree(x.buf);
            if (x.links)
                cudaFree(x.links);
            if (x.sc)
                cudaFree(x.sc);
        }
    }
};

// the active link layout of the domain precision: its compression mask and
// the bytes of one parity
int link_mask(const Domains &D) { return D.lat->links_c12[D.prec] ? D.lat->c12_mask[D.prec] : 0; }
size_t link_half_bytes(const Domains &D) {
    return link_parity_bytes(D.prec, link_mask(D), (size_t)D.lat->geom.stride);
}
const void *link_base(const Domains &D) {
    return D.lat->links_c12[D.prec] ? D.lat->links_c12[D.prec] : D.lat->links[D.prec];
}

// the planes of one kind's layout (link_kind_bytes): offset within the
// kind, bytes per site, bytes between consecutive planes of the same shape,
// and how many such planes
struct Planes {
    size_t base, elem, pitch, count;
};
int kind_planes(int prec, bool c12, size_t S, Planes pl[3]) {
    if (c12) {
        if (prec == STAG_F32) {
            pl[0] = {0, 16, 16 * S, 3};  // float4 [3][S]
            return 1;
        }
        pl[0] = {0, 16, 16 * S, 1};      // int4 [S]
        pl[1] = {16 * S, 8, 8 * S, 1};   // int2 [S]
        return 2;
    }
    if (prec == STAG_F16) {
        pl[0] = {0, 16, 16 * S, 2};      // int4 [2][S]
        pl[1] = {32 * S, 4, 4 * S, 1};   // int [S]
        return 2;
    }
    const size_t eb = prec_link_elem_bytes(prec);
    pl[0] = {0, eb, eb * S, 9};          // Elem [9][S]
    return 1;
}

// copy the links of slices [t, t + n) (one contiguous range) of both
// parities: every plane of every kind, one 2-D copy per group of planes
int copy_link_range(const Domains &D, void *dst, int t, int n) {
    stag_lattice lat = D.lat;
    const size_t S = (size_t)lat->geom.stride;
    const size_t per = (size_t)lat->geom.plane[3];
    const size_t half = link_half_bytes(D);
    const int mask = link_mask(D);
    const char *src = (const char *)link_base(D);
    for (int par = 0; par < 2; par++)
        for (int kind = 0; kind < 8; kind++) {
            Planes pl[3];
            const int np = kind_planes(D.prec, (mask >> (kind >> 2)) & 1, S, pl);
            for (int q = 0; q < np; q++) {
                const size_t off = par * half + link_kind_offset(D.prec, mask, kind, S) + pl[q].base +
                                   (size_t)t * per * pl[q].elem;
                CUDA_TRY(cudaMemcpy2DAsync((char *)dst + off, pl[q].pitch, src + off, pl[q].pitch,
                                           (size_t)n * per * pl[q].elem, pl[q].count, cudaMemcpyDeviceToDevice,
                                           lat->stream));
            }
        }
    return STAG_OK;
}

// domain i's links: slices [t0 - 3, t0 + nt) (periodic), zero elsewhere
int fill_links(const Domains &D, int i) {
    const Domain &x = D.d[i];
    const int Lt = D.lat->geom.L[3];
    int t = x.t0 - kHalo, n = x.nt + kHalo;
    if (n >= Lt) {
        t = 0;
        n = Lt;
    }
    t = (t % Lt + Lt) % Lt;
    const int first = std::min(n, Lt - t);  // up to the end of the lattice, then from slice 0
    STAG_TRY(copy_link_range(D, x.links, t, first));
    if (n > first)
        STAG_TRY(copy_link_range(D, x.links, 0, n - first));
    return STAG_OK;
}

int make_domains(Domains &D, int k) {
    stag_lattice lat = D.lat;
    const int Lt = lat->geom.L[3];
    if (k < 1 || k > Lt)
        return fail(STAG_ERR_ARG, "domain decomposition: %d domains for %d time slices", k, Lt);
    D.d.resize(k);
    int t = 0;
    const size_t fb = field_bytes(lat, D.prec);
    for (int i = 0; i < k; i++) {
        Domain &x = D.d[i];
        x.t0 = t;
        x.nt = Lt / k + (i < Lt % k ? 1 : 0);
        t += x.nt;
        const size_t lb = 2 * link_half_bytes(D);
        cudaError_t e = cudaMalloc(&x.buf, fb);
        if (e == cudaSuccess)
            e = cudaMalloc(&x.links, lb);
        if (e == cudaSuccess)
            e = cudaMalloc(&x.sc, sizeof(CgScalars));
        if (e == cudaSuccess)
            e = cudaMemsetAsync(x.buf, 0, fb, lat->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(x.links, 0, lb, lat->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(x.sc, 0, sizeof(CgScalars), lat->stream);
        if (e != cudaSuccess)
            return fail(e == cudaErrorMemoryAllocation ? STAG_ERR_NOMEM : STAG_ERR_CUDA,
                        "domain decomposition: %s", cudaGetErrorString(e));
        STAG_TRY(fill_links(D, i));
    }
    return STAG_OK;
}

// copy slices [t, t + n) (periodic in t) of one checkerboard field
int copy_slices(const Domains &D, const void *src, void *dst, int t, int n) {
    stag_lattice lat = D.lat;
    const Geom &g = lat->geom;
    const int Lt = g.L[3];
    const size_t per = (size_t)g.plane[3];  // checkerboard sites of one time slice
    const size_t S = (size_t)g.stride;
    const size_t eb = vec_site_bytes(D.prec);
    const int planes = D.prec == STAG_F16 ? 1 : 3;  // 16-bit: one cell per site holds all
    for (int k = 0; k < n; k++) {
        const size_t tt = (size_t)(((t + k) % Lt + Lt) % Lt);
        for (int a = 0; a < planes; a++) {
            const size_t off = (a * S + tt * per) * eb;
            CUDA_TRY(cudaMemcpyAsync((char *)dst + off, (const char *)src + off, per * eb,
                                     cudaMemcpyDeviceToDevice, lat->stream));
        }
    }
    return STAG_OK;
}

// domain i's input: its slab of `global` and the halo slices on either side
int assemble(const Domains &D, int i, const void *global) {
    const Domain &x = D.d[i];
    const int Lt = D.lat->geom.L[3];
    if (x.nt + 2 * kHalo >= Lt)  // the halos cover the whole lattice
        return copy_slices(D, global, x.buf, 0, Lt);
    return copy_slices(D, global, x.buf, x.t0 - kHalo, x.nt + 2 * kHalo);
}

// domain i's Dslash from its assembled input: the outputs of its slab
int domain_dslash(const Domains &D, int i, int out_par, int epi, void *out, const void *p, double m2) {
    const Domain &x = D.d[i];
    stag_lattice lat = D.lat;
    DslashArgs a = dslash_args(lat, D.prec, out_par, x.buf, out);
    // the domain's own copy of the links, same layout
    const size_t half = link_half_bytes(D);
    a.links_out = (const char *)x.links + (size_t)out_par * half;
    a.links_in = (const char *)x.links + (size_t)(1 - out_par) * half;
    a.c0 = x.t0 * lat->geom.plane[3];
    a.cn = x.nt * lat->geom.plane[3];
    a.p = p;
    a.sc = x.sc;
    a.m2 = make_dpair(m2);
    a.m2_in_args = 1;
    CUDA_TRY(launch_dslash(D.prec, epi, a, lat->dslash_block[D.prec], lat->stream));
    return STAG_OK;
}

// the vector kernels on domain i's slab: same field layout, base moved to
// the first site of the slab, Vh = the slab's sites
Geom slab_geom(const Domains &D, int i) {
    Geom g = D.lat->geom;
    g.Vh = D.d[i].nt * g.plane[3];
    return g;
}
void *slab(const Domains &D, int i, void *v) {
    return (char *)v + (size_t)D.d[i].t0 * D.lat->geom.plane[3] * vec_site_bytes(D.prec);
}

// scalars of domain i before a reducing kernel: running, no stopping test
int put_scalars(const Domains &D, int i, double rr, double alpha, double beta) {
    CgScalars h;
    memset(&h, 0, sizeof h);
    h.status = CG_RUNNING;
    h.max_iter = INT_MAX;
    h.rr = rr;
    h.rr_stop = -1.0;
    h.alpha = make_dpair(alpha);
    h.beta = make_dpair(beta);
    // pageable source: read by the time the call returns
    CUDA_TRY(cudaMemcpyAsync(D.d[i].sc, &h, sizeof h, cudaMemcpyHostToDevice, D.lat->stream));
    return STAG_OK;
}

// the "allreduce": one double field of every domain's scalars, summed in order
int host_sum(const Domains &D, size_t field_off, double *out) {
    CUDA_TRY(cudaStreamSynchronize(D.lat->stream));
    double s = 0.0;
    for (const auto &x : D.d) {
        double v = 0.0;
        CUDA_TRY(cudaMemcpy(&v, (const char *)x.sc + field_off, sizeof v, cudaMemcpyDeviceToHost));
        s += v;
    }
    *out = s;
    return STAG_OK;
}

}  // namespace

extern "C" int stag_dd_dslash(stag_lattice lat, int ndomains, stag_field out, const stag_field in) {
    STAG_NVTX("stag_dd_dslash");
    if (!lat || !out || !in)
        return fail(STAG_ERR_ARG, "stag_dd_dslash: NULL argument");
    if (out->lat != lat || in->lat != lat)
        return fail(STAG_ERR_ARG, "stag_dd_dslash: field belongs to another lattice");
    if (out->parity == in->parity || out->prec != in->prec || out == in)
        return fail(STAG_ERR_STATE, "stag_dd_dslash: need two fields of opposite parity and one precision");
    const int prec = in->prec;
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_dd_dslash: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    Domains D{lat, prec, {}};
    STAG_TRY(make_domains(D, ndomains));
    for (int i = 0; i < ndomains; i++) {
        STAG_TRY(assemble(D, i, in->data));
        STAG_TRY(domain_dslash(D, i, out->parity, EPI_NONE, out->data, nullptr, 0.0));
    }
    CUDA_TRY(cudaStreamSynchronize(lat->stream));
    return STAG_OK;
}

static int dd_cg_impl(stag_lattice lat, int ndomains, stag_field x, const stag_field b, double mass,
                      double rel_tol, int max_iter, stag_solve_info *info);

extern "C" int stag_dd_cg_solve(stag_lattice lat, int ndomains, stag_field x, const stag_field b, double mass,
                                double rel_tol, int max_iter, stag_solve_info *info) {
    STAG_NVTX("stag_dd_cg_solve");
    if (!lat || !x || !b || x == b || b->lat != lat || b->parity != STAG_EVEN || x->prec != b->prec)
        return dd_cg_impl(lat, ndomains, x, b, mass, rel_tol, max_iter, info);  // reports the error
    RhsScale rs;
    STAG_TRY(rhs_scale_begin(b, &rs));
    const int st = dd_cg_impl(lat, ndomains, x, rs.scaled ? rs.scaled : b, mass, rel_tol, max_iter, info);
    STAG_TRY(rhs_scale_end(&rs, &x, 1));
    return st;
}

static int dd_cg_impl(stag_lattice lat, int ndomains, stag_field x, const stag_field b, double mass,
                      double rel_tol, int max_iter, stag_solve_info *info) {
    if (info)
        memset(info, 0, sizeof *info);
    if (!lat || !x || !b)
        return fail(STAG_ERR_ARG, "stag_dd_cg_solve: NULL argument");
    if (x->lat != lat || b->lat != lat)
        return fail(STAG_ERR_ARG, "stag_dd_cg_solve: field belongs to another lattice");
    if (x->parity != STAG_EVEN || b->parity != STAG_EVEN || x->prec != b->prec || x == b)
        return fail(STAG_ERR_STATE, "stag_dd_cg_solve: x and b must be distinct even fields of one precision");
    if (x->prec != STAG_F64 && x->prec != STAG_DF64)
        return fail(STAG_ERR_STATE, "stag_dd_cg_solve: fields must be F64 or DF64 (got %s)", prec_name(x->prec));
    if (!(mass > 0) || !std::isfinite(mass) || !(rel_tol >= 0) || !std::isfinite(rel_tol) || max_iter < 0)
        return fail(STAG_ERR_ARG, "stag_dd_cg_solve: need mass > 0, rel_tol >= 0, max_iter >= 0");
    const int prec = x->prec;
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_dd_cg_solve: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    const auto t_start = std::chrono::steady_clock::now();
    STAG_TRY(ensure_cg_work(lat, prec));
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    Domains D{lat, prec, {}};
    STAG_TRY(make_domains(D, ndomains));
    const int k = ndomains;
    const double m2 = mass * mass;

    // x = 0, r = b, p = b and the slab sums of |b|^2
    for (int i = 0; i < k; i++) {
        STAG_TRY(put_scalars(D, i, 0.0, 0.0, 0.0));
        CUDA_TRY(launch_cg_init(prec, slab_geom(D, i), slab(D, i, w.xw), slab(D, i, w.r), slab(D, i, w.p),
                                slab(D, i, b->data), lat->partial, D.d[i].sc, s));
    }
    double bb = 0.0;
    STAG_TRY(host_sum(D, offsetof(CgScalars, bb), &bb));
    if (!(bb < INFINITY))
        return fail(STAG_ERR_ARG, "stag_dd_cg_solve: |b|^2 is not finite");
    const double stop = rel_tol * rel_tol * bb;
    double rr = bb;
    int it = 0;
    int status = rr <= stop ? CG_CONVERGED : CG_RUNNING;
    while (status == CG_RUNNING && it < max_iter) {
        // t = D_oe p on every slab (halo of p), then Ap = m^2 p - D_eo t and
        // the slab sums of <p, Ap> (halo of t)
        for (int i = 0; i < k; i++) {
            STAG_TRY(assemble(D, i, w.p));
            STAG_TRY(domain_dslash(D, i, STAG_ODD, EPI_NONE, w.t, nullptr, m2));
        }
        for (int i = 0; i < k; i++) {
            STAG_TRY(put_scalars(D, i, rr, 0.0, 0.0));
            STAG_TRY(assemble(D, i, w.t));
            STAG_TRY(domain_dslash(D, i, STAG_EVEN, EPI_M_PAP, w.Ap, w.p, m2));
        }
        double pAp = 0.0;
        STAG_TRY(host_sum(D, offsetof(CgScalars, pAp), &pAp));
        if (!(pAp > 0.0 && pAp < INFINITY)) {
            status = CG_BREAKDOWN;
            break;
        }
        const double alpha = rr / pAp;
        // x += alpha p, r -= alpha Ap on every slab, and the slab sums of |r|^2
        for (int i = 0; i < k; i++) {
            STAG_TRY(put_scalars(D, i, rr, alpha, 0.0));
            CUDA_TRY(launch_cg_update(prec, slab_geom(D, i), slab(D, i, w.xw), slab(D, i, w.r), slab(D, i, w.p),
                                      slab(D, i, w.Ap), lat->partial, D.d[i].sc, s));
        }
        double rr_new = 0.0;
        STAG_TRY(host_sum(D, offsetof(CgScalars, rr), &rr_new));
        it++;
        const double beta = rr_new / rr;
        rr = rr_new;
        if (!(rr < INFINITY)) {
            status = CG_BREAKDOWN;
            break;
        }
        if (rr <= stop) {
            status = CG_CONVERGED;
            break;
        }
        // p = r + beta p on every slab
        for (int i = 0; i < k; i++) {
            STAG_TRY(put_scalars(D, i, rr, alpha, beta));
            CUDA_TRY(launch_cg_p_update(prec, slab_geom(D, i), slab(D, i, w.r), slab(D, i, w.p), D.d[i].sc, s));
        }
    }
    if (status == CG_RUNNING)
        status = CG_MAXITER;
    CUDA_TRY(cudaMemcpyAsync(x->data, w.xw, x->bytes, cudaMemcpyDeviceToDevice, s));
    // true residual |b - M x|^2 on the whole lattice
    double rr_true = 0.0;
    STAG_TRY(shifted_residual(lat, prec, x->data, b->data, mass, nullptr, &rr_true));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    stag_solve_info local;
    memset(&local, 0, sizeof local);
    local.iters = it;
    local.status = status == CG_CONVERGED ? STAG_OK
                   : status == CG_BREAKDOWN ? STAG_ERR_BREAKDOWN
                                            : STAG_ERR_NOT_CONVERGED;
    local.true_rel_resid = bb > 0 ? std::sqrt(rr_true / bb) : 0.0;
    local.iter_rel_resid = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    local.seconds = secs;
    if (info)
        *info = local;
    if (local.status != STAG_OK)
        return fail(local.status, "stag_dd_cg_solve: %s after %d iterations (|r|/|b| = %.3e)",
                    local.status == STAG_ERR_BREAKDOWN ? "breakdown" : "not converged", it, local.iter_rel_resid);
    return STAG_OK;
}
