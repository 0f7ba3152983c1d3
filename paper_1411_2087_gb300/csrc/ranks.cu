// Domain decomposition over ranks (stag_ddr_*; documentation in
// include/stag.h).  The paper's multi-node runs (Sec. 2, 3) split the lattice
// over MPI ranks; here the t direction is cut into one slab per rank, each
// rank a process with its own GPU and a full-size lattice whose slab it owns.
//
// Per Dslash a rank packs the three lowest and three highest slices of the
// input (one parity, every component plane) into two messages, hands them to
// the caller's communicator with its halo buffers, unpacks what arrives into
// the three slices on either side of its slab, and runs the stencil on its
// slab's output sites only.  The exchange runs on a second stream while the
// stencil covers the slab's interior (the slices more than three away from
// either face), and the two three-slice boundary ranges follow once the halo
// has landed.  The CG's global sums are slab sums that the communicator adds;
// the CG's scalar recurrence (alpha, beta, the stopping test) runs on the
// device from those sums, so that with a communicator that sums device
// values on the stream (NCCL) the host waits only every few iterations.  The
// vector kernels see the slab as a field of its own: the same layout with
// the base moved to the slab's first site.
#include "api_internal.h"

#include <climits>

namespace {

constexpr int kHaloSlices = 3;  // reach of the three-link term

struct Slab {
    int t0 = 0, nt = 0;
};

int slab_of(const int dims[4], int size, int rank, Slab *out) {
    if (!dims)
        return fail(STAG_ERR_ARG, "domain layout: dims is NULL");
    for (int k = 0; k < 4; k++)
        if (dims[k] < 2 || dims[k] % 2)
            return fail(STAG_ERR_ARG, "domain layout: dims must be even and >= 2");
    const int Lt = dims[3];
    if (size < 1 || rank < 0 || rank >= size)
        return fail(STAG_ERR_ARG, "domain layout: rank %d of %d", rank, size);
    if (Lt / size < kHaloSlices)
        return fail(STAG_ERR_ARG, "domain layout: %d ranks leave slabs thinner than %d of the %d time slices",
                    size, kHaloSlices, Lt);
    out->nt = Lt / size + (rank < Lt % size ? 1 : 0);
    out->t0 = rank * (Lt / size) + (rank < Lt % size ? rank : Lt % size);
    return STAG_OK;
}

// the four slice ranges of the exchange: what goes to rank - 1 and rank + 1
// (the slab's lowest and highest three slices) and where the messages from
// them land (the halo below and above), each kHaloSlices slices, periodic
struct HaloRanges {
    int send_prev, send_next, recv_prev, recv_next;
};

HaloRanges halo_ranges(int Lt, const Slab &s) {
    HaloRanges h;
    h.send_prev = s.t0;
    h.send_next = s.t0 + s.nt - kHaloSlices;
    h.recv_prev = ((s.t0 - kHaloSlices) % Lt + Lt) % Lt;
    h.recv_next = (s.t0 + s.nt) % Lt;
    return h;
}

// one message: for each component plane the kHaloSlices * per entries
// starting at slice t (a 16-bit field has one plane of 16-byte cells)
struct PlaneSet {
    size_t elem;   // bytes of one site's entry in a plane
    int count;     // planes
};

PlaneSet planes_of(int prec) { return PlaneSet{vec_site_bytes(prec), prec == STAG_F16 ? 1 : 3}; }

size_t message_bytes(const Geom &g, int prec) {
    const PlaneSet p = planes_of(prec);
    return (size_t)kHaloSlices * g.plane[3] * p.elem * p.count;
}

// field (device, internal layout) slices [t, t + kHaloSlices) <-> message (device)
cudaError_t copy_message(const Geom &g, int prec, void *field, int t, void *msg, bool pack, cudaStream_t s) {
    const PlaneSet p = planes_of(prec);
    const size_t per = (size_t)g.plane[3], S = (size_t)g.stride;
    const size_t width = kHaloSlices * per * p.elem;
    char *f = (char *)field + (size_t)t * per * p.elem;
    return pack ? cudaMemcpy2DAsync(msg, width, f, S * p.elem, width, p.count, cudaMemcpyDeviceToDevice, s)
                : cudaMemcpy2DAsync(f, S * p.elem, msg, width, width, p.count, cudaMemcpyDeviceToDevice, s);
}

bool comm_valid(const stag_comm *c) {
    return c && c->exchange && c->allreduce && c->size >= 1 && c->rank >= 0 && c->rank < c->size &&
           (c->device_buffers == 0 || c->device_buffers == 1) && (!c->allreduce_dev || c->device_buffers == 1);
}

// The global scalars of the rank CG, on the device next to the slab's
// CgScalars: the slab's partial sums are copied here, summed over the ranks
// in place, and turned into alpha, beta and the status by the kernels below.
struct DdScal {
    double pap;      // <p, M p>: the slab's, then the global sum
    double rr;       // |r|^2 of this iteration: the slab's, then the global sum
    double rr_prev;  // the global |r|^2 of the previous iteration
    double rr_stop;  // tol^2 |b|^2
    int max_iter;
    int iter_seen;   // sc->iter when dd_rr_kernel last ran
    int ran;         // the update kernel ran in this iteration
    int pad;
};

// one block: the slab's <p, Mp> from the n block partials, in block order
__global__ void dd_pap_kernel(const double *__restrict__ partial, int n, DdScal *dd) {
    __shared__ double smem[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 256)
        acc += partial[i];
    acc = block_sum<256>(acc, smem);
    if (threadIdx.x == 0)
        dd->pap = acc;
}

// alpha = |r|^2 / <p, Mp> from the global sums; breakdown on every rank alike
__global__ void dd_alpha_kernel(CgScalars *sc, DdScal *dd) {
    if (sc->status != CG_RUNNING)
        return;
    const double pap = dd->pap;
    sc->pAp = pap;
    if (!(pap > 0.0 && pap < INFINITY)) {
        sc->status = CG_BREAKDOWN;
        sc->alpha = make_dpair(0.0);
    } else {
        sc->alpha = make_dpair(dd->rr_prev / pap);
    }
}

// the slab's |r|^2 if the update kernel ran in this iteration, else 0
__global__ void dd_rr_kernel(const CgScalars *sc, DdScal *dd) {
    dd->ran = sc->iter != dd->iter_seen;
    dd->iter_seen = sc->iter;
    dd->rr = dd->ran ? sc->rr : 0.0;
}

// beta and the stopping test from the global |r|^2 (the status the update
// kernel may have set from the slab's sum is replaced by the global one)
__global__ void dd_beta_kernel(CgScalars *sc, DdScal *dd) {
    if (!dd->ran)
        return;
    const double rr = dd->rr;
    sc->beta = make_dpair(rr / dd->rr_prev);
    sc->rr = rr;
    dd->rr_prev = rr;
    if (!(rr < INFINITY))
        sc->status = CG_BREAKDOWN;
    else if (rr <= dd->rr_stop)
        sc->status = CG_CONVERGED;
    else if (sc->iter >= dd->max_iter)
        sc->status = CG_MAXITER;
    else
        sc->status = CG_RUNNING;
}

}  // namespace

struct stag_ddr_s {
    stag_lattice lat = nullptr;
    stag_comm comm;
    Slab slab;
    size_t msg_cap = 0;              // bytes of the largest message (any precision)
    void *dsend[2] = {}, *drecv[2] = {};  // device messages: [0] prev side, [1] next side
    void *hsend[2] = {}, *hrecv[2] = {};  // pinned host copies (host-memory communicators)
    CgScalars *sc = nullptr;         // the slab's partial sums
    DdScal *dd = nullptr;            // the global scalars of the CG (device)
    double *partial = nullptr;       // block partials of the split M Dslash
    double *hval = nullptr;          // pinned: one value through a host allreduce
    CgScalars *hsc = nullptr;        // pinned: the status read every few iterations
    cudaStream_t side = nullptr;     // the halo exchange, beside the interior stencil
    cudaEvent_t ev_in = nullptr, ev_halo = nullptr;
};

static void ddr_free(stag_ddr d) {
    for (int k = 0; k < 2; k++) {
        if (d->dsend[k])
            cudaFree(d->dsend[k]);
        if (d->drecv[k])
            cudaFree(d->drecv[k]);
        if (d->hsend[k])
            cudaFreeHost(d->hsend[k]);
        if (d->hrecv[k])
            cudaFreeHost(d->hrecv[k]);
    }
    if (d->sc)
        cudaFree(d->sc);
    if (d->dd)
        cudaFree(d->dd);
    if (d->partial)
        cudaFree(d->partial);
    if (d->hval)
        cudaFreeHost(d->hval);
    if (d->hsc)
        cudaFreeHost(d->hsc);
    if (d->ev_in)
        cudaEventDestroy(d->ev_in);
    if (d->ev_halo)
        cudaEventDestroy(d->ev_halo);
    if (d->side)
        cudaStreamDestroy(d->side);
}

extern "C" int stag_ddr_layout(const int dims[4], int size, int rank, int *t0, int *nt) {
    if (!t0 || !nt)
        return fail(STAG_ERR_ARG, "stag_ddr_layout: NULL argument");
    Slab s;
    STAG_TRY(slab_of(dims, size, rank, &s));
    *t0 = s.t0;
    *nt = s.nt;
    return STAG_OK;
}

extern "C" int stag_ddr_exchange_host(const int dims[4], int parity, const stag_comm *comm, double *field) {
    if (!dims || !field || !comm_valid(comm) || comm->device_buffers)
        return fail(STAG_ERR_ARG, "stag_ddr_exchange_host: NULL argument or a device-buffer communicator");
    if (parity != STAG_EVEN && parity != STAG_ODD)
        return fail(STAG_ERR_ARG, "stag_ddr_exchange_host: bad parity %d", parity);
    Slab s;
    STAG_TRY(slab_of(dims, comm->size, comm->rank, &s));
    const Geom g = geom_of(dims, (long long)dims[0] * dims[1] * dims[2] * dims[3] / 2);
    const HaloRanges h = halo_ranges(dims[3], s);
    const size_t per = (size_t)g.plane[3];
    const size_t n = kHaloSlices * per;  // sites of one message
    // canonical [Vh][3] complex128 <-> message: component plane by plane
    std::vector<double> to_prev(6 * n), to_next(6 * n), from_prev(6 * n), from_next(6 * n);
    auto pack = [&](int t, std::vector<double> &m) {
        for (int a = 0; a < 3; a++)
            for (size_t k = 0; k < n; k++) {
                const size_t c = (size_t)t * per + k;
                m[2 * (a * n + k)] = field[2 * (3 * c + a)];
                m[2 * (a * n + k) + 1] = field[2 * (3 * c + a) + 1];
            }
    };
    auto unpack = [&](int t, const std::vector<double> &m) {
        for (int a = 0; a < 3; a++)
            for (size_t k = 0; k < n; k++) {
                const size_t c = (size_t)t * per + k;
                field[2 * (3 * c + a)] = m[2 * (a * n + k)];
                field[2 * (3 * c + a) + 1] = m[2 * (a * n + k) + 1];
            }
    };
    pack(h.send_prev, to_prev);
    pack(h.send_next, to_next);
    if (comm->exchange(comm->ctx, to_prev.data(), to_next.data(), from_prev.data(), from_next.data(),
                       6 * n * sizeof(double), nullptr) != 0)
        return fail(STAG_ERR_STATE, "stag_ddr_exchange_host: the communicator's exchange failed");
    unpack(h.recv_prev, from_prev);
    unpack(h.recv_next, from_next);
    return STAG_OK;
}

extern "C" int stag_ddr_create(stag_lattice lat, const stag_comm *comm, stag_ddr *out) {
    if (!out)
        return fail(STAG_ERR_ARG, "stag_ddr_create: out is NULL");
    *out = nullptr;
    if (!lat || !comm_valid(comm))
        return fail(STAG_ERR_ARG, "stag_ddr_create: NULL lattice or an incomplete communicator");
    Slab s;
    STAG_TRY(slab_of(lat->dims, comm->size, comm->rank, &s));
    DEVICE_SCOPE(lat->device);
    stag_ddr d = new (std::nothrow) stag_ddr_s();
    if (!d)
        return fail(STAG_ERR_NOMEM, "stag_ddr_create: host allocation failed");
    d->lat = lat;
    d->comm = *comm;
    d->slab = s;
    d->msg_cap = message_bytes(lat->geom, STAG_F64);  // 16-byte entries: the largest message
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        e = cudaMalloc(&d->dsend[k], d->msg_cap);
        if (e == cudaSuccess)
            e = cudaMalloc(&d->drecv[k], d->msg_cap);
        if (e == cudaSuccess && !comm->device_buffers) {
            e = cudaMallocHost(&d->hsend[k], d->msg_cap);
            if (e == cudaSuccess)
                e = cudaMallocHost(&d->hrecv[k], d->msg_cap);
        }
    }
    if (e == cudaSuccess)
        e = cudaMalloc(&d->sc, sizeof(CgScalars));
    if (e == cudaSuccess)
        e = cudaMalloc(&d->dd, sizeof(DdScal));
    if (e == cudaSuccess)  // the split M Dslash: up to three launches of blocks of 64 or more
        e = cudaMalloc(&d->partial, sizeof(double) * ((size_t)lat->Vh / 64 + 4));
    if (e == cudaSuccess)
        e = cudaMallocHost(&d->hval, sizeof(double));
    if (e == cudaSuccess)
        e = cudaMallocHost(&d->hsc, sizeof(CgScalars));
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&d->side, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&d->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&d->ev_halo, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ddr_free(d);
        delete d;
        return fail(STAG_ERR_NOMEM, "stag_ddr_create: %s", cudaGetErrorString(e));
    }
    lat->live_fields++;  // the lattice outlives its decompositions
    *out = d;
    return STAG_OK;
}

extern "C" int stag_ddr_destroy(stag_ddr d) {
    if (!d)
        return STAG_OK;
    DEVICE_SCOPE(d->lat->device);
    cudaStreamSynchronize(d->lat->stream);
    ddr_free(d);
    d->lat->live_fields--;
    delete d;
    return STAG_OK;
}

// fill the halo of a field (device, precision prec) from the neighbours,
// in order on stream s
static int exchange_halo(stag_ddr d, int prec, void *field, cudaStream_t s) {
    stag_lattice lat = d->lat;
    const Geom &g = lat->geom;
    const HaloRanges h = halo_ranges(g.L[3], d->slab);
    const size_t bytes = message_bytes(g, prec);
    CUDA_TRY(copy_message(g, prec, field, h.send_prev, d->dsend[0], true, s));
    CUDA_TRY(copy_message(g, prec, field, h.send_next, d->dsend[1], true, s));
    int rc;
    if (d->comm.device_buffers) {
        rc = d->comm.exchange(d->comm.ctx, d->dsend[0], d->dsend[1], d->drecv[0], d->drecv[1], bytes, s);
    } else {
        for (int k = 0; k < 2; k++)
            CUDA_TRY(cudaMemcpyAsync(d->hsend[k], d->dsend[k], bytes, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        rc = d->comm.exchange(d->comm.ctx, d->hsend[0], d->hsend[1], d->hrecv[0], d->hrecv[1], bytes, nullptr);
        for (int k = 0; rc == 0 && k < 2; k++)
            CUDA_TRY(cudaMemcpyAsync(d->drecv[k], d->hrecv[k], bytes, cudaMemcpyHostToDevice, s));
    }
    if (rc != 0)
        return fail(STAG_ERR_STATE, "domain decomposition: the communicator's exchange failed (%d)", rc);
    CUDA_TRY(copy_message(g, prec, field, h.recv_prev, d->drecv[0], false, s));
    CUDA_TRY(copy_message(g, prec, field, h.recv_next, d->drecv[1], false, s));
    return STAG_OK;
}

// the stencil on slices [t, t + n) (and [t2, t2 + n2) in the same launch)
// of the slab, with the halo of `in` filled where they need it; EPI_M_PART
// writes its block partials from d->partial + *np on and advances *np
static int slab_range(stag_ddr d, int prec, int out_par, int epi, const void *in, void *out, const void *p,
                      const void *b, double m2, int t, int n, int t2, int n2, int *np) {
    stag_lattice lat = d->lat;
    if (n <= 0)
        return STAG_OK;
    const int P = lat->geom.plane[3];
    DslashArgs a = dslash_args(lat, prec, out_par, in, out);
    a.c0 = t * P;
    a.cn = n * P;
    a.c0b = t2 * P;
    a.cnb = n2 > 0 ? n2 * P : 0;
    a.p = p;
    a.b = b;
    a.sc = d->sc;
    a.skip_if_done = epi == EPI_NONE || epi == EPI_M_PART;  // the CG's no-op iterations after it stops
    a.partial = d->partial + (np ? *np : 0);
    a.m2 = make_dpair(m2);
    a.m2_in_args = 1;
    int block = lat->dslash_block[prec] > 0 ? lat->dslash_block[prec] : dslash_default_block(prec);
    if (epi != EPI_NONE) {  // the M Dslash's own tuning, as in the single-lattice solvers
        block = m_block(lat, prec);
        a.regs = lat->mdslash_block[prec] > 0 ? lat->mdslash_regs[prec] : lat->dslash_regs[prec];
    }
    CUDA_TRY(launch_dslash(prec, epi, a, block, lat->stream));
    if (np)
        *np += (a.cn + a.cnb + block - 1) / block;
    return STAG_OK;
}

// exchange the halo of `in`, then the stencil on the whole slab (EPI_NONE
// or EPI_M_PART; *np receives the number of block partials).  The interior
// (slices more than kHaloSlices from a face) runs while the exchange is in
// flight on the side stream, the two boundary ranges in one launch after it.
// One rank owns the whole lattice: its halo is its own slices, so there is
// nothing to exchange.
static int slab_dslash(stag_ddr d, int prec, int out_par, int epi, const void *in, void *out, const void *p,
                       double m2, int *np) {
    stag_lattice lat = d->lat;
    cudaStream_t s = lat->stream;
    const int t0 = d->slab.t0, nt = d->slab.nt, h = kHaloSlices;
    if (np)
        *np = 0;
    if (d->comm.size == 1)
        return slab_range(d, prec, out_par, epi, in, out, p, nullptr, m2, t0, nt, 0, 0, np);
    if (nt <= 2 * h) {
        STAG_TRY(exchange_halo(d, prec, (void *)in, s));
        return slab_range(d, prec, out_par, epi, in, out, p, nullptr, m2, t0, nt, 0, 0, np);
    }
    CUDA_TRY(cudaEventRecord(d->ev_in, s));
    CUDA_TRY(cudaStreamWaitEvent(d->side, d->ev_in, 0));
    STAG_TRY(slab_range(d, prec, out_par, epi, in, out, p, nullptr, m2, t0 + h, nt - 2 * h, 0, 0, np));
    STAG_TRY(exchange_halo(d, prec, (void *)in, d->side));
    CUDA_TRY(cudaEventRecord(d->ev_halo, d->side));
    CUDA_TRY(cudaStreamWaitEvent(s, d->ev_halo, 0));
    return slab_range(d, prec, out_par, epi, in, out, p, nullptr, m2, t0, h, t0 + nt - h, h, np);
}

// sum one device double over the ranks, in place, in order on the lattice
// stream: through the communicator's device allreduce, or through host
// memory (then the host waits)
static int allreduce_value(stag_ddr d, double *dev) {
    cudaStream_t s = d->lat->stream;
    if (d->comm.allreduce_dev) {
        if (d->comm.allreduce_dev(d->comm.ctx, dev, 1, s) != 0)
            return fail(STAG_ERR_STATE, "domain decomposition: the communicator's device allreduce failed");
        return STAG_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(d->hval, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (d->comm.allreduce(d->comm.ctx, d->hval, 1) != 0)
        return fail(STAG_ERR_STATE, "domain decomposition: the communicator's allreduce failed");
    CUDA_TRY(cudaMemcpyAsync(dev, d->hval, sizeof(double), cudaMemcpyHostToDevice, s));
    return STAG_OK;
}

// the slab as a field of its own for the pointwise kernels
static Geom slab_geom(const stag_ddr d) {
    Geom g = d->lat->geom;
    g.Vh = d->slab.nt * g.plane[3];
    return g;
}
static void *slab_ptr(const stag_ddr d, int prec, void *v) {
    return (char *)v + (size_t)d->slab.t0 * d->lat->geom.plane[3] * vec_site_bytes(prec);
}

// scalars before a reducing kernel: running, no stopping test
static int put_scalars(stag_ddr d, double rr, double alpha, double beta) {
    CgScalars h;
    memset(&h, 0, sizeof h);
    h.status = CG_RUNNING;
    h.max_iter = INT_MAX;
    h.rr = rr;
    h.rr_stop = -1.0;
    h.alpha = make_dpair(alpha);
    h.beta = make_dpair(beta);
    // pageable source: read by the time the call returns
    CUDA_TRY(cudaMemcpyAsync(d->sc, &h, sizeof h, cudaMemcpyHostToDevice, d->lat->stream));
    return STAG_OK;
}

// one field of the slab's scalars summed over all ranks
static int global_sum(stag_ddr d, size_t field_off, double *out) {
    double v = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&v, (const char *)d->sc + field_off, sizeof v, cudaMemcpyDeviceToHost, d->lat->stream));
    CUDA_TRY(cudaStreamSynchronize(d->lat->stream));
    if (d->comm.allreduce(d->comm.ctx, &v, 1) != 0)
        return fail(STAG_ERR_STATE, "domain decomposition: the communicator's allreduce failed");
    *out = v;
    return STAG_OK;
}

extern "C" int stag_ddr_dslash(stag_ddr d, stag_field out, stag_field in) {
    STAG_NVTX("stag_ddr_dslash");
    if (!d || !out || !in)
        return fail(STAG_ERR_ARG, "stag_ddr_dslash: NULL argument");
    stag_lattice lat = d->lat;
    if (out->lat != lat || in->lat != lat || out->parity == in->parity || out->prec != in->prec || out == in)
        return fail(STAG_ERR_ARG, "stag_ddr_dslash: need two fields of the rank's lattice, opposite parity, one "
                    "precision");
    const int prec = in->prec;
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_ddr_dslash: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    STAG_TRY(put_scalars(d, 0.0, 0.0, 0.0));  // running: the stencil's gate
    STAG_TRY(slab_dslash(d, prec, out->parity, EPI_NONE, in->data, out->data, nullptr, 0.0, nullptr));
    CUDA_TRY(cudaStreamSynchronize(lat->stream));
    return STAG_OK;
}

extern "C" int stag_ddr_cg_solve(stag_ddr d, stag_field x, const stag_field b, double mass, double rel_tol,
                                 int max_iter, stag_solve_info *info) {
    STAG_NVTX("stag_ddr_cg_solve");
    if (info)
        memset(info, 0, sizeof *info);
    if (!d || !x || !b)
        return fail(STAG_ERR_ARG, "stag_ddr_cg_solve: NULL argument");
    stag_lattice lat = d->lat;
    if (x->lat != lat || b->lat != lat || x->parity != STAG_EVEN || b->parity != STAG_EVEN || x->prec != b->prec ||
        x == b)
        return fail(STAG_ERR_ARG, "stag_ddr_cg_solve: x and b must be distinct even fields of the rank's lattice "
                    "and one precision");
    if (x->prec != STAG_F64 && x->prec != STAG_DF64)
        return fail(STAG_ERR_STATE, "stag_ddr_cg_solve: fields must be F64 or DF64 (got %s)", prec_name(x->prec));
    if (!(mass > 0) || !std::isfinite(mass) || !(rel_tol >= 0) || !std::isfinite(rel_tol) || max_iter < 0)
        return fail(STAG_ERR_ARG, "stag_ddr_cg_solve: need mass > 0, rel_tol >= 0, max_iter >= 0");
    const int prec = x->prec;
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_ddr_cg_solve: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    const auto t_start = std::chrono::steady_clock::now();
    STAG_TRY(ensure_cg_work(lat, prec));
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    const Geom sg = slab_geom(d);
    const double m2 = mass * mass;
    auto sl = [&](void *v) { return slab_ptr(d, prec, v); };

    // x = 0, r = b, p = b on the slab, and |b|^2 over the ranks
    STAG_TRY(put_scalars(d, 0.0, 0.0, 0.0));
    CUDA_TRY(launch_cg_init(prec, sg, sl(w.xw), sl(w.r), sl(w.p), sl(b->data), lat->partial, d->sc, s));
    double bb = 0.0;
    STAG_TRY(global_sum(d, offsetof(CgScalars, bb), &bb));
    const double stop = rel_tol * rel_tol * bb;
    {
        // the device scalars: running (the slab's kernels test nothing
        // themselves), |r|^2 = |b|^2; the global test lives in DdScal
        int st0 = !(bb < INFINITY) ? CG_BREAKDOWN : bb <= stop ? CG_CONVERGED : max_iter <= 0 ? CG_MAXITER
                                                                                             : CG_RUNNING;
        STAG_TRY(put_scalars(d, bb, 0.0, 0.0));
        CUDA_TRY(cudaMemcpyAsync(&d->sc->status, &st0, sizeof st0, cudaMemcpyHostToDevice, s));
        DdScal h;
        memset(&h, 0, sizeof h);
        h.rr_prev = bb;
        h.rr_stop = stop;
        h.max_iter = max_iter;
        CUDA_TRY(cudaMemcpyAsync(d->dd, &h, sizeof h, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaStreamSynchronize(s));  // pageable sources
    }
    // the iteration, enqueued in chunks: with a device allreduce the host
    // reads the status once per chunk, and iterations after the stop are
    // no-ops on every rank alike (the status derives from global sums only)
    const int chunk = d->comm.allreduce_dev ? 8 : 1;
    int enqueued = 0;
    for (;;) {
        CUDA_TRY(cudaMemcpyAsync(d->hsc, d->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (d->hsc->status != CG_RUNNING || enqueued >= max_iter)
            break;
        for (int k = 0; k < chunk && enqueued < max_iter; k++, enqueued++) {
            // t = D_oe p, then Ap = m^2 p - D_eo t with the slab's <p, Ap> partials
            int np = 0;
            STAG_TRY(slab_dslash(d, prec, STAG_ODD, EPI_NONE, w.p, w.t, nullptr, m2, nullptr));
            STAG_TRY(slab_dslash(d, prec, STAG_EVEN, EPI_M_PART, w.t, w.Ap, w.p, m2, &np));
            dd_pap_kernel<<<1, 256, 0, s>>>(d->partial, np, d->dd);
            CUDA_TRY(cudaGetLastError());
            STAG_TRY(allreduce_value(d, &d->dd->pap));
            dd_alpha_kernel<<<1, 1, 0, s>>>(d->sc, d->dd);
            CUDA_TRY(cudaGetLastError());
            // x += alpha p, r -= alpha Ap and the slab's |r|^2; then the global
            // |r|^2, beta and the stopping test; p = r + beta p
            CUDA_TRY(launch_cg_update(prec, sg, sl(w.xw), sl(w.r), sl(w.p), sl(w.Ap), lat->partial, d->sc, s));
            dd_rr_kernel<<<1, 1, 0, s>>>(d->sc, d->dd);
            CUDA_TRY(cudaGetLastError());
            STAG_TRY(allreduce_value(d, &d->dd->rr));
            dd_beta_kernel<<<1, 1, 0, s>>>(d->sc, d->dd);
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(launch_cg_p_update(prec, sg, sl(w.r), sl(w.p), d->sc, s));
        }
    }
    int status = d->hsc->status == CG_RUNNING ? CG_MAXITER : d->hsc->status;
    const int it = d->hsc->iter;
    double rr = 0.0;
    CUDA_TRY(cudaMemcpy(&rr, &d->dd->rr_prev, sizeof rr, cudaMemcpyDeviceToHost));
    // the slab of x, then |b - M x|^2 over all ranks
    CUDA_TRY(cudaMemcpyAsync(x->data, w.xw, x->bytes, cudaMemcpyDeviceToDevice, s));
    STAG_TRY(put_scalars(d, 0.0, 0.0, 0.0));
    STAG_TRY(slab_dslash(d, prec, STAG_ODD, EPI_NONE, x->data, w.t, nullptr, m2, nullptr));
    if (d->comm.size > 1)
        STAG_TRY(exchange_halo(d, prec, w.t, s));
    STAG_TRY(slab_range(d, prec, STAG_EVEN, EPI_RESID, w.t, nullptr, x->data, b->data, m2, d->slab.t0,
                        d->slab.nt, 0, 0, nullptr));
    double rr_true = 0.0;
    STAG_TRY(global_sum(d, offsetof(CgScalars, true_rr), &rr_true));
    stag_solve_info local;
    memset(&local, 0, sizeof local);
    local.iters = it;
    local.status = status == CG_CONVERGED ? STAG_OK
                   : status == CG_BREAKDOWN ? STAG_ERR_BREAKDOWN
                                            : STAG_ERR_NOT_CONVERGED;
    local.true_rel_resid = bb > 0 ? std::sqrt(rr_true / bb) : 0.0;
    local.iter_rel_resid = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    // model: the whole lattice's bytes of the plain CG
    const double rb = 8.0;
    if (local.seconds > 0) {
        local.gbs = (2.0 * 300 + 60) * rb * (double)lat->Vh * it / local.seconds / 1e9;
        local.gflops = (2.0 * 1146 + 72) * (double)lat->Vh * it / local.seconds / 1e9;
    }
    if (info)
        *info = local;
    if (local.status != STAG_OK)
        return fail(local.status, "stag_ddr_cg_solve: %s after %d iterations (|r|/|b| = %.3e)",
                    local.status == STAG_ERR_BREAKDOWN ? "breakdown" : "not converged", it, local.iter_rel_resid);
    return STAG_OK;
}
