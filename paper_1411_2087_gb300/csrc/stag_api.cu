// libstag C ABI: handles, argument checking, memory, uploads, Dslash and the
// plain CG solve graph.  The other solvers are in solvers.cu, the learned
// preconditioner in learned.cu; declarations and documentation in
// include/stag.h.
#include "api_internal.h"

#include <cstdint>

// --------------------------------------------------------------------------
// errors
// --------------------------------------------------------------------------
static thread_local std::string g_last_error;

namespace stag {
void set_error_message(const char *msg) { g_last_error = msg; }

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}
}  // namespace stag

// --------------------------------------------------------------------------
// lattice
// --------------------------------------------------------------------------
extern "C" int stag_lattice_create(stag_lattice *out, const int dims[4], const double bc[4],
                                   int device, void *cuda_stream) {
    if (!out)
        return fail(STAG_ERR_ARG, "stag_lattice_create: out is NULL");
    *out = nullptr;
    if (!dims)
        return fail(STAG_ERR_ARG, "stag_lattice_create: dims is NULL");
    long long V = 1;
    for (int k = 0; k < 4; k++) {
        if (dims[k] < 2 || dims[k] % 2)
            return fail(STAG_ERR_ARG, "stag_lattice_create: dims[%d] = %d must be even and >= 2", k,
                        dims[k]);
        V *= dims[k];
        if (V > (1LL << 31) - 2)
            return fail(STAG_ERR_ARG, "stag_lattice_create: volume too large");
    }
    // 72 component planes of one parity must be addressable with 32-bit offsets
    const long long Vh = V / 2;
    const long long stride = (Vh + 255) / 256 * 256;
    if (72 * stride >= (1LL << 31))
        return fail(STAG_ERR_ARG, "stag_lattice_create: volume too large for 32-bit link offsets");
    double bcv[4] = {1.0, 1.0, 1.0, -1.0};
    if (bc) {
        for (int k = 0; k < 4; k++) {
            if (bc[k] != 1.0 && bc[k] != -1.0)
                return fail(STAG_ERR_ARG, "stag_lattice_create: bc[%d] = %g must be +1 or -1", k, bc[k]);
            bcv[k] = bc[k];
        }
    }
    if (device < 0)
        return fail(STAG_ERR_ARG, "stag_lattice_create: device %d < 0", device);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(STAG_ERR_CUDA, "stag_lattice_create: no CUDA device available");
    }
    if (device >= ndev)
        return fail(STAG_ERR_ARG, "stag_lattice_create: device %d >= device count %d", device, ndev);

    DEVICE_SCOPE(device);
    stag_lattice lat = new (std::nothrow) stag_lattice_s();
    if (!lat)
        return fail(STAG_ERR_NOMEM, "stag_lattice_create: host allocation failed");
    lat->device = device;
    for (int k = 0; k < 4; k++) {
        lat->dims[k] = dims[k];
        lat->bc[k] = bcv[k];
    }
    lat->V = V;
    lat->Vh = Vh;
    lat->geom = geom_of(dims, stride);

    auto cleanup = [&](int code) {
        stag_lattice_destroy(lat);
        return code;
    };
    cudaError_t e;
    if (cuda_stream) {
        lat->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&lat->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess)
            return cleanup(fail(STAG_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
        lat->own_stream = true;
    }
    const int nblk = (int)((Vh + 63) / 64) + 1;
    if ((e = cudaMalloc(&lat->partial, sizeof(double) * nblk)) != cudaSuccess ||
        (e = cudaMalloc(&lat->sc, sizeof(CgScalars))) != cudaSuccess ||
        (e = cudaMemset(lat->sc, 0, sizeof(CgScalars))) != cudaSuccess ||
        (e = cudaMallocHost(&lat->sc_host, sizeof(CgScalars))) != cudaSuccess ||
        (e = cudaEventCreate(&lat->ev0)) != cudaSuccess ||
        (e = cudaEventCreate(&lat->ev1)) != cudaSuccess)
        return cleanup(fail(STAG_ERR_NOMEM, "stag_lattice_create: %s", cudaGetErrorString(e)));
    memset(lat->sc_host, 0, sizeof(CgScalars));
    *out = lat;
    return STAG_OK;
}

extern "C" int stag_lattice_destroy(stag_lattice lat) {
    if (!lat)
        return STAG_OK;
    if (lat->live_fields > 0)
        return fail(STAG_ERR_STATE, "stag_lattice_destroy: %d fields still alive", lat->live_fields);
    DEVICE_SCOPE(lat->device);
    if (lat->stream)
        cudaStreamSynchronize(lat->stream);
    for (int p = 0; p < 4; p++) {
        free_cg(lat->cg[p]);
        if (lat->links[p])
            cudaFree(lat->links[p]);
        if (lat->links_c12[p])
            cudaFree(lat->links_c12[p]);
    }
    if (lat->partial)
        cudaFree(lat->partial);
    if (lat->staging)
        cudaFree(lat->staging);
    if (lat->xs)
        cudaFree(lat->xs);
    if (lat->ms_state)
        cudaFree(lat->ms_state);
    if (lat->ms_state_host)
        cudaFreeHost(lat->ms_state_host);
    if (lat->ms_true)
        cudaFree(lat->ms_true);
    if (lat->ms_true_host)
        cudaFreeHost(lat->ms_true_host);
    for (int q = 0; q < 4; q++) {
        for (int k = 0; k < MS_MAX; k++)
            if (lat->ms_p[q][k])
                cudaFree(lat->ms_p[q][k]);
        if (lat->ms_rhi[q])
            cudaFree(lat->ms_rhi[q]);
        if (lat->ms_ehi[q])
            cudaFree(lat->ms_ehi[q]);
    }
    for (int k = 0; k < MS_MAX; k++)
        if (lat->ms_xlo[k])
            cudaFree(lat->ms_xlo[k]);
    for (int q = 0; q < 4; q++)
        for (int k = 0; k < BATCH_MAX_G * BATCH_KMAX; k++)
            for (int v = 0; v < 4; v++)
                if (lat->bwork[q][k][v])
                    cudaFree(lat->bwork[q][k][v]);
    for (int k = 0; k < BATCH_MAX_G * BATCH_KMAX; k++) {
        if (lat->bxlo[k])
            cudaFree(lat->bxlo[k]);
        if (lat->bblo[k])
            cudaFree(lat->bblo[k]);
    }
    if (lat->ms_blo)
        cudaFree(lat->ms_blo);
    if (lat->absmax)
        cudaFree(lat->absmax);
    for (int h = 0; h < 4; h++)
        for (int l = 0; l < 4; l++) {
            if (lat->mixed[h][l].exec)
                cudaGraphExecDestroy(lat->mixed[h][l].exec);
            if (lat->mixed[h][l].graph)
                cudaGraphDestroy(lat->mixed[h][l].graph);
        }
    if (lat->sc)
        cudaFree(lat->sc);
    if (lat->sc_host)
        cudaFreeHost(lat->sc_host);
    if (lat->ev0)
        cudaEventDestroy(lat->ev0);
    if (lat->ev1)
        cudaEventDestroy(lat->ev1);
    if (lat->own_stream && lat->stream)
        cudaStreamDestroy(lat->stream);
    delete lat;
    return STAG_OK;
}

extern "C" int stag_lattice_volume(const stag_lattice lat, long long *V, long long *Vh) {
    if (!lat)
        return fail(STAG_ERR_ARG, "stag_lattice_volume: lattice is NULL");
    if (V)
        *V = lat->V;
    if (Vh)
        *Vh = lat->Vh;
    return STAG_OK;
}

extern "C" int stag_lattice_set_cg_launch(stag_lattice lat, int mode, int chunk) {
    if (!lat)
        return fail(STAG_ERR_ARG, "stag_lattice_set_cg_launch: lattice is NULL");
    if (mode != STAG_CG_LAUNCH_GRAPH && mode != STAG_CG_LAUNCH_HOST)
        return fail(STAG_ERR_ARG, "stag_lattice_set_cg_launch: bad mode %d", mode);
    if (mode == STAG_CG_LAUNCH_HOST && (chunk < 1 || chunk > 4096))
        return fail(STAG_ERR_ARG, "stag_lattice_set_cg_launch: chunk must be in [1, 4096]");
    lat->cg_launch = mode;
    if (mode == STAG_CG_LAUNCH_HOST)
        lat->cg_chunk = chunk;
    return STAG_OK;
}

// --------------------------------------------------------------------------
// gauge upload
// --------------------------------------------------------------------------

// device copy of a canonical gauge field: returns a device pointer, allocating
// a temporary when the source is on the host
static int gauge_to_device(stag_lattice lat, const double *src, int ptr_kind, double **dev,
                           bool *owned) {
    const size_t bytes = 4ull * lat->V * 18 * sizeof(double);
    if (ptr_kind == STAG_PTR_DEVICE) {
        *dev = (double *)src;
        *owned = false;
        return STAG_OK;
    }
    CUDA_TRY(cudaMalloc(dev, bytes));
    *owned = true;
    cudaError_t e = cudaMemcpyAsync(*dev, src, bytes, cudaMemcpyHostToDevice, lat->stream);
    if (e != cudaSuccess) {
        cudaFree(*dev);
        *dev = nullptr;
        return fail(STAG_ERR_CUDA, "gauge copy to device: %s", cudaGetErrorString(e));
    }
    return STAG_OK;
}

extern "C" int stag_gauge_upload(stag_lattice lat, const double *fat, const double *lng, double c1,
                                 double c3, int ptr_kind, unsigned prec_mask) {
    STAG_NVTX("stag_gauge_upload");
    if (!lat || !fat)
        return fail(STAG_ERR_ARG, "stag_gauge_upload: lattice or fat links NULL");
    if (ptr_kind != STAG_PTR_HOST && ptr_kind != STAG_PTR_DEVICE)
        return fail(STAG_ERR_ARG, "stag_gauge_upload: bad ptr_kind %d", ptr_kind);
    if (!std::isfinite(c1) || !std::isfinite(c3))
        return fail(STAG_ERR_ARG, "stag_gauge_upload: coefficients must be finite");
    if ((prec_mask & STAG_COMPRESS12) && (prec_mask & STAG_COMPRESS12_LONG))
        return fail(STAG_ERR_ARG, "stag_gauge_upload: STAG_COMPRESS12 and STAG_COMPRESS12_LONG exclude each other");
    // which link groups take the 12-real layout: bit 0 one-link, bit 1 three-link
    const int cmask = (prec_mask & STAG_COMPRESS12) ? 3 : (prec_mask & STAG_COMPRESS12_LONG) ? 2 : 0;
    const bool compress = cmask != 0;
    prec_mask &= ~(unsigned)(STAG_COMPRESS12 | STAG_COMPRESS12_LONG);
    if (prec_mask == 0)
        prec_mask = STAG_PREC_BIT(STAG_F64) | STAG_PREC_BIT(STAG_DF64);
    for (int p = 0; p < 32; p++)
        if ((prec_mask >> p) & 1u)
            if (!prec_valid(p))
                return fail(STAG_ERR_ARG, "stag_gauge_upload: precision %d (%s) not available", p,
                            prec_name(p));
    if (compress && !(prec_mask & (STAG_PREC_BIT(STAG_F32) | STAG_PREC_BIT(STAG_F16))))
        return fail(STAG_ERR_ARG, "stag_gauge_upload: 12-real compression applies to F32 and F16 copies only");
    if (compress && (((cmask & 1) && c1 == 0.0) || c3 == 0.0))
        return fail(STAG_ERR_ARG, "stag_gauge_upload: 12-real compression needs a nonzero coefficient on the "
                    "compressed links");
    DEVICE_SCOPE(lat->device);
    // device sources may have been written on any stream of the caller
    if (ptr_kind == STAG_PTR_DEVICE)
        CUDA_TRY(cudaDeviceSynchronize());
    double *fat_d = nullptr, *lng_d = nullptr;
    bool fat_owned = false, lng_owned = false;
    int st = gauge_to_device(lat, fat, ptr_kind, &fat_d, &fat_owned);
    if (st != STAG_OK)
        return st;
    auto release = [&]() {
        cudaStreamSynchronize(lat->stream);
        if (fat_owned)
            cudaFree(fat_d);
        if (lng_owned)
            cudaFree(lng_d);
    };
    if (lng) {
        st = gauge_to_device(lat, lng, ptr_kind, &lng_d, &lng_owned);
    } else {
        cudaError_t e = cudaMalloc(&lng_d, 4ull * lat->V * 18 * sizeof(double));
        if (e == cudaSuccess) {
            lng_owned = true;
            e = launch_long_links(lat->geom, fat_d, lng_d, lat->stream);
        }
        if (e != cudaSuccess)
            st = fail(STAG_ERR_CUDA, "long-link build: %s", cudaGetErrorString(e));
    }
    if (st != STAG_OK) {
        release();
        return st;
    }
    // drop old copies and solver graphs; until the new copies exist the
    // lattice has no gauge field
    cudaStreamSynchronize(lat->stream);
    lat->has_gauge = false;
    for (int p = 0; p < 4; p++) {
        free_cg(lat->cg[p]);
        if (lat->links[p]) {
            cudaFree(lat->links[p]);
            lat->links[p] = nullptr;
        }
        if (lat->links_c12[p]) {
            cudaFree(lat->links_c12[p]);
            lat->links_c12[p] = nullptr;
        }
        lat->c12_mask[p] = 0;
    }
    drop_mixed_graphs(lat);
    if (compress) {
        // the 12-real form rebuilds row 3 from rows 1 and 2: only valid for
        // links in SU(3) (the paper's Sec. 4 notes smeared links are not)
        unsigned *dev_bits = nullptr;
        cudaError_t e = cudaMalloc(&dev_bits, 2 * sizeof(unsigned));
        if (e == cudaSuccess)
            e = launch_su3_deviation(fat_d, 4LL * lat->V, dev_bits, lat->stream);
        if (e == cudaSuccess)
            e = launch_su3_deviation(lng_d, 4LL * lat->V, dev_bits + 1, lat->stream);
        unsigned bits[2] = {0u, 0u};
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bits, dev_bits, sizeof bits, cudaMemcpyDeviceToHost, lat->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(lat->stream);
        if (dev_bits)
            cudaFree(dev_bits);
        if (e != cudaSuccess) {
            release();
            return fail(STAG_ERR_CUDA, "SU(3) check: %s", cudaGetErrorString(e));
        }
        float dev[2];
        memcpy(dev, bits, sizeof dev);
        if (((cmask & 1) && !(dev[0] <= 1e-6f)) || !(dev[1] <= 1e-6f)) {
            release();
            return fail(STAG_ERR_ARG, "stag_gauge_upload: links deviate from SU(3) by %.2e (fat) / %.2e (long); "
                        "12-real compression needs special unitary links%s", dev[0], dev[1],
                        (cmask & 1) ? " (STAG_COMPRESS12_LONG compresses the long links only)" : "");
        }
    }
    lat->has_gauge = false;
    float inv_scale[2] = {0.f, 0.f};
    {
        // largest |entry| of each field: rejects non-finite links, and is the
        // scale of the 16-bit copy (one per field, after folding)
        cudaError_t e = lat->absmax ? cudaSuccess : cudaMalloc(&lat->absmax, 2 * sizeof(unsigned));
        const long long n = 4LL * lat->V * 18;
        if (e == cudaSuccess)
            e = launch_absmax(fat_d, n, lat->absmax, lat->stream);
        if (e == cudaSuccess)
            e = launch_absmax(lng_d, n, lat->absmax + 1, lat->stream);
        unsigned bits[2] = {0u, 0u};
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bits, lat->absmax, sizeof bits, cudaMemcpyDeviceToHost, lat->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(lat->stream);
        if (e != cudaSuccess) {
            release();
            return fail(STAG_ERR_CUDA, "16-bit link scales: %s", cudaGetErrorString(e));
        }
        const double cf[2] = {std::fabs(c1), std::fabs(c3)};
        for (int h = 0; h < 2; h++) {
            float m;
            memcpy(&m, &bits[h], sizeof m);
            if (!std::isfinite(m)) {
                release();
                return fail(STAG_ERR_ARG, "stag_gauge_upload: the %s links hold NaN, infinite or out-of-range "
                            "entries", h ? "long" : "fat");
            }
            if ((prec_mask >> STAG_F16) & 1u) {
                const double mx = (double)m * cf[h];
                lat->link_scale[h] = mx > 0 ? (float)(mx / 32767.0) : 0.f;
                inv_scale[h] = mx > 0 ? (float)(32767.0 / mx) : 0.f;
            }
        }
    }
    for (int p = 0; p < 4; p++) {
        if (!((prec_mask >> p) & 1u))
            continue;
        cudaError_t e = cudaMalloc(&lat->links[p], link_bytes(lat, p));
        if (e == cudaSuccess)
            e = cudaMemsetAsync(lat->links[p], 0, link_bytes(lat, p), lat->stream);
        if (e == cudaSuccess)
            e = launch_fold_links(p, lat->geom, lat->bc, c1, c3, fat_d, lng_d, lat->links[p], inv_scale,
                                  lat->stream);
        if (e == cudaSuccess && compress && (p == STAG_F32 || p == STAG_F16)) {
            const size_t cb = c12_link_bytes(p, (size_t)lat->geom.stride, cmask);
            e = cudaMalloc(&lat->links_c12[p], cb);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(lat->links_c12[p], 0, cb, lat->stream);
            if (e == cudaSuccess)
                e = launch_fold_links_c12(p, lat->geom, lat->bc, c1, c3, fat_d, lng_d, lat->links_c12[p],
                                          inv_scale, cmask, lat->stream);
            if (e == cudaSuccess)
                lat->c12_mask[p] = cmask;
        }
        if (e != cudaSuccess) {
            release();
            return fail(e == cudaErrorMemoryAllocation ? STAG_ERR_NOMEM : STAG_ERR_CUDA,
                        "gauge fold (%s): %s", prec_name(p), cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaStreamSynchronize(lat->stream);
    release();
    if (e != cudaSuccess)
        return fail(STAG_ERR_CUDA, "stag_gauge_upload: %s", cudaGetErrorString(e));
    lat->has_gauge = true;
    lat->c1 = c1;
    lat->c3 = c3;
    return STAG_OK;
}

extern "C" int stag_long_links_build(stag_lattice lat, const double *fat, double *lng, int ptr_kind) {
    STAG_NVTX("stag_long_links_build");
    if (!lat || !fat || !lng)
        return fail(STAG_ERR_ARG, "stag_long_links_build: NULL argument");
    if (ptr_kind != STAG_PTR_HOST && ptr_kind != STAG_PTR_DEVICE)
        return fail(STAG_ERR_ARG, "stag_long_links_build: bad ptr_kind %d", ptr_kind);
    DEVICE_SCOPE(lat->device);
    if (ptr_kind == STAG_PTR_DEVICE)
        CUDA_TRY(cudaDeviceSynchronize());
    const size_t bytes = 4ull * lat->V * 18 * sizeof(double);
    double *fat_d = nullptr;
    bool owned = false;
    STAG_TRY(gauge_to_device(lat, fat, ptr_kind, &fat_d, &owned));
    double *out_d = (double *)lng;
    cudaError_t e = cudaSuccess;
    if (ptr_kind == STAG_PTR_HOST)
        e = cudaMalloc(&out_d, bytes);
    if (e == cudaSuccess)
        e = launch_long_links(lat->geom, fat_d, out_d, lat->stream);
    if (e == cudaSuccess && ptr_kind == STAG_PTR_HOST)
        e = cudaMemcpyAsync(lng, out_d, bytes, cudaMemcpyDeviceToHost, lat->stream);
    cudaError_t e2 = cudaStreamSynchronize(lat->stream);
    if (owned)
        cudaFree(fat_d);
    if (ptr_kind == STAG_PTR_HOST && out_d)
        cudaFree(out_d);
    if (e == cudaSuccess)
        e = e2;
    if (e != cudaSuccess)
        return fail(STAG_ERR_CUDA, "stag_long_links_build: %s", cudaGetErrorString(e));
    return STAG_OK;
}

// --------------------------------------------------------------------------
// fields
// --------------------------------------------------------------------------
extern "C" int stag_field_create(stag_lattice lat, int parity, int prec, stag_field *out) {
    if (!out)
        return fail(STAG_ERR_ARG, "stag_field_create: out is NULL");
    *out = nullptr;
    if (!lat)
        return fail(STAG_ERR_ARG, "stag_field_create: lattice is NULL");
    if (parity != STAG_EVEN && parity != STAG_ODD)
        return fail(STAG_ERR_ARG, "stag_field_create: bad parity %d", parity);
    if (!prec_valid(prec))
        return fail(STAG_ERR_ARG, "stag_field_create: precision %d (%s) not available", prec,
                    prec_name(prec));
    DEVICE_SCOPE(lat->device);
    stag_field f = new (std::nothrow) stag_field_s();
    if (!f)
        return fail(STAG_ERR_NOMEM, "stag_field_create: host allocation failed");
    f->lat = lat;
    f->parity = parity;
    f->prec = prec;
    f->bytes = field_bytes(lat, prec);
    cudaError_t e = cudaMalloc(&f->data, f->bytes);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(f->data, 0, f->bytes, lat->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) {
        if (f->data)
            cudaFree(f->data);
        delete f;
        return fail(e == cudaErrorMemoryAllocation ? STAG_ERR_NOMEM : STAG_ERR_CUDA,
                    "stag_field_create: %s", cudaGetErrorString(e));
    }
    lat->live_fields++;
    *out = f;
    return STAG_OK;
}

extern "C" int stag_field_bytes(stag_lattice lat, int prec, unsigned long long *bytes) {
    if (!lat || !bytes)
        return fail(STAG_ERR_ARG, "stag_field_bytes: NULL argument");
    if (!prec_valid(prec))
        return fail(STAG_ERR_ARG, "stag_field_bytes: bad precision %d", prec);
    *bytes = field_bytes(lat, prec);
    return STAG_OK;
}

extern "C" int stag_field_wrap(stag_lattice lat, int parity, int prec, void *dev_ptr, unsigned long long bytes,
                               stag_field *out) {
    if (!out)
        return fail(STAG_ERR_ARG, "stag_field_wrap: out is NULL");
    *out = nullptr;
    if (!lat || !dev_ptr)
        return fail(STAG_ERR_ARG, "stag_field_wrap: NULL argument");
    if (parity != STAG_EVEN && parity != STAG_ODD)
        return fail(STAG_ERR_ARG, "stag_field_wrap: bad parity %d", parity);
    if (!prec_valid(prec))
        return fail(STAG_ERR_ARG, "stag_field_wrap: bad precision %d", prec);
    const size_t need = field_bytes(lat, prec);
    if (bytes < need)
        return fail(STAG_ERR_ARG, "stag_field_wrap: %llu bytes given, %zu needed", bytes, need);
    if ((uintptr_t)dev_ptr % 16 != 0)
        return fail(STAG_ERR_ARG, "stag_field_wrap: the buffer must be 16-byte aligned");
    DEVICE_SCOPE(lat->device);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, dev_ptr) != cudaSuccess) {
        cudaGetLastError();
        return fail(STAG_ERR_ARG, "stag_field_wrap: not a CUDA pointer");
    }
    if ((attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) || attr.device != lat->device)
        return fail(STAG_ERR_ARG, "stag_field_wrap: the buffer is not device memory of device %d", lat->device);
    stag_field f = new (std::nothrow) stag_field_s();
    if (!f)
        return fail(STAG_ERR_NOMEM, "stag_field_wrap: host allocation failed");
    f->lat = lat;
    f->parity = parity;
    f->prec = prec;
    f->bytes = need;
    f->data = dev_ptr;
    f->owned = false;
    lat->live_fields++;
    *out = f;
    return STAG_OK;
}

extern "C" int stag_field_destroy(stag_field f) {
    if (!f)
        return STAG_OK;
    DEVICE_SCOPE(f->lat->device);
    cudaStreamSynchronize(f->lat->stream);
    if (f->owned)
        cudaFree(f->data);
    f->lat->live_fields--;
    delete f;
    return STAG_OK;
}

static int field_io(stag_field f, const double *src, double *dst, int ptr_kind) {
    stag_lattice lat = f->lat;
    DEVICE_SCOPE(lat->device);
    const size_t bytes = (size_t)lat->Vh * 6 * sizeof(double);
    double *canon = nullptr;
    cudaError_t e = cudaSuccess;
    if (ptr_kind == STAG_PTR_DEVICE) {
        canon = src ? (double *)src : dst;
        // a device source may still be written by work on another stream
        // (the caller's): let all of it finish before the lattice stream reads
        if (src)
            e = cudaDeviceSynchronize();
    } else {
        if (!lat->staging)
            e = cudaMalloc(&lat->staging, bytes);
        canon = lat->staging;
        if (e == cudaSuccess && src)
            e = cudaMemcpyAsync(canon, src, bytes, cudaMemcpyHostToDevice, lat->stream);
    }
    if (e == cudaSuccess && src && f->prec != STAG_F64) {
        // the float-based formats hold entries up to the FP32 range only
        if (!lat->absmax)
            e = cudaMalloc(&lat->absmax, 2 * sizeof(unsigned));
        unsigned flag = 0;
        if (e == cudaSuccess)
            e = launch_finite_overflow(canon, (long long)lat->Vh * 6, lat->absmax, lat->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&flag, lat->absmax, sizeof flag, cudaMemcpyDeviceToHost, lat->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(lat->stream);
        if (e == cudaSuccess && flag)
            return fail(STAG_ERR_ARG, "field import: a finite entry lies beyond the FP32 range of a %s field "
                        "(the field is unchanged)", prec_name(f->prec));
    }
    if (e == cudaSuccess)
        e = src ? launch_import(f->prec, lat->geom, canon, f->data, lat->stream)
                : launch_export(f->prec, lat->geom, f->data, canon, lat->stream);
    if (e == cudaSuccess && dst && ptr_kind == STAG_PTR_HOST)
        e = cudaMemcpyAsync(dst, canon, bytes, cudaMemcpyDeviceToHost, lat->stream);
    cudaError_t e2 = cudaStreamSynchronize(lat->stream);
    if (e == cudaSuccess)
        e = e2;
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? STAG_ERR_NOMEM : STAG_ERR_CUDA,
                    "field %s: %s", src ? "import" : "export", cudaGetErrorString(e));
    return STAG_OK;
}

extern "C" int stag_field_import(stag_field f, const double *src, int ptr_kind) {
    STAG_NVTX("stag_field_import");
    if (!f || !src)
        return fail(STAG_ERR_ARG, "stag_field_import: NULL argument");
    if (ptr_kind != STAG_PTR_HOST && ptr_kind != STAG_PTR_DEVICE)
        return fail(STAG_ERR_ARG, "stag_field_import: bad ptr_kind %d", ptr_kind);
    return field_io(f, src, nullptr, ptr_kind);
}

extern "C" int stag_field_export(const stag_field f, double *dst, int ptr_kind) {
    STAG_NVTX("stag_field_export");
    if (!f || !dst)
        return fail(STAG_ERR_ARG, "stag_field_export: NULL argument");
    if (ptr_kind != STAG_PTR_HOST && ptr_kind != STAG_PTR_DEVICE)
        return fail(STAG_ERR_ARG, "stag_field_export: bad ptr_kind %d", ptr_kind);
    return field_io((stag_field)f, nullptr, dst, ptr_kind);
}

extern "C" int stag_field_zero(stag_field f) {
    if (!f)
        return fail(STAG_ERR_ARG, "stag_field_zero: NULL field");
    DEVICE_SCOPE(f->lat->device);
    CUDA_TRY(cudaMemsetAsync(f->data, 0, f->bytes, f->lat->stream));
    return STAG_OK;
}

extern "C" int stag_field_storage(const stag_field f, void **dev_ptr, unsigned long long *bytes) {
    if (!f)
        return fail(STAG_ERR_ARG, "stag_field_storage: NULL field");
    if (dev_ptr)
        *dev_ptr = f->data;
    if (bytes)
        *bytes = f->bytes;
    return STAG_OK;
}

// --------------------------------------------------------------------------
// Dslash and M
// --------------------------------------------------------------------------
static int check_pair(stag_lattice lat, const stag_field out, const stag_field in, int out_par,
                      const char *who) {
    if (!lat || !out || !in)
        return fail(STAG_ERR_ARG, "%s: NULL argument", who);
    if (out->lat != lat || in->lat != lat)
        return fail(STAG_ERR_ARG, "%s: field belongs to another lattice", who);
    if (out->parity != out_par || in->parity != 1 - out_par)
        return fail(STAG_ERR_STATE, "%s: parity mismatch (out %d, in %d)", who, out->parity,
                    in->parity);
    if (out->prec != in->prec)
        return fail(STAG_ERR_STATE, "%s: precision mismatch (%s vs %s)", who, prec_name(out->prec),
                    prec_name(in->prec));
    if (out == in)
        return fail(STAG_ERR_ARG, "%s: out and in must differ", who);
    if (!lat->has_gauge || !lat->links[out->prec])
        return fail(STAG_ERR_STATE, "%s: no %s gauge copy uploaded", who, prec_name(out->prec));
    return STAG_OK;
}

static int dslash_impl(stag_lattice lat, stag_field out, const stag_field in, int out_par,
                       const char *who) {
    STAG_TRY(check_pair(lat, out, in, out_par, who));
    DEVICE_SCOPE(lat->device);
    DslashArgs a = dslash_args(lat, out->prec, out_par, in->data, out->data);
    CUDA_TRY(launch_dslash(out->prec, EPI_NONE, a, lat->dslash_block[out->prec], lat->stream));
    return STAG_OK;
}

extern "C" int stag_dslash_eo(stag_lattice lat, stag_field out_even, const stag_field in_odd) {
    STAG_NVTX("stag_dslash_eo");
    return dslash_impl(lat, out_even, in_odd, STAG_EVEN, "stag_dslash_eo");
}

extern "C" int stag_dslash_oe(stag_lattice lat, stag_field out_odd, const stag_field in_even) {
    STAG_NVTX("stag_dslash_oe");
    return dslash_impl(lat, out_odd, in_even, STAG_ODD, "stag_dslash_oe");
}

// odd temporary of the CG workspace of one precision
extern "C" int stag_apply_M(stag_lattice lat, stag_field out_even, const stag_field in_even,
                            double mass) {
    STAG_NVTX("stag_apply_M");
    if (!lat || !out_even || !in_even)
        return fail(STAG_ERR_ARG, "stag_apply_M: NULL argument");
    if (out_even->parity != STAG_EVEN || in_even->parity != STAG_EVEN)
        return fail(STAG_ERR_STATE, "stag_apply_M: fields must be even");
    if (out_even->prec != in_even->prec)
        return fail(STAG_ERR_STATE, "stag_apply_M: precision mismatch");
    if (out_even == in_even)
        return fail(STAG_ERR_ARG, "stag_apply_M: out and in must differ");
    if (!std::isfinite(mass))
        return fail(STAG_ERR_ARG, "stag_apply_M: mass must be finite");
    const int prec = in_even->prec;
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_apply_M: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    STAG_TRY(ensure_cg_work(lat, prec));
    CgWork &w = lat->cg[prec];
    DslashArgs a1 = dslash_args(lat, prec, STAG_ODD, in_even->data, w.t);
    CUDA_TRY(launch_dslash(prec, EPI_NONE, a1, lat->dslash_block[prec], lat->stream));
    DslashArgs a2 = dslash_args(lat, prec, STAG_EVEN, w.t, out_even->data);
    a2.p = in_even->data;
    a2.m2 = make_dpair(mass * mass);
    a2.m2_in_args = 1;
    CUDA_TRY(launch_dslash(prec, EPI_M, a2, lat->dslash_block[prec], lat->stream));
    return STAG_OK;
}

// --------------------------------------------------------------------------
// CG solve graph:
//   init (x=0, r=p=b, |b|^2)
//   while (running) { t = D_oe p; Ap = m^2 p - D_eo t, alpha;
//                     x += alpha p, r -= alpha Ap, beta; p = r + beta p }
//   true residual |b - M x|^2
// --------------------------------------------------------------------------
cudaError_t enqueue_cg_body(stag_lattice lat, CgWork &w, cudaStream_t s, bool skip_if_done) {
    const int prec = w.prec;
    cudaError_t e;
    DslashArgs a1 = dslash_args(lat, prec, STAG_ODD, w.p, w.t);
    a1.skip_if_done = skip_if_done;
    if ((e = launch_dslash(prec, EPI_NONE, a1, lat->dslash_block[prec], s)) != cudaSuccess)
        return e;
    // Ap = M p with one partial of <p, Ap> per block; a one-block kernel sums
    // them (cheaper at these grid sizes than a last-block ticket in the Dslash)
    if ((e = enqueue_m_pap(lat, prec, w.t, w.Ap, w.p, skip_if_done, s)) != cudaSuccess)
        return e;
    if ((e = launch_cg_update(prec, lat->geom, w.xw, w.r, w.p, w.Ap, lat->partial, lat->sc, s)) !=
        cudaSuccess)
        return e;
    return launch_cg_p_update(prec, lat->geom, w.r, w.p, lat->sc, s);
}

static cudaError_t enqueue_true_residual(stag_lattice lat, CgWork &w, cudaStream_t s) {
    const int prec = w.prec;
    cudaError_t e;
    DslashArgs a1 = dslash_args(lat, prec, STAG_ODD, w.xw, w.t);
    if ((e = launch_dslash(prec, EPI_NONE, a1, lat->dslash_block[prec], s)) != cudaSuccess)
        return e;
    DslashArgs a2 = dslash_args(lat, prec, STAG_EVEN, w.t, nullptr);
    a2.p = w.xw;
    a2.b = w.bw;
    return launch_dslash(prec, EPI_RESID, a2, lat->dslash_block[prec], s);
}

static int build_cg_graph(stag_lattice lat, CgWork &w) {
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
            if (junk && junk != graph)
                cudaGraphDestroy(junk);
        }
        cudaGetLastError();
        cudaGraphDestroy(graph);
        return fail(STAG_ERR_CUDA, "CG graph (%s): %s", what, cudaGetErrorString(err));
    };
    // init, then the loop node, then the true residual, captured into `graph`
    if ((e = cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail("begin capture", e);
    if ((e = launch_cg_init(w.prec, lat->geom, w.xw, w.r, w.p, w.bw, lat->partial, lat->sc, s)) !=
        cudaSuccess)
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
    if ((e = enqueue_true_residual(lat, w, s)) != cudaSuccess)
        return bail("true residual", e);
    cudaGraph_t captured = nullptr;
    if ((e = cudaStreamEndCapture(s, &captured)) != cudaSuccess)
        return bail("end capture", e);
    // loop body
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail("begin body capture", e);
    if ((e = enqueue_cg_body(lat, w, s, false)) != cudaSuccess)
        return bail("body", e);
    cudaGraph_t body_out = nullptr;
    if ((e = cudaStreamEndCapture(s, &body_out)) != cudaSuccess)
        return bail("end body capture", e);
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
        return bail("instantiate", e);
    w.graph = graph;
    w.exec = exec;
    w.cond = cond;
    return STAG_OK;
}

static void fill_info(stag_lattice lat, int prec, const CgScalars &h, float ms,
                      stag_solve_info *info) {
    if (!info)
        return;
    memset(info, 0, sizeof *info);
    info->iters = h.iter;
    info->status = h.status == CG_CONVERGED ? STAG_OK
                   : h.status == CG_BREAKDOWN ? STAG_ERR_BREAKDOWN
                                              : STAG_ERR_NOT_CONVERGED;
    info->true_rel_resid = h.bb > 0 ? std::sqrt(h.true_rr / h.bb) : 0.0;
    info->iter_rel_resid = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
    info->seconds = ms * 1e-3;
    const double rb = prec == STAG_F32 ? 4.0 : 8.0;
    // per iteration and even site: two Dslash (1146 flops, 300 reals each)
    // plus the vector passes (p read again, x/r/p/Ap update, p update)
    const double flops = (2.0 * 1146 + 72) * (double)lat->Vh * h.iter;
    const double bytes = (2.0 * 300 + 60) * rb * (double)lat->Vh * h.iter;
    if (ms > 0) {
        info->gflops = flops / (ms * 1e-3) / 1e9;
        info->gbs = bytes / (ms * 1e-3) / 1e9;
    }
}

// --------------------------------------------------------------------------
// source normalisation of the solvers
// --------------------------------------------------------------------------
// Double-float and FP32 keep the float exponent range, so a source whose
// entries are far from 1 would push the residual's squares out of it as the
// solve proceeds.  When the exponent of b's largest entry lies outside
// [-kRhsWindow, kRhsWindow], the solve runs on a copy b 2^-k and the solution
// is multiplied by 2^k afterwards; powers of two scale every intermediate
// exactly, so the arithmetic is that of the unscaled solve wherever the
// latter stays in range.  FP64 fields are left alone.
constexpr int kRhsWindow = 16;

int rhs_scale_begin(const stag_field b, RhsScale *rs) {
    rs->k = 0;
    rs->scaled = nullptr;
    if (b->prec != STAG_DF64 && b->prec != STAG_F32)
        return STAG_OK;  // FP64 has the range; 16-bit fields carry a norm per site
    stag_lattice lat = b->lat;
    DEVICE_SCOPE(lat->device);
    if (!lat->absmax)
        CUDA_TRY(cudaMalloc(&lat->absmax, 2 * sizeof(unsigned)));
    unsigned bits = 0;
    CUDA_TRY(launch_field_absmax(b->prec, lat->geom, b->data, lat->absmax, lat->stream));
    CUDA_TRY(cudaMemcpyAsync(&bits, lat->absmax, sizeof bits, cudaMemcpyDeviceToHost, lat->stream));
    CUDA_TRY(cudaStreamSynchronize(lat->stream));
    float m;
    memcpy(&m, &bits, sizeof m);
    if (!(m > 0.f) || !(m < INFINITY))
        return STAG_OK;
    int k = 0;
    std::frexp(m, &k);
    k -= 1;  // m in [2^k, 2^(k+1))
    if (k >= -kRhsWindow && k <= kRhsWindow)
        return STAG_OK;
    stag_field f = nullptr;
    STAG_TRY(stag_field_create(lat, STAG_EVEN, b->prec, &f));
    cudaError_t e = cudaMemcpyAsync(f->data, b->data, b->bytes, cudaMemcpyDeviceToDevice, lat->stream);
    if (e == cudaSuccess)
        e = launch_field_ldexp(b->prec, lat->geom, f->data, -k, lat->stream);
    if (e != cudaSuccess) {
        stag_field_destroy(f);
        return fail(STAG_ERR_CUDA, "source normalisation: %s", cudaGetErrorString(e));
    }
    rs->k = k;
    rs->scaled = f;
    return STAG_OK;
}

int rhs_scale_end(RhsScale *rs, stag_field const *xs, int n) {
    if (!rs->scaled)
        return STAG_OK;
    stag_lattice lat = rs->scaled->lat;
    DEVICE_SCOPE(lat->device);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; i++)
        e = launch_field_ldexp(xs[i]->prec, xs[i]->lat->geom, xs[i]->data, rs->k, xs[i]->lat->stream);
    for (int i = 0; i < n && e == cudaSuccess; i++)
        e = cudaStreamSynchronize(xs[i]->lat->stream);
    stag_field_destroy(rs->scaled);
    rs->scaled = nullptr;
    if (e != cudaSuccess)
        return fail(STAG_ERR_CUDA, "source normalisation: %s", cudaGetErrorString(e));
    return STAG_OK;
}

// trace (may be NULL): (alpha_k, beta_k, |r_{k+1}|^2) of the first trace_len
// iterations; tracing runs those iterations host-driven, one at a time
static int cg_solve_impl(stag_lattice lat, stag_field x, const stag_field b, double mass,
                         double rel_tol, int max_iter, stag_solve_info *info, double *trace,
                         int trace_len) {
    if (info)
        memset(info, 0, sizeof *info);
    if (!lat || !x || !b)
        return fail(STAG_ERR_ARG, "stag_cg_solve: NULL argument");
    if (x->lat != lat || b->lat != lat)
        return fail(STAG_ERR_ARG, "stag_cg_solve: field belongs to another lattice");
    if (x->parity != STAG_EVEN || b->parity != STAG_EVEN)
        return fail(STAG_ERR_STATE, "stag_cg_solve: x and b must be even fields");
    if (x->prec != b->prec)
        return fail(STAG_ERR_STATE, "stag_cg_solve: precision mismatch");
    if (x == b)
        return fail(STAG_ERR_ARG, "stag_cg_solve: x and b must differ");
    if (x->prec != STAG_F64 && x->prec != STAG_DF64)
        return fail(STAG_ERR_STATE, "stag_cg_solve: fields must be F64 or DF64 (got %s)",
                    prec_name(x->prec));
    if (!(mass > 0) || !std::isfinite(mass))
        return fail(STAG_ERR_ARG, "stag_cg_solve: mass must be positive and finite");
    if (!(rel_tol >= 0) || !std::isfinite(rel_tol))
        return fail(STAG_ERR_ARG, "stag_cg_solve: rel_tol must be >= 0");
    if (max_iter < 0)
        return fail(STAG_ERR_ARG, "stag_cg_solve: max_iter must be >= 0");
    const int prec = x->prec;
    if (!lat->has_gauge || !lat->links[prec])
        return fail(STAG_ERR_STATE, "stag_cg_solve: no %s gauge copy uploaded", prec_name(prec));
    DEVICE_SCOPE(lat->device);
    STAG_TRY(ensure_cg_work(lat, prec));
    CgWork &w = lat->cg[prec];
    cudaStream_t s = lat->stream;
    CUDA_TRY(cudaMemcpyAsync(w.bw, b->data, b->bytes, cudaMemcpyDeviceToDevice, s));
    if (lat->cg_launch == STAG_CG_LAUNCH_GRAPH && !trace) {
        if (!w.exec)
            STAG_TRY(build_cg_graph(lat, w));
        STAG_TRY(upload_scalars(lat, mass, rel_tol, max_iter, true, w.cond));
        CUDA_TRY(cudaEventRecord(lat->ev0, s));
        CUDA_TRY(cudaGraphLaunch(w.exec, s));
        CUDA_TRY(cudaEventRecord(lat->ev1, s));
    } else {
        // the same kernels launched one by one; the host reads the status
        // every cg_chunk iterations, and kernels of iterations past the end
        // return at once
        STAG_TRY(upload_scalars(lat, mass, rel_tol, max_iter, false, 0));
        CUDA_TRY(cudaEventRecord(lat->ev0, s));
        CUDA_TRY(launch_cg_init(prec, lat->geom, w.xw, w.r, w.p, w.bw, lat->partial, lat->sc, s));
        for (int k = 0; trace && k < trace_len && k < max_iter; k++) {
            CUDA_TRY(cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            if (lat->sc_host->status != CG_RUNNING)
                break;
            CUDA_TRY(enqueue_cg_body(lat, w, s, true));
            CUDA_TRY(cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            trace[3 * k + 0] = lat->sc_host->alpha.d;
            trace[3 * k + 1] = lat->sc_host->beta.d;
            trace[3 * k + 2] = lat->sc_host->rr;
        }
        const int chunk = lat->cg_chunk;
        const long long max_chunks = (long long)max_iter / chunk + 2;
        for (long long k = 0; k < max_chunks; k++) {
            CUDA_TRY(cudaMemcpyAsync(&lat->sc_host->status, &lat->sc->status, sizeof(int),
                                     cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            if (lat->sc_host->status != CG_RUNNING)
                break;
            for (int j = 0; j < chunk; j++)
                CUDA_TRY(enqueue_cg_body(lat, w, s, true));
        }
        CUDA_TRY(enqueue_true_residual(lat, w, s));
        CUDA_TRY(cudaEventRecord(lat->ev1, s));
    }
    CUDA_TRY(cudaMemcpyAsync(x->data, w.xw, x->bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, lat->ev0, lat->ev1));
    stag_solve_info local;
    fill_info(lat, prec, *lat->sc_host, ms, &local);
    if (info)
        *info = local;
    if (local.status != STAG_OK)
        return fail(local.status, "stag_cg_solve: %s after %d iterations (|r|/|b| = %.3e)",
                    local.status == STAG_ERR_BREAKDOWN ? "breakdown" : "not converged", local.iters,
                    local.iter_rel_resid);
    return STAG_OK;
}

// cg_solve_impl on b, or on b 2^-k with the solution scaled back
static int cg_solve_scaled(stag_lattice lat, stag_field x, const stag_field b, double mass, double rel_tol,
                           int max_iter, stag_solve_info *info, double *trace, int trace_len) {
    if (!lat || !x || !b || x == b || x->prec != b->prec || b->lat != lat || b->parity != STAG_EVEN)
        return cg_solve_impl(lat, x, b, mass, rel_tol, max_iter, info, trace, trace_len);  // reports the error
    RhsScale rs;
    STAG_TRY(rhs_scale_begin(b, &rs));
    stag_solve_info local;
    const int st = cg_solve_impl(lat, x, rs.scaled ? rs.scaled : b, mass, rel_tol, max_iter, &local, trace,
                                 trace_len);
    if (info)
        *info = local;
    // |r_{k+1}|^2 of the entries written, back in the units of b
    if (trace && rs.k)
        for (int k = 0; k < trace_len && k < local.iters; k++)
            trace[3 * k + 2] = std::ldexp(trace[3 * k + 2], 2 * rs.k);
    STAG_TRY(rhs_scale_end(&rs, &x, 1));
    return st;
}

extern "C" int stag_cg_solve(stag_lattice lat, stag_field x, const stag_field b, double mass,
                             double rel_tol, int max_iter, stag_solve_info *info) {
    STAG_NVTX("stag_cg_solve");
    return cg_solve_scaled(lat, x, b, mass, rel_tol, max_iter, info, nullptr, 0);
}

extern "C" int stag_cg_solve_traced(stag_lattice lat, stag_field x, const stag_field b, double mass,
                                    double rel_tol, int max_iter, double *trace, int trace_len,
                                    stag_solve_info *info) {
    STAG_NVTX("stag_cg_solve_traced");
    if (info)
        memset(info, 0, sizeof *info);
    if (!trace || trace_len < 0)
        return fail(STAG_ERR_ARG, "stag_cg_solve_traced: need a trace buffer and trace_len >= 0");
    return cg_solve_scaled(lat, x, b, mass, rel_tol, max_iter, info, trace, trace_len);
}


// --------------------------------------------------------------------------
extern "C" int stag_cb_neighbor(const int dims[4], int parity, long long cb, int mu, int steps,
                                long long *out_cb, int *out_wraps) {
    if (!dims || !out_cb || !out_wraps)
        return fail(STAG_ERR_ARG, "stag_cb_neighbor: NULL argument");
    long long V = 1;
    for (int k = 0; k < 4; k++) {
        if (dims[k] < 2 || dims[k] % 2 != 0 || dims[k] > 4096)
            return fail(STAG_ERR_ARG, "stag_cb_neighbor: dims[%d] = %d must be even, 2..4096", k, dims[k]);
        V *= dims[k];
    }
    if (V / 2 > (1LL << 30))
        return fail(STAG_ERR_ARG, "stag_cb_neighbor: volume too large");
    if ((parity != 0 && parity != 1) || cb < 0 || cb >= V / 2 || mu < 0 || mu > 3 ||
        (steps != 1 && steps != -1 && steps != 3 && steps != -3))
        return fail(STAG_ERR_ARG, "stag_cb_neighbor: parity 0/1, 0 <= cb < V/2, mu 0..3, steps +-1 or +-3");
    const Geom g = geom_of(dims, V / 2);
    int x[4];
    cb_coords(g, (int)cb, parity, x);
    *out_cb = cb_hop(g, (int)cb, x, mu, steps);
    *out_wraps = hop_wraps(x[mu], steps, g.L[mu]);
    return STAG_OK;
}

// --------------------------------------------------------------------------
extern "C" const char *stag_strerror(int status) {
    switch (status) {
    case STAG_OK: return "ok";
    case STAG_ERR_ARG: return "invalid argument";
    case STAG_ERR_STATE: return "invalid state";
    case STAG_ERR_CUDA: return "CUDA error";
    case STAG_ERR_NOT_CONVERGED: return "not converged";
    case STAG_ERR_BREAKDOWN: return "solver breakdown";
    case STAG_ERR_TIMEOUT: return "device wait timed out";
    case STAG_ERR_NOMEM: return "out of memory";
    default: return "unknown status";
    }
}

extern "C" const char *stag_last_error_message(void) { return g_last_error.c_str(); }

extern "C" const char *stag_version(void) { return "0.1.0"; }

