// NCCL as the communicator of the rank decomposition (stag_comm_nccl_*;
// documentation in include/stag.h).  The exchange is one NCCL group of two
// sends and two receives on the stream it is given, ordered so that each pair of
// ranks matches them the same way for any number of ranks (including one,
// where a rank sends to itself, and two, where both neighbours are the same
// rank): every rank sends towards rank + 1 first and receives from rank - 1
// first.  The host allreduce sums the doubles through a device buffer on the
// communicator's own stream; the device allreduce sums in place on the
// caller's stream.  Compiled against nccl.h when the build finds
// it; otherwise the entry points report that NCCL is missing.
#include "api_internal.h"

#ifdef STAG_HAVE_NCCL
#include <nccl.h>

namespace {

struct NcclCtx {
    ncclComm_t comm = nullptr;
    int rank = 0, size = 1, device = 0;
    cudaStream_t stream = nullptr;
    double *dbuf = nullptr;
    static constexpr int kMaxReduce = 64;
};

int nccl_exchange(void *ctx, const void *to_prev, const void *to_next, void *from_prev, void *from_next,
                  unsigned long long bytes, void *stream) {
    NcclCtx *c = (NcclCtx *)ctx;
    const int prev = (c->rank - 1 + c->size) % c->size, next = (c->rank + 1) % c->size;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    if (ncclGroupStart() != ncclSuccess)
        return 1;
    ncclResult_t r = ncclSend(to_next, bytes, ncclChar, next, c->comm, s);
    if (r == ncclSuccess)
        r = ncclSend(to_prev, bytes, ncclChar, prev, c->comm, s);
    if (r == ncclSuccess)
        r = ncclRecv(from_prev, bytes, ncclChar, prev, c->comm, s);
    if (r == ncclSuccess)
        r = ncclRecv(from_next, bytes, ncclChar, next, c->comm, s);
    const ncclResult_t r2 = ncclGroupEnd();
    return (r == ncclSuccess && r2 == ncclSuccess) ? 0 : 2;
}

int nccl_allreduce(void *ctx, double *vals, int n) {
    NcclCtx *c = (NcclCtx *)ctx;
    if (n < 0 || n > NcclCtx::kMaxReduce)
        return 1;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != c->device && cudaSetDevice(c->device) != cudaSuccess)
        return 2;
    int rc = 0;
    if (cudaMemcpyAsync(c->dbuf, vals, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        ncclAllReduce(c->dbuf, c->dbuf, n, ncclDouble, ncclSum, c->comm, c->stream) != ncclSuccess ||
        cudaMemcpyAsync(vals, c->dbuf, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        rc = 3;
    if (prev_dev >= 0 && prev_dev != c->device)
        cudaSetDevice(prev_dev);
    return rc;
}

int nccl_allreduce_dev(void *ctx, double *dev_vals, int n, void *stream) {
    NcclCtx *c = (NcclCtx *)ctx;
    if (n < 0)
        return 1;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    return ncclAllReduce(dev_vals, dev_vals, n, ncclDouble, ncclSum, c->comm, s) == ncclSuccess ? 0 : 2;
}

}  // namespace

extern "C" int stag_comm_nccl_id(unsigned char id[128]) {
    if (!id)
        return fail(STAG_ERR_ARG, "stag_comm_nccl_id: NULL argument");
    static_assert(sizeof(ncclUniqueId) == 128, "NCCL unique id size");
    ncclUniqueId u;
    const ncclResult_t r = ncclGetUniqueId(&u);
    if (r != ncclSuccess)
        return fail(STAG_ERR_STATE, "stag_comm_nccl_id: %s", ncclGetErrorString(r));
    memcpy(id, &u, 128);
    return STAG_OK;
}

extern "C" int stag_comm_nccl_create(int rank, int size, const unsigned char id[128], int device, stag_comm *out) {
    if (!id || !out)
        return fail(STAG_ERR_ARG, "stag_comm_nccl_create: NULL argument");
    memset(out, 0, sizeof *out);
    if (size < 1 || rank < 0 || rank >= size || device < 0)
        return fail(STAG_ERR_ARG, "stag_comm_nccl_create: rank %d of %d on device %d", rank, size, device);
    DEVICE_SCOPE(device);
    NcclCtx *c = new (std::nothrow) NcclCtx();
    if (!c)
        return fail(STAG_ERR_NOMEM, "stag_comm_nccl_create: host allocation failed");
    c->rank = rank;
    c->size = size;
    c->device = device;
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMalloc(&c->dbuf, sizeof(double) * NcclCtx::kMaxReduce);
    if (e != cudaSuccess) {
        if (c->stream)
            cudaStreamDestroy(c->stream);
        delete c;
        return fail(STAG_ERR_CUDA, "stag_comm_nccl_create: %s", cudaGetErrorString(e));
    }
    ncclUniqueId u;
    memcpy(&u, id, 128);
    const ncclResult_t r = ncclCommInitRank(&c->comm, size, u, rank);
    if (r != ncclSuccess) {
        cudaFree(c->dbuf);
        cudaStreamDestroy(c->stream);
        delete c;
        return fail(STAG_ERR_STATE, "stag_comm_nccl_create: %s", ncclGetErrorString(r));
    }
    out->ctx = c;
    out->rank = rank;
    out->size = size;
    out->device_buffers = 1;
    out->exchange = nccl_exchange;
    out->allreduce = nccl_allreduce;
    out->allreduce_dev = nccl_allreduce_dev;
    return STAG_OK;
}

extern "C" int stag_comm_nccl_destroy(stag_comm *out) {
    if (!out || !out->ctx)
        return STAG_OK;
    if (out->exchange != nccl_exchange)
        return fail(STAG_ERR_ARG, "stag_comm_nccl_destroy: not an NCCL communicator");
    NcclCtx *c = (NcclCtx *)out->ctx;
    {
        DEVICE_SCOPE(c->device);
        cudaStreamSynchronize(c->stream);
        ncclCommDestroy(c->comm);
        cudaFree(c->dbuf);
        cudaStreamDestroy(c->stream);
    }
    delete c;
    memset(out, 0, sizeof *out);
    return STAG_OK;
}

#else  // built without NCCL

extern "C" int stag_comm_nccl_id(unsigned char id[128]) {
    (void)id;
    return fail(STAG_ERR_STATE, "stag_comm_nccl_id: libstag was built without NCCL (nccl.h not found)");
}

extern "C" int stag_comm_nccl_create(int rank, int size, const unsigned char id[128], int device, stag_comm *out) {
    (void)rank;
    (void)size;
    (void)id;
    (void)device;
    if (out)
        memset(out, 0, sizeof *out);
    return fail(STAG_ERR_STATE, "stag_comm_nccl_create: libstag was built without NCCL (nccl.h not found)");
}

extern "C" int stag_comm_nccl_destroy(stag_comm *out) {
    if (out && out->ctx)
        return fail(STAG_ERR_STATE, "stag_comm_nccl_destroy: libstag was built without NCCL");
    return STAG_OK;
}

#endif
