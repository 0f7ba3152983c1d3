// stag_apply_M_noalloc: M x = m^2 x - D_eo D_oe x for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted, e.g. a host callback or library hook that is invoked while the
// caller is capturing work into a CUDA graph, a memory-budgeted service that
// hands out fixed device buffers up front, or a caller whose allocator owns
// all device memory.  Creating a lattice allocates (link copies, work
// vectors), so these callers cannot use stag_apply_M.  This entry point works
// on the caller's own device buffers in the canonical layouts and keeps its
// one intermediate (D_oe x on the odd sites) in a fixed array compiled into
// the library.
//
// The arithmetic is plain FP64 with the Kogut-Susskind phases, boundary
// signs and Naik coefficients applied at every hop (nothing pre-folded),
// one thread per output site.  It is not the tuned path: stag_apply_M on an
// uploaded lattice is several times faster.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/stag.h"
#include "common.cuh"
#include "kernels.h"

namespace {

using stag::Geom;

// Maximum sites per parity; the scratch array holds one colour vector per
// odd site: 65536 * 3 complex doubles = 3 MiB, resident on every GPU that
// loads the library until the process exits.
constexpr long long kNoAllocMaxVh = 65536;

static __device__ __align__(256) double2 g_noalloc_scratch[3 * kNoAllocMaxVh];

struct NoAllocArgs {
    Geom g;
    double bc[4];
    double c1, c3;
    const double2 *fat;  // canonical [4][V][3][3]
    const double2 *lng;
    const double2 *in;   // canonical [Vh][3], parity 1 - out_par
    double2 *out;        // canonical [Vh][3], parity out_par
    const double2 *p;    // even input for the m^2 p term (second pass only)
    double m2;
};

__device__ int full_index(const Geom &g, const int x[4]) {
    return x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]));
}

// coordinate after s steps along one direction and the number of wraps
__device__ int step_coord(int v, int s, int L, int *wraps) {
    int y = v + s, w = 0;
    while (y >= L) {
        y -= L;
        w++;
    }
    while (y < 0) {
        y += L;
        w--;
    }
    *wraps = w;
    return y;
}

// out(x) = (D in)(x) for one output site, links read in canonical order
template <bool M_EPI>
__global__ void noalloc_dslash_kernel(NoAllocArgs a, int out_par) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.g.Vh)
        return;
    const long long V = 2LL * a.g.Vh;
    int x[4];
    stag::cb_coords(a.g, c, out_par, x);
    const int i = full_index(a.g, x);
    double2 acc[3];
    for (int k = 0; k < 3; k++)
        acc[k] = make_double2(0.0, 0.0);
    for (int mu = 0; mu < 4; mu++) {
        int es = 0;
        for (int nu = 0; nu < mu; nu++)
            es += x[nu];
        const double eta = (es & 1) ? -1.0 : 1.0;
        for (int h = 0; h < 2; h++) {
            const int s = h ? 3 : 1;
            const double coef = eta * (h ? a.c3 : a.c1);
            const double2 *G = h ? a.lng : a.fat;
            for (int dir = 0; dir < 2; dir++) {
                const int ss = dir ? -s : s;
                int w;
                int y[4] = {x[0], x[1], x[2], x[3]};
                y[mu] = step_coord(x[mu], ss, a.g.L[mu], &w);
                const double sign = (w & 1) && a.bc[mu] < 0 ? -1.0 : 1.0;
                const int j = full_index(a.g, y);
                const double2 *v = a.in + (size_t)(j >> 1) * 3;
                // forward: + U(x) in(x+s mu); backward: - U(x-s mu)^+ in(x-s mu)
                const double2 *U = G + ((size_t)mu * V + (dir ? j : i)) * 9;
                const double f = dir ? -coef * sign : coef * sign;
                for (int r = 0; r < 3; r++) {
                    double re = 0.0, im = 0.0;
                    for (int k = 0; k < 3; k++) {
                        const double2 u = dir ? make_double2(U[3 * k + r].x, -U[3 * k + r].y)
                                              : U[3 * r + k];
                        const double2 b = v[k];
                        re += u.x * b.x - u.y * b.y;
                        im += u.x * b.y + u.y * b.x;
                    }
                    acc[r].x += f * re;
                    acc[r].y += f * im;
                }
            }
        }
    }
    for (int r = 0; r < 3; r++) {
        double2 o = acc[r];
        if (M_EPI) {
            const double2 pv = a.p[(size_t)c * 3 + r];
            o = make_double2(a.m2 * pv.x - o.x, a.m2 * pv.y - o.y);
        }
        a.out[(size_t)c * 3 + r] = o;
    }
}

std::mutex g_scratch_mutex;
double2 *g_scratch_addr[64] = {nullptr};

// device memory of device `dev` (managed memory is reachable from any
// device; plain device memory of another GPU is not without peer access)
bool is_device_pointer_of(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged)
        return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int stag_apply_M_noalloc(const int dims[4], const double bc[4], double c1, double c3,
                                    const double *fat, const double *lng, double mass,
                                    const double *in_even, double *out_even, void *cuda_stream) {
    if (!dims || !fat || !lng || !in_even || !out_even)
        return stag::set_error(STAG_ERR_ARG, "stag_apply_M_noalloc: NULL argument");
    long long V = 1;
    for (int k = 0; k < 4; k++) {
        if (dims[k] < 2 || dims[k] % 2)
            return stag::set_error(STAG_ERR_ARG,
                                   "stag_apply_M_noalloc: dims must be even and >= 2");
        V *= dims[k];
        if (V > (1LL << 40))
            break;
    }
    if (V / 2 > kNoAllocMaxVh)
        return stag::set_error(STAG_ERR_ARG,
                               "stag_apply_M_noalloc: Vh = V/2 exceeds the fixed scratch size "
                               "of 65536 sites per parity");
    double bcv[4] = {1.0, 1.0, 1.0, -1.0};
    if (bc)
        for (int k = 0; k < 4; k++) {
            if (bc[k] != 1.0 && bc[k] != -1.0)
                return stag::set_error(STAG_ERR_ARG, "stag_apply_M_noalloc: bc must be +1 or -1");
            bcv[k] = bc[k];
        }
    if (!std::isfinite(c1) || !std::isfinite(c3) || !std::isfinite(mass))
        return stag::set_error(STAG_ERR_ARG, "stag_apply_M_noalloc: c1, c3, mass must be finite");
    if (in_even == out_even)
        return stag::set_error(STAG_ERR_ARG, "stag_apply_M_noalloc: in and out must differ");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return stag::set_error(STAG_ERR_CUDA, "stag_apply_M_noalloc: no current CUDA device");
    const void *ptrs[4] = {fat, lng, in_even, out_even};
    for (const void *p : ptrs)
        if (!is_device_pointer_of(p, dev))
            return stag::set_error(STAG_ERR_ARG,
                                   "stag_apply_M_noalloc: every buffer must be device memory of the "
                                   "current device (%d)", dev);

    // set-up, once per device, with that device current: the device address
    // of the scratch array (its host-side name is only a stand-in)
    double2 *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return stag::set_error(STAG_ERR_CUDA, "stag_apply_M_noalloc: cudaGetSymbolAddress: %s",
                                       cudaGetErrorString(e));
            g_scratch_addr[dev] = (double2 *)p;
        }
        scratch = g_scratch_addr[dev];
    }

    NoAllocArgs a;
    for (int k = 0; k < 4; k++) {
        a.g.L[k] = dims[k];
        a.bc[k] = bcv[k];
    }
    a.g.Lxh = dims[0] / 2;
    a.g.Vh = (int)(V / 2);
    a.g.stride = a.g.Vh;
    a.g.plane[0] = 0;
    a.g.plane[1] = dims[0] / 2;
    a.g.plane[2] = dims[0] * dims[1] / 2;
    a.g.plane[3] = dims[0] * dims[1] * dims[2] / 2;
    geom_set_div(a.g);
    a.c1 = c1;
    a.c3 = c3;
    a.fat = (const double2 *)fat;
    a.lng = (const double2 *)lng;
    a.m2 = mass * mass;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int block = 128, grid = (a.g.Vh + block - 1) / block;
    // pass 1: scratch = D_oe in (odd sites)
    a.in = (const double2 *)in_even;
    a.out = scratch;
    a.p = nullptr;
    noalloc_dslash_kernel<false><<<grid, block, 0, s>>>(a, STAG_ODD);
    // pass 2: out = m^2 in - D_eo scratch (even sites)
    a.in = scratch;
    a.out = (double2 *)out_even;
    a.p = (const double2 *)in_even;
    noalloc_dslash_kernel<true><<<grid, block, 0, s>>>(a, STAG_EVEN);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return stag::set_error(STAG_ERR_CUDA, "stag_apply_M_noalloc: launch: %s", cudaGetErrorString(e));
    return STAG_OK;
}
