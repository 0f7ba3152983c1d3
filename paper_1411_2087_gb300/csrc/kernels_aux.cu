// CG vector kernels, field import/export, link folding and the three-link
// products.
#include "dslash.cuh"
#include "kernels.h"

#include <cfloat>

namespace stag {

// --------------------------------------------------------------------------
// CG vector kernels.  Each reads the device scalars written by the previous
// kernel; the last block of a reducing kernel updates them and, inside the
// solve graph, sets the loop condition.
// --------------------------------------------------------------------------

STAG_D void set_loop_condition(CgScalars *sc) {
    if (sc->has_cond)
        cudaGraphSetConditional(sc->cond, sc->status == CG_RUNNING ? 1u : 0u);
}

// x = 0, r = b, p = b, |b|^2
template <int P, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
cg_init_kernel(Geom g, typename Fmt<P>::Elem *x, typename Fmt<P>::Elem *r,
               typename Fmt<P>::Elem *p, const typename Fmt<P>::Elem *b, double *partial,
               CgScalars *sc) {
    using F = Fmt<P>;
    using R = typename F::R;
    __shared__ double smem[32];
    const int c = blockIdx.x * BLOCK + threadIdx.x;
    red_t<R> dot = red_zero<red_t<R>>();
    if (c < g.Vh) {
        cplx<R> bv[3], z[3];
        load_vec<P>(b, g.stride, c, bv);
#pragma unroll
        for (int k = 0; k < 3; k++)
            z[k] = czero<R>();
        store_vec<P>(x, g.stride, c, z);
        store_vec<P>(r, g.stride, c, bv);
        store_vec<P>(p, g.stride, c, bv);
        dot = re_dot3<R>(bv, bv);
    }
    double total;
    if (grid_sum<BLOCK>(dot, partial, &sc->ticket, smem, total) && threadIdx.x == 0) {
        sc->bb = total;
        sc->rr = total;
        sc->rr_stop = sc->tol2 * total;
        sc->iter = 0;
        sc->alpha = make_dpair(0.0);
        sc->beta = make_dpair(0.0);
        if (!(total < INFINITY))
            sc->status = CG_BREAKDOWN;
        else if (total <= sc->rr_stop)
            sc->status = CG_CONVERGED;
        else if (sc->max_iter <= 0)
            sc->status = CG_MAXITER;
        else
            sc->status = CG_RUNNING;
        set_loop_condition(sc);
    }
}

// x += alpha p, r -= alpha Ap, |r|^2 -> beta, convergence
template <int P, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
cg_update_kernel(Geom g, typename Fmt<P>::Elem *x, typename Fmt<P>::Elem *r,
                 const typename Fmt<P>::Elem *p, const typename Fmt<P>::Elem *Ap,
                 double *partial, CgScalars *sc) {
    using F = Fmt<P>;
    using R = typename F::R;
    __shared__ double smem[32];
    const int c = blockIdx.x * BLOCK + threadIdx.x;
    const bool run = sc->status == CG_RUNNING;
    red_t<R> dot = red_zero<red_t<R>>();
    if (run && c < g.Vh) {
        const R alpha = scalar_as<R>(sc->alpha);
        const R malpha = -alpha;
        cplx<R> xv[3], rv[3], pv[3], av[3];
        load_vec<P>(x, g.stride, c, xv);
        load_vec<P>(r, g.stride, c, rv);
        load_vec<P>(p, g.stride, c, pv);
        load_vec<P>(Ap, g.stride, c, av);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            mac(xv[k].re, alpha, pv[k].re);
            mac(xv[k].im, alpha, pv[k].im);
            mac(rv[k].re, malpha, av[k].re);
            mac(rv[k].im, malpha, av[k].im);
            xv[k].re = rnorm<R>(xv[k].re);
            xv[k].im = rnorm<R>(xv[k].im);
            rv[k].re = rnorm<R>(rv[k].re);
            rv[k].im = rnorm<R>(rv[k].im);
        }
        store_vec<P>(x, g.stride, c, xv);
        store_vec<P>(r, g.stride, c, rv);
        dot = re_dot3<R>(rv, rv);
    }
    double total;
    if (grid_sum<BLOCK>(dot, partial, &sc->ticket, smem, total) && threadIdx.x == 0) {
        if (sc->status == CG_RUNNING) {
            const double beta = total / sc->rr;
            sc->beta = make_dpair(beta);
            sc->rr = total;
            sc->iter += 1;
            if (!(total < INFINITY))
                sc->status = CG_BREAKDOWN;
            else if (total <= sc->rr_stop)
                sc->status = CG_CONVERGED;
            else if (sc->iter >= sc->max_iter)
                sc->status = CG_MAXITER;
        } else {
            sc->beta = make_dpair(0.0);
        }
        set_loop_condition(sc);
    }
}

// p = r + beta p
template <int P, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
cg_p_kernel(Geom g, const typename Fmt<P>::Elem *r, typename Fmt<P>::Elem *p, const CgScalars *sc) {
    using F = Fmt<P>;
    using R = typename F::R;
    const int c = blockIdx.x * BLOCK + threadIdx.x;
    // after convergence or breakdown p is no longer used
    if (c >= g.Vh || sc->status != CG_RUNNING)
        return;
    const R beta = scalar_as<R>(sc->beta);
    cplx<R> rv[3], pv[3];
    load_vec<P>(r, g.stride, c, rv);
    load_vec<P>(p, g.stride, c, pv);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        mac(rv[k].re, beta, pv[k].re);
        mac(rv[k].im, beta, pv[k].im);
        rv[k].re = rnorm<R>(rv[k].re);
        rv[k].im = rnorm<R>(rv[k].im);
    }
    store_vec<P>(p, g.stride, c, rv);
}

// one block: sum of the block partials of an EPI_M_PART Dslash, then alpha
constexpr int FINISH_BLOCK = 1024;

__global__ void __launch_bounds__(FINISH_BLOCK)
pap_finish_kernel(const double *__restrict__ partial, int n, CgScalars *sc, int skip_if_done, const int *gate) {
    __shared__ double smem[32];
    if (skip_if_done && sc->status != CG_RUNNING)
        return;
    if (gate && *gate == 0)
        return;
    // four independent sums per thread over a fixed assignment, then the block tree
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * FINISH_BLOCK < n; i += 4 * FINISH_BLOCK) {
        a0 += partial[i];
        a1 += partial[i + FINISH_BLOCK];
        a2 += partial[i + 2 * FINISH_BLOCK];
        a3 += partial[i + 3 * FINISH_BLOCK];
    }
    for (; i < n; i += FINISH_BLOCK)
        a0 += partial[i];
    const double total = block_sum<FINISH_BLOCK>((a0 + a1) + (a2 + a3), smem);
    if (threadIdx.x == 0) {
        sc->pAp = total;
        if (sc->status == CG_RUNNING && !(total > 0.0 && total < INFINITY))
            sc->status = CG_BREAKDOWN;
        sc->alpha = make_dpair(sc->status == CG_RUNNING ? sc->rr / total : 0.0);
    }
}

cudaError_t launch_pap_finish(const double *partial, int n, CgScalars *sc, bool skip_if_done, cudaStream_t s,
                              const int *gate) {
    pap_finish_kernel<<<1, FINISH_BLOCK, 0, s>>>(partial, n, sc, skip_if_done ? 1 : 0, gate);
    return cudaGetLastError();
}

static int cg_grid(const Geom &g) { return (g.Vh + CG_BLOCK - 1) / CG_BLOCK; }

#define STAG_PREC_SWITCH(prec, ...)                                   \
    switch (prec) {                                                   \
    case P_F64: { constexpr int P = P_F64; __VA_ARGS__; } break;      \
    case P_DF64: { constexpr int P = P_DF64; __VA_ARGS__; } break;    \
    case P_F32: { constexpr int P = P_F32; __VA_ARGS__; } break;      \
    case P_F16: { constexpr int P = P_F16; __VA_ARGS__; } break;      \
    default: return cudaErrorInvalidValue;                            \
    }

cudaError_t launch_cg_init(int prec, const Geom &g, void *x, void *r, void *p, const void *b,
                           double *partial, CgScalars *sc, cudaStream_t s) {
    STAG_PREC_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        cg_init_kernel<P, CG_BLOCK><<<cg_grid(g), CG_BLOCK, 0, s>>>(g, (E *)x, (E *)r, (E *)p,
                                                                    (const E *)b, partial, sc);
    });
    return cudaGetLastError();
}

cudaError_t launch_cg_update(int prec, const Geom &g, void *x, void *r, const void *p,
                             const void *Ap, double *partial, CgScalars *sc, cudaStream_t s) {
    STAG_PREC_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        cg_update_kernel<P, CG_BLOCK><<<cg_grid(g), CG_BLOCK, 0, s>>>(
            g, (E *)x, (E *)r, (const E *)p, (const E *)Ap, partial, sc);
    });
    return cudaGetLastError();
}

cudaError_t launch_cg_p_update(int prec, const Geom &g, const void *r, void *p,
                               const CgScalars *sc, cudaStream_t s) {
    STAG_PREC_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        cg_p_kernel<P, CG_BLOCK><<<cg_grid(g), CG_BLOCK, 0, s>>>(g, (const E *)r, (E *)p, sc);
    });
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// import / export between canonical complex128 [Vh][3] and the SoA layout
// --------------------------------------------------------------------------
template <int P>
__global__ void import_kernel(Geom g, const double *__restrict__ canon, typename Fmt<P>::Elem *f) {
    using R = typename Fmt<P>::R;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.Vh)
        return;
    cplx<R> w[3];
#pragma unroll
    for (int a = 0; a < 3; a++)
        w[a] = Fmt<P>::make(canon[(3 * (size_t)c + a) * 2], canon[(3 * (size_t)c + a) * 2 + 1]);
    store_vec<P>(f, g.stride, c, w);
}

template <int P>
__global__ void export_kernel(Geom g, const typename Fmt<P>::Elem *f, double *__restrict__ canon) {
    using R = typename Fmt<P>::R;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.Vh)
        return;
    cplx<R> w[3];
    load_vec<P>(f, g.stride, c, w);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        canon[(3 * (size_t)c + a) * 2] = to_double<R>(w[a].re);
        canon[(3 * (size_t)c + a) * 2 + 1] = to_double<R>(w[a].im);
    }
}

cudaError_t launch_import(int prec, const Geom &g, const double *canon, void *field, cudaStream_t s) {
    const int grid = (g.Vh + 255) / 256;
    STAG_PREC_SWITCH(prec, {
        import_kernel<P><<<grid, 256, 0, s>>>(g, canon, (typename Fmt<P>::Elem *)field);
    });
    return cudaGetLastError();
}

cudaError_t launch_export(int prec, const Geom &g, const void *field, double *canon, cudaStream_t s) {
    const int grid = (g.Vh + 255) / 256;
    STAG_PREC_SWITCH(prec, {
        export_kernel<P><<<grid, 256, 0, s>>>(g, (const typename Fmt<P>::Elem *)field, canon);
    });
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// link folding: entry j of kind `kind` = mu (+4 long) at (par, cb) = coef * L[mu][i][j]
// (the kinds' layouts as link_kind_offset describes)
//   coef = c * eta_mu(x) * bc_mu^w,  w = floor((x_mu + s) / L_mu), s = 1 or 3
// so that the stencil applies  + G(x) psi(x+s mu)  and  - G(x-s mu)^+ psi(x-s mu).
// --------------------------------------------------------------------------
struct FoldArgs {
    Geom g;
    double bc[4];
    double c1, c3;
    float inv_scale[2];  // 16-bit links: 32767 / field max (one-link, three-link)
};

STAG_D void full_coords(const Geom &g, long long i, int x[4]) {
    x[0] = (int)(i % g.L[0]);
    i /= g.L[0];
    x[1] = (int)(i % g.L[1]);
    i /= g.L[1];
    x[2] = (int)(i % g.L[2]);
    x[3] = (int)(i / g.L[2]);
}

// entry e of the full link at checkerboard site cb of one kind (kind base kb)
template <int P>
STAG_D void store_full_link(char *kb, size_t S, size_t cb, int e, double re, double im, float inv_scale) {
    if constexpr (P == P_F16)
        *L16::slot(kb, S, cb, e) = Fmt<P>::pack_link(re, im, inv_scale);
    else
        ((typename Fmt<P>::Elem *)kb)[(size_t)e * S + cb] = Fmt<P>::pack_link(re, im, inv_scale);
}

template <int P>
__global__ void fold_kernel(FoldArgs fa, const double *__restrict__ fat, const double *__restrict__ lng,
                            char *G) {
    const Geom &g = fa.g;
    const long long V = 2LL * g.Vh;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 8 * V)
        return;
    const int kind = (int)(t / V);
    const long long i = t % V;
    const int mu = kind & 3;
    const bool three = kind >= 4;
    int x[4];
    full_coords(g, i, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int cb = (int)(i >> 1);
    int eta_sum = 0;
    for (int nu = 0; nu < mu; nu++)
        eta_sum += x[nu];
    const int s = three ? 3 : 1;
    const int wraps = (x[mu] + s) / g.L[mu];
    double coef = three ? fa.c3 : fa.c1;
    if (eta_sum & 1)
        coef = -coef;
    if ((wraps & 1) && fa.bc[mu] < 0)
        coef = -coef;
    const double *src = (three ? lng : fat) + ((size_t)mu * V + i) * 18;
    const size_t S = (size_t)g.stride;
    char *kb = G + (size_t)par * link_parity_bytes(P, 0, S) + link_kind_offset(P, 0, kind, S);
    for (int j = 0; j < 9; j++)
        store_full_link<P>(kb, S, cb, j, coef * src[2 * j], coef * src[2 * j + 1], fa.inv_scale[three ? 1 : 0]);
}

// the same folding into a copy whose kinds of the groups in `mask` (bit 0
// one-link, bit 1 three-link) take the 12-real layout (rows 0 and 1 only)
template <int P>
__global__ void fold_c12_kernel(FoldArgs fa, const double *__restrict__ fat, const double *__restrict__ lng,
                                char *G, int mask) {
    const Geom &g = fa.g;
    const long long V = 2LL * g.Vh;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 8 * V)
        return;
    const int kind = (int)(t / V);
    const long long i = t % V;
    const int mu = kind & 3;
    const bool three = kind >= 4;
    int x[4];
    full_coords(g, i, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const size_t cb = (size_t)(i >> 1);
    int eta_sum = 0;
    for (int nu = 0; nu < mu; nu++)
        eta_sum += x[nu];
    const int s = three ? 3 : 1;
    const int wraps = (x[mu] + s) / g.L[mu];
    double coef = three ? fa.c3 : fa.c1;
    if (eta_sum & 1)
        coef = -coef;
    if ((wraps & 1) && fa.bc[mu] < 0)
        coef = -coef;
    const double *src = (three ? lng : fat) + ((size_t)mu * V + i) * 18;
    const size_t S = (size_t)g.stride;
    char *kb = G + (size_t)par * link_parity_bytes(P, mask, S) + link_kind_offset(P, mask, kind, S);
    const float inv = fa.inv_scale[three ? 1 : 0];
    if ((mask >> (three ? 1 : 0)) & 1) {
        for (int e = 0; e < 6; e++)
            C12<P>::store(kb, S, cb, e, coef * src[2 * e], coef * src[2 * e + 1], inv);
    } else {
        for (int e = 0; e < 9; e++)
            store_full_link<P>(kb, S, cb, e, coef * src[2 * e], coef * src[2 * e + 1], inv);
    }
}

cudaError_t launch_fold_links_c12(int prec, const Geom &g, const double bc[4], double c1, double c3,
                                  const double *fat, const double *lng, void *links, const float inv_scale[2],
                                  int mask, cudaStream_t s) {
    FoldArgs fa;
    fa.g = g;
    for (int k = 0; k < 4; k++)
        fa.bc[k] = bc[k];
    fa.c1 = c1;
    fa.c3 = c3;
    fa.inv_scale[0] = inv_scale ? inv_scale[0] : 0.f;
    fa.inv_scale[1] = inv_scale ? inv_scale[1] : 0.f;
    const long long n = 16LL * g.Vh;
    const int grid = (int)((n + 255) / 256);
    if (mask != 2 && mask != 3)
        return cudaErrorInvalidValue;
    if (prec == P_F32)
        fold_c12_kernel<P_F32><<<grid, 256, 0, s>>>(fa, fat, lng, (char *)links, mask);
    else if (prec == P_F16)
        fold_c12_kernel<P_F16><<<grid, 256, 0, s>>>(fa, fat, lng, (char *)links, mask);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// largest deviation of a link field from SU(3): max over links of
// |U U^+ - 1| (entry-wise) and |det U - 1|, as float bits in *out
__global__ void su3_dev_kernel(const double2 *__restrict__ U, long long nlinks, unsigned *out) {
    float m = 0.f;
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < nlinks;
         l += (long long)gridDim.x * blockDim.x) {
        double2 A[9];
        for (int e = 0; e < 9; e++)
            A[e] = U[l * 9 + e];
        double dev = 0.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double re = 0.0, im = 0.0;
                for (int k = 0; k < 3; k++) {  // (U U^+)_ab = sum_k U_ak conj(U_bk)
                    re += A[3 * a + k].x * A[3 * b + k].x + A[3 * a + k].y * A[3 * b + k].y;
                    im += A[3 * a + k].y * A[3 * b + k].x - A[3 * a + k].x * A[3 * b + k].y;
                }
                dev = fmax(dev, fabs(re - (a == b ? 1.0 : 0.0)));
                dev = fmax(dev, fabs(im));
            }
        // det by the first row's cofactors
        double dre = 0.0, dim = 0.0;
        for (int j = 0; j < 3; j++) {
            const int k = (j + 1) % 3, q = (j + 2) % 3;
            const double2 p = A[3 + k], r = A[6 + q], u = A[3 + q], v = A[6 + k];
            const double cre = (p.x * r.x - p.y * r.y) - (u.x * v.x - u.y * v.y);
            const double cim = (p.x * r.y + p.y * r.x) - (u.x * v.y + u.y * v.x);
            dre += A[j].x * cre - A[j].y * cim;
            dim += A[j].x * cim + A[j].y * cre;
        }
        dev = fmax(dev, fabs(dre - 1.0));
        dev = fmax(dev, fabs(dim));
        m = fmaxf(m, (float)dev);
    }
    for (int o = 16; o > 0; o >>= 1)
        m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, __float_as_uint(m));
}

cudaError_t launch_su3_deviation(const double *U, long long nlinks, unsigned *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    su3_dev_kernel<<<1024, 256, 0, s>>>((const double2 *)U, nlinks, out);
    return cudaGetLastError();
}

cudaError_t launch_fold_links(int prec, const Geom &g, const double bc[4], double c1, double c3,
                              const double *fat, const double *lng, void *links,
                              const float inv_scale[2], cudaStream_t s) {
    FoldArgs fa;
    fa.g = g;
    fa.inv_scale[0] = inv_scale ? inv_scale[0] : 0.f;
    fa.inv_scale[1] = inv_scale ? inv_scale[1] : 0.f;
    for (int k = 0; k < 4; k++)
        fa.bc[k] = bc[k];
    fa.c1 = c1;
    fa.c3 = c3;
    const long long n = 16LL * g.Vh;
    const int grid = (int)((n + 255) / 256);
    STAG_PREC_SWITCH(prec, {
        fold_kernel<P><<<grid, 256, 0, s>>>(fa, fat, lng, (char *)links);
    });
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// largest |re| or |im| of a canonical link field (for the 16-bit scales);
// non-negative floats order like their bit patterns, so atomicMax on the
// bits finds the maximum
// --------------------------------------------------------------------------
__global__ void absmax_kernel(const double *__restrict__ a, long long n, unsigned *out) {
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v = (float)fabs(a[i]);
        if (!(v <= FLT_MAX))  // NaN, infinity and FP32 overflow all count as infinite
            v = INFINITY;
        m = fmaxf(m, v);
    }
    for (int o = 16; o > 0; o >>= 1)
        m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, __float_as_uint(m));
}

cudaError_t launch_absmax(const double *a, long long n, unsigned *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    absmax_kernel<<<1024, 256, 0, s>>>(a, n, out);
    return cudaGetLastError();
}

// *flag = 1 if a finite entry lies beyond the FP32 range (NaN and infinity
// pass: the solvers report them as breakdowns)
__global__ void finite_overflow_kernel(const double *__restrict__ a, long long n, unsigned *flag) {
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = fabs(a[i]);
        bad |= v > (double)FLT_MAX && v < INFINITY;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
        atomicOr(flag, 1u);
}

cudaError_t launch_finite_overflow(const double *a, long long n, unsigned *flag, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    finite_overflow_kernel<<<1024, 256, 0, s>>>(a, n, flag);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// exact power-of-two rescaling of a colour field (the solvers' source
// normalisation): the largest |component| (double-float: of the hi parts)
// as float bits, and v *= 2^e
// --------------------------------------------------------------------------
template <int P> STAG_D float elem_absmax(typename Fmt<P>::Elem v);
template <> STAG_D float elem_absmax<P_F64>(double2 v) { return (float)fmax(fabs(v.x), fabs(v.y)); }
template <> STAG_D float elem_absmax<P_DF64>(float4 v) { return fmaxf(fabsf(v.x), fabsf(v.z)); }
template <> STAG_D float elem_absmax<P_F32>(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }

template <int P> STAG_D typename Fmt<P>::Elem elem_ldexp(typename Fmt<P>::Elem v, int e);
template <> STAG_D double2 elem_ldexp<P_F64>(double2 v, int e) { return make_double2(ldexp(v.x, e), ldexp(v.y, e)); }
template <> STAG_D float4 elem_ldexp<P_DF64>(float4 v, int e) {
    return make_float4(ldexpf(v.x, e), ldexpf(v.y, e), ldexpf(v.z, e), ldexpf(v.w, e));
}
template <> STAG_D float2 elem_ldexp<P_F32>(float2 v, int e) { return make_float2(ldexpf(v.x, e), ldexpf(v.y, e)); }

template <int P>
__global__ void field_absmax_kernel(Geom g, const typename Fmt<P>::Elem *__restrict__ v, unsigned *out) {
    float m = 0.f;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.Vh; c += gridDim.x * blockDim.x)
#pragma unroll
        for (int a = 0; a < 3; a++)
            m = fmaxf(m, elem_absmax<P>(v[(size_t)a * g.stride + c]));  // fmaxf drops NaN
    for (int o = 16; o > 0; o >>= 1)
        m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, __float_as_uint(m));
}

template <int P>
__global__ void field_ldexp_kernel(Geom g, typename Fmt<P>::Elem *v, int e) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.Vh)
        return;
#pragma unroll
    for (int a = 0; a < 3; a++)
        v[(size_t)a * g.stride + c] = elem_ldexp<P>(v[(size_t)a * g.stride + c], e);
}

#define STAG_SRC_SWITCH(prec, ...)                                    \
    switch (prec) {                                                   \
    case P_F64: { constexpr int P = P_F64; __VA_ARGS__; } break;      \
    case P_DF64: { constexpr int P = P_DF64; __VA_ARGS__; } break;    \
    case P_F32: { constexpr int P = P_F32; __VA_ARGS__; } break;      \
    default: return cudaErrorInvalidValue;                            \
    }

cudaError_t launch_field_absmax(int prec, const Geom &g, const void *v, unsigned *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    STAG_SRC_SWITCH(prec, field_absmax_kernel<P><<<512, 256, 0, s>>>(g, (const typename Fmt<P>::Elem *)v, out));
    return cudaGetLastError();
}

cudaError_t launch_field_ldexp(int prec, const Geom &g, void *v, int e, cudaStream_t s) {
    STAG_SRC_SWITCH(prec, field_ldexp_kernel<P><<<(g.Vh + 255) / 256, 256, 0, s>>>(g, (typename Fmt<P>::Elem *)v, e));
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// three-link products (FP64): N_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu)
// --------------------------------------------------------------------------
STAG_D void mat_mul_c(double2 C[9], const double2 A[9], const double2 B[9]) {
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < 3; k++) {
                const double2 x = A[3 * a + k], y = B[3 * k + b];
                re = fma(x.x, y.x, re);
                re = fma(-x.y, y.y, re);
                im = fma(x.x, y.y, im);
                im = fma(x.y, y.x, im);
            }
            C[3 * a + b] = make_double2(re, im);
        }
}

__global__ void long_links_kernel(Geom g, const double2 *__restrict__ U, double2 *__restrict__ N) {
    const long long V = 2LL * g.Vh;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 4 * V)
        return;
    const int mu = (int)(t / V);
    const long long i = t % V;
    int x[4];
    full_coords(g, i, x);
    long long step = 1;
    for (int nu = 0; nu < mu; nu++)
        step *= g.L[nu];
    const int L = g.L[mu];
    const long long i1 = i + ((x[mu] + 1) % L - x[mu]) * step;
    const long long i2 = i + ((x[mu] + 2) % L - x[mu]) * step;
    double2 A[9], B[9], T[9];
    for (int j = 0; j < 9; j++) {
        A[j] = U[((size_t)mu * V + i) * 9 + j];
        B[j] = U[((size_t)mu * V + i1) * 9 + j];
    }
    mat_mul_c(T, A, B);
    for (int j = 0; j < 9; j++)
        B[j] = U[((size_t)mu * V + i2) * 9 + j];
    mat_mul_c(A, T, B);
    for (int j = 0; j < 9; j++)
        N[((size_t)mu * V + i) * 9 + j] = A[j];
}

cudaError_t launch_long_links(const Geom &g, const double *fat, double *lng, cudaStream_t s) {
    const long long n = 8LL * g.Vh;
    const int grid = (int)((n + 127) / 128);
    long_links_kernel<<<grid, 128, 0, s>>>(g, (const double2 *)fat, (double2 *)lng);
    return cudaGetLastError();
}

}  // namespace stag
