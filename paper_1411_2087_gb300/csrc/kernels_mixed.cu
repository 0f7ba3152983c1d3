// Mixed-precision CG with reliable updates (Sleijpen & van der Vorst's
// reliable-updated residuals, as used for lattice solvers by Clark et al.).
//
// The iteration runs in a low precision `lo` (FP32 or 16-bit storage): the
// search direction p, M p, the iterated residual r_s and the correction x_s
// accumulated since the last update.  Whenever |r_s| falls below
// delta * (largest |r_s| since the last update), or the low-precision
// residual claims convergence, the correction is added to the solution x in
// the high precision `hi` (FP64 or double-float), the true residual
// r = b - M x is recomputed in `hi`, and r_s restarts from it.  Convergence
// is only declared on a recomputed true residual.
//
// Per iteration (one graph body):
//   D_oe p -> t_s;  Ap = m^2 p - D_eo t_s, alpha          (lo, Dslash kernels)
//   x_s += alpha p, r_s -= alpha Ap, |r_s|^2, decide      (mixed_update)
//   if reliable: x += x_s, x_s = 0                        (mixed_accum, gated)
//                r = b - M x, |r|^2                        (hi Dslash kernels, gated)
//                r_s = r, beta = |r|^2/rr                  (mixed_restart, gated)
//   (in a graph the four gated kernels sit in a conditional IF node that
//   mixed_update opens, so that iterations without an update launch none)
//   p = r_s + beta p                                      (cg_p_kernel)
// With a flexible preconditioner (sc->fcg) the direction update is
// p = z + beta p, z = N(r_s), and the preconditioner step sets beta and
// rr = <r_s, z>; mixed_update and mixed_restart then leave both alone.
#include "dslash.cuh"
#include "kernels.h"

namespace stag {

STAG_D void set_loop_condition_m(CgScalars *sc) {
    if (sc->has_cond)
        cudaGraphSetConditional(sc->cond, sc->status == CG_RUNNING ? 1u : 0u);
}

constexpr int MB = 256;

static int grid_of(const Geom &g) { return (g.Vh + MB - 1) / MB; }

// x = 0, r = b (hi); x_s = 0 (F32); r_s = p = b (lo); |b|^2
template <int PH, int PL>
__global__ void __launch_bounds__(MB)
mixed_init_kernel(Geom g, typename Fmt<PH>::Elem *x, typename Fmt<PH>::Elem *r,
                  const typename Fmt<PH>::Elem *b, float2 *xs, typename Fmt<PL>::Elem *rs,
                  typename Fmt<PL>::Elem *p, double *partial, CgScalars *sc) {
    using RH = typename Fmt<PH>::R;
    using RL = typename Fmt<PL>::R;
    __shared__ double smem[32];
    const int c = blockIdx.x * MB + threadIdx.x;
    red_t<RH> dot = red_zero<red_t<RH>>();
    if (c < g.Vh) {
        cplx<RH> bv[3], zh[3];
        cplx<RL> bl[3];
        cplx<float> zf[3];
        load_vec<PH>(b, g.stride, c, bv);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            zh[k] = czero<RH>();
            zf[k] = czero<float>();
            bl[k] = cconv<RL, RH>(bv[k]);
        }
        store_vec<PH>(x, g.stride, c, zh);
        store_vec<PH>(r, g.stride, c, bv);
        store_vec<P_F32>(xs, g.stride, c, zf);
        store_vec<PL>(rs, g.stride, c, bl);
        store_vec<PL>(p, g.stride, c, bl);
        dot = re_dot3<RH>(bv, bv);
    }
    double total;
    if (grid_sum<MB>(dot, partial, &sc->ticket, smem, total) && threadIdx.x == 0) {
        sc->bb = total;
        sc->rr = total;
        sc->true_rr = total;
        sc->rr_stop = sc->tol2 * total;
        sc->rmax = sqrt(total);
        sc->iter = 0;
        sc->restarts = 0;
        sc->reliable = 0;
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
        set_loop_condition_m(sc);
    }
}

// x_s += alpha p, r_s -= alpha Ap, |r_s|^2; decide whether to update
template <int PL>
__global__ void __launch_bounds__(MB)
mixed_update_kernel(Geom g, float2 *xs, typename Fmt<PL>::Elem *rs, const typename Fmt<PL>::Elem *p,
                    const typename Fmt<PL>::Elem *Ap, double *partial, CgScalars *sc) {
    using RL = typename Fmt<PL>::R;
    __shared__ double smem[32];
    const int c = blockIdx.x * MB + threadIdx.x;
    const bool run = sc->status == CG_RUNNING;
    red_t<RL> dot = red_zero<red_t<RL>>();
    if (run && c < g.Vh) {
        const float alpha = scalar_as<float>(sc->alpha);
        cplx<float> xv[3];
        cplx<RL> rv[3], pv[3], av[3];
        load_vec<P_F32>(xs, g.stride, c, xv);
        load_vec<PL>(rs, g.stride, c, rv);
        load_vec<PL>(p, g.stride, c, pv);
        load_vec<PL>(Ap, g.stride, c, av);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            xv[k].re = fmaf(alpha, (float)pv[k].re, xv[k].re);
            xv[k].im = fmaf(alpha, (float)pv[k].im, xv[k].im);
            rv[k].re = fmaf(-alpha, av[k].re, rv[k].re);
            rv[k].im = fmaf(-alpha, av[k].im, rv[k].im);
        }
        store_vec<P_F32>(xs, g.stride, c, xv);
        store_vec<PL>(rs, g.stride, c, rv);
        dot = re_dot3<RL>(rv, rv);
    }
    double total;
    if (grid_sum<MB>(dot, partial, &sc->ticket, smem, total) && threadIdx.x == 0) {
        sc->reliable = 0;
        if (sc->status == CG_RUNNING) {
            sc->iter += 1;
            const double rn = sqrt(total);
            if (!(total < INFINITY)) {
                sc->status = CG_BREAKDOWN;
            } else if (sc->iter > sc->max_iter) {
                // the update requested at max_iter ends the solve; this only
                // guards the loop if that update did not run
                sc->status = CG_MAXITER;
            } else if (rn < sc->delta * sc->rmax || total <= sc->rr_stop || sc->iter >= sc->max_iter) {
                sc->reliable = 1;
            } else {
                if (sc->fcg) {
                    sc->fcg_rr = total;
                } else {
                    sc->beta = make_dpair(total / sc->rr);
                    sc->rr = total;
                }
                sc->rmax = fmax(sc->rmax, rn);
            }
        }
        if (sc->has_rel_cond)
            cudaGraphSetConditional(sc->rel_cond, sc->reliable ? 1u : 0u);
        set_loop_condition_m(sc);
    }
}

// x += x_s, x_s = 0 (only when this iteration updates)
template <int PH>
__global__ void __launch_bounds__(MB)
mixed_accum_kernel(Geom g, typename Fmt<PH>::Elem *x, float2 *xs, const CgScalars *sc) {
    using RH = typename Fmt<PH>::R;
    if (sc->reliable == 0)
        return;
    const int c = blockIdx.x * MB + threadIdx.x;
    if (c >= g.Vh)
        return;
    cplx<RH> xv[3];
    cplx<float> sv[3], z[3];
    load_vec<PH>(x, g.stride, c, xv);
    load_vec<P_F32>(xs, g.stride, c, sv);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        xv[k].re = radd(xv[k].re, rconv<RH, float>(sv[k].re));
        xv[k].im = radd(xv[k].im, rconv<RH, float>(sv[k].im));
        z[k] = czero<float>();
    }
    store_vec<PH>(x, g.stride, c, xv);
    store_vec<P_F32>(xs, g.stride, c, z);
}

// r_s = r; scalars after the true residual (only when this iteration updates)
template <int PH, int PL>
__global__ void __launch_bounds__(MB)
mixed_restart_kernel(Geom g, const typename Fmt<PH>::Elem *r, typename Fmt<PL>::Elem *rs, CgScalars *sc) {
    using RH = typename Fmt<PH>::R;
    using RL = typename Fmt<PL>::R;
    // every block reads the gate before block 0 changes any scalar below,
    // and block 0 does not change the gate
    if (sc->reliable == 0)
        return;
    const int c = blockIdx.x * MB + threadIdx.x;
    if (c < g.Vh) {
        cplx<RH> rv[3];
        cplx<RL> lv[3];
        load_vec<PH>(r, g.stride, c, rv);
#pragma unroll
        for (int k = 0; k < 3; k++)
            lv[k] = cconv<RL, RH>(rv[k]);
        store_vec<PL>(rs, g.stride, c, lv);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rt = sc->true_rr;
        sc->restarts += 1;
        if (!(rt < INFINITY))
            sc->status = CG_BREAKDOWN;
        else if (rt <= sc->rr_stop)
            sc->status = CG_CONVERGED;
        else if (sc->iter >= sc->max_iter)
            sc->status = CG_MAXITER;
        if (sc->fcg) {
            sc->fcg_rr = rt;
        } else {
            sc->beta = make_dpair(rt / sc->rr);
            sc->rr = rt;
        }
        sc->rmax = sqrt(rt);
        set_loop_condition_m(sc);
    }
}

#define HI_SWITCH(hi, ...)                                                    \
    switch (hi) {                                                             \
    case P_F64: { constexpr int PH = P_F64; __VA_ARGS__; } break;             \
    case P_DF64: { constexpr int PH = P_DF64; __VA_ARGS__; } break;           \
    default: return cudaErrorInvalidValue;                                    \
    }
#define LO_SWITCH(lo, ...)                                                    \
    switch (lo) {                                                             \
    case P_F32: { constexpr int PL = P_F32; __VA_ARGS__; } break;             \
    case P_F16: { constexpr int PL = P_F16; __VA_ARGS__; } break;             \
    default: return cudaErrorInvalidValue;                                    \
    }

cudaError_t launch_mixed_init(int hi, int lo, const Geom &g, void *x, void *r, const void *b, float *xs,
                              void *rs, void *p, double *partial, CgScalars *sc, cudaStream_t s) {
    HI_SWITCH(hi, LO_SWITCH(lo, {
        using EH = typename Fmt<PH>::Elem;
        using EL = typename Fmt<PL>::Elem;
        mixed_init_kernel<PH, PL><<<grid_of(g), MB, 0, s>>>(g, (EH *)x, (EH *)r, (const EH *)b,
                                                            (float2 *)xs, (EL *)rs, (EL *)p, partial, sc);
    }));
    return cudaGetLastError();
}

cudaError_t launch_mixed_update(int lo, const Geom &g, float *xs, void *rs, const void *p, const void *Ap,
                                double *partial, CgScalars *sc, cudaStream_t s) {
    LO_SWITCH(lo, {
        using EL = typename Fmt<PL>::Elem;
        mixed_update_kernel<PL><<<grid_of(g), MB, 0, s>>>(g, (float2 *)xs, (EL *)rs, (const EL *)p,
                                                          (const EL *)Ap, partial, sc);
    });
    return cudaGetLastError();
}

cudaError_t launch_mixed_accum(int hi, const Geom &g, void *x, float *xs, const CgScalars *sc,
                               cudaStream_t s) {
    HI_SWITCH(hi, {
        using EH = typename Fmt<PH>::Elem;
        mixed_accum_kernel<PH><<<grid_of(g), MB, 0, s>>>(g, (EH *)x, (float2 *)xs, sc);
    });
    return cudaGetLastError();
}

cudaError_t launch_mixed_restart(int hi, int lo, const Geom &g, const void *r, void *rs, CgScalars *sc,
                                 cudaStream_t s) {
    HI_SWITCH(hi, LO_SWITCH(lo, {
        using EH = typename Fmt<PH>::Elem;
        using EL = typename Fmt<PL>::Elem;
        mixed_restart_kernel<PH, PL><<<grid_of(g), MB, 0, s>>>(g, (const EH *)r, (EL *)rs, sc);
    }));
    return cudaGetLastError();
}

}  // namespace stag
