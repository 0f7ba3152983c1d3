// Multi-shift CG: (M + sigma_s) x_s = b for all shifts s at the price of one
// Krylov space (Jegerlehner's shifted CG; the paper's Sec. 3 benchmarks the
// HISQ multishift solver with 9 or 11 shifts).
//
// The base system is the smallest shift sigma_0 (the worst conditioned); the
// Dslash pair and the residual r belong to it.  For a shift with
// Delta_s = sigma_s - sigma_0 >= 0 the residual stays collinear,
// r_s = zeta_s r, and with the base CG's alpha_k, beta_k:
//
//   zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
//                [ alpha_k beta_{k-1} (zeta_{k-1} - zeta_k)
//                  + zeta_{k-1} alpha_{k-1} (1 + Delta_s alpha_k) ]
//   alpha^s_k  = alpha_k zeta_{k+1} / zeta_k
//   x_s       += alpha^s_k p_s
//   beta^s_k   = beta_k (zeta_{k+1} / zeta_k)^2
//   p_s        = zeta_{k+1} r + beta^s_k p_s
//
// starting from zeta_{-1} = zeta_0 = 1, alpha_{-1} = 1, beta_{-1} = 0,
// x_s = 0, p_s = b.  The base is the shift with Delta = 0, for which the
// recurrence keeps zeta = 1, so every system, the base included, is updated
// by the same code.  A shift stops (its x_s and p_s freeze) once
// zeta_{k+1}^2 |r|^2 <= tol^2 |b|^2.
//
// Mixed precision (MsArgs::p_lo set): the vectors stay in the high precision
// P and only the Dslash pair runs in the low precision PL, on a copy p_lo of
// the base direction that ms_p_kernel writes; M p arrives in PL.  Whenever
// |r| has dropped below delta times its largest value since the last update,
// or every shift claims convergence, the base residual is recomputed in P,
// r = b - (M + sigma_0) x_0 (reliable update; the shifted residuals stay
// zeta_s r), and convergence is only declared on such a residual.  The
// Dslash pair of an iteration runs in P instead while |r| > theta |b|: a
// rounding error of the operator enters every shifted solution in proportion
// to |r| at the time, and the shifted solutions cannot be corrected inside
// the shared space later, so the early iterations, where |r| is large, use
// the exact operator (sc->ms_hi_op / ms_lo_op gate the two paths).
#include "dslash.cuh"
#include "kernels.h"

namespace stag {

constexpr int MSB = 256;

static int grid_of(const Geom &g) { return (g.Vh + MSB - 1) / MSB; }

STAG_D void ms_set_condition(CgScalars *sc) {
    if (sc->has_cond)
        cudaGraphSetConditional(sc->cond, sc->status == CG_RUNNING ? 1u : 0u);
}

// x_s = 0, p_s = b for all shifts; r = b; |b|^2; shift state reset
template <int P, int PL>
__global__ void __launch_bounds__(MSB)
ms_init_kernel(Geom g, MsArgs a, double *partial, CgScalars *sc, ShiftState *st) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    __shared__ double smem[32];
    const int c = blockIdx.x * MSB + threadIdx.x;
    red_t<R> dot = red_zero<red_t<R>>();
    if (c < g.Vh) {
        cplx<R> bv[3], z[3];
        load_vec<P>((const E *)a.b, g.stride, c, bv);
#pragma unroll
        for (int k = 0; k < 3; k++)
            z[k] = czero<R>();
        store_vec<P>((E *)a.r, g.stride, c, bv);
        for (int s = 0; s < a.n; s++) {
            store_vec<P>((E *)a.x[s], g.stride, c, z);
            store_vec<P>((E *)a.p[s], g.stride, c, bv);
        }
        if constexpr (PL >= 0) {
            using RL = typename Fmt<PL>::R;
            cplx<RL> lv[3];
#pragma unroll
            for (int k = 0; k < 3; k++)
                lv[k] = cconv<RL, R>(bv[k]);
            store_vec<PL>((typename Fmt<PL>::Elem *)a.p_lo, g.stride, c, lv);
        }
        dot = re_dot3<R>(bv, bv);
    }
    double total;
    if (grid_sum<MSB>(dot, partial, &sc->ticket, smem, total) && threadIdx.x == 0) {
        sc->bb = total;
        sc->rr = total;
        sc->rr_stop = sc->tol2 * total;
        sc->iter = 0;
        sc->alpha = make_dpair(0.0);
        sc->beta = make_dpair(0.0);
        sc->alpha_prev = 1.0;
        sc->beta_prev = 0.0;
        sc->ms_xdone = 0;
        sc->rmax = sqrt(total);
        sc->reliable = 0;
        sc->restarts = 0;
        sc->ms_hi_op = total > a.theta2 * total ? 1 : 0;
        sc->ms_lo_op = 1 - sc->ms_hi_op;
        const bool done = total <= sc->rr_stop;
        for (int s = 0; s < a.n; s++) {
            st[s].zeta_prev = 1.0;
            st[s].zeta = 1.0;
            st[s].active = done ? 0 : 1;
            st[s].iters = 0;
            st[s].alpha_s = make_dpair(0.0);
            st[s].beta_s = make_dpair(0.0);
            st[s].zeta_next = make_dpair(1.0);
        }
        if (!(total < INFINITY))
            sc->status = CG_BREAKDOWN;
        else if (done)
            sc->status = CG_CONVERGED;
        else if (sc->max_iter <= 0)
            sc->status = CG_MAXITER;
        else
            sc->status = CG_RUNNING;
        ms_set_condition(sc);
    }
}

// zeta_{k+1}, alpha^s for every shift from the scalars of the base CG; every
// block computes them (one lane per shift) into shared memory
STAG_D void ms_shift_scalars(const MsArgs &a, const CgScalars *sc, const ShiftState *st,
                             double *zeta_next, double *alpha_s) {
    const int s = threadIdx.x;
    if (s < a.n) {
        const double al = sc->alpha.d, alp = sc->alpha_prev, bep = sc->beta_prev;
        const double z = st[s].zeta, zp = st[s].zeta_prev;
        const double den = al * bep * (zp - z) + zp * alp * (1.0 + a.delta[s] * al);
        const double zn = z * zp * alp / den;
        zeta_next[s] = zn;
        alpha_s[s] = al * zn / z;
    }
}

// r -= alpha Ap, |r|^2; the shift scalars of this iteration (the solution
// updates x_s += alpha^s p_s run in ms_p_kernel, which reads p_s anyway)
template <int P, int PA>
__global__ void __launch_bounds__(MSB)
ms_update_kernel(Geom g, MsArgs a, const void *Ap, double *partial, CgScalars *sc, ShiftState *st) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    using RA = typename Fmt<PA>::R;
    __shared__ double smem[32];
    __shared__ double zeta_next[MS_MAX], alpha_s[MS_MAX];
    __shared__ int active[MS_MAX];
    // the previous iteration's solution updates are done (ms_p_kernel has
    // finished); written before this block's ticket, so before the last
    // block below advances the iteration count
    if (blockIdx.x == 0 && threadIdx.x == 0)
        sc->ms_xdone = sc->iter;
    const bool run = sc->status == CG_RUNNING;
    // which path computed M p this iteration (read before any block's ticket,
    // so before the last block below sets it for the next iteration)
    const bool hi_path = PA == P || sc->ms_hi_op;
    if (run)
        ms_shift_scalars(a, sc, st, zeta_next, alpha_s);
    if (threadIdx.x < MS_MAX)
        active[threadIdx.x] = threadIdx.x < a.n ? st[threadIdx.x].active : 0;
    __syncthreads();
    const int c = blockIdx.x * MSB + threadIdx.x;
    red_t<R> dot = red_zero<red_t<R>>();
    if (run && c < g.Vh) {
        const R alpha = scalar_as<R>(sc->alpha);
        cplx<R> rv[3], av[3];
        load_vec<P>((const E *)a.r, g.stride, c, rv);
        if (hi_path) {
            load_vec<P>((const E *)(PA == P ? Ap : a.Ap_hi), g.stride, c, av);
        } else {
            cplx<RA> al[3];
            load_vec<PA>((const typename Fmt<PA>::Elem *)Ap, g.stride, c, al);
#pragma unroll
            for (int k = 0; k < 3; k++)
                av[k] = cconv<R, RA>(al[k]);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            mac(rv[k].re, -alpha, av[k].re);
            mac(rv[k].im, -alpha, av[k].im);
            rv[k].re = rnorm<R>(rv[k].re);
            rv[k].im = rnorm<R>(rv[k].im);
        }
        store_vec<P>((E *)a.r, g.stride, c, rv);
        dot = re_dot3<R>(rv, rv);
    }
    double total;
    if (grid_sum<MSB>(dot, partial, &sc->ticket, smem, total) && threadIdx.x == 0) {
        if (sc->status == CG_RUNNING) {
            const double beta = total / sc->rr;
            sc->beta = make_dpair(beta);
            sc->iter += 1;
            bool any = false;
            for (int s = 0; s < a.n; s++) {
                if (!active[s])
                    continue;
                const double zn = zeta_next[s], z = st[s].zeta;
                const double ratio = zn / z;
                st[s].alpha_s = make_dpair(alpha_s[s]);
                st[s].beta_s = make_dpair(beta * ratio * ratio);
                st[s].zeta_next = make_dpair(zn);
                st[s].zeta_prev = z;
                st[s].zeta = zn;
                st[s].iters = sc->iter;
                // the shifted residual zeta r meets the tolerance: freeze
                // after this iteration's x update (iters == iter marks it
                // for ms_p_kernel; p_s is not needed again)
                if (zn * zn * total <= sc->rr_stop)
                    st[s].active = 0;
                else
                    any = true;
            }
            sc->alpha_prev = sc->alpha.d;
            sc->beta_prev = beta;
            sc->rr = total;
            const double rn = sqrt(total);
            sc->reliable = 0;
            if (!(total < INFINITY)) {
                sc->status = CG_BREAKDOWN;
            } else if (sc->delta > 0.0 && ((!hi_path && rn < sc->delta * sc->rmax) || !any ||
                                           sc->iter >= sc->max_iter)) {
                // mixed precision: the base residual is recomputed first, and
                // the stop is decided on it (ms_restart_kernel); iterations on
                // the exact operator need no update on the way
                sc->reliable = 1;
            } else if (!any) {
                sc->status = CG_CONVERGED;
            } else if (sc->iter >= sc->max_iter) {
                sc->status = CG_MAXITER;
            }
            sc->rmax = fmax(sc->rmax, rn);
            sc->ms_hi_op = total > a.theta2 * sc->bb ? 1 : 0;
            sc->ms_lo_op = 1 - sc->ms_hi_op;
        }
        if (sc->has_rel_cond)
            cudaGraphSetConditional(sc->rel_cond, sc->reliable ? 1u : 0u);
        ms_set_condition(sc);
    }
}

// after a reliable update (r = b - (M + sigma_0) x_0 recomputed, |r|^2 in
// true_rr): the base CG continues from the true residual; the stop decided
// on it (one block, one thread)
__global__ void ms_restart_kernel(const MsArgs a, CgScalars *sc, ShiftState *st) {
    if (sc->reliable == 0 || threadIdx.x != 0)
        return;
    const double rt = sc->true_rr;
    sc->restarts += 1;
    sc->rr = rt;
    sc->rmax = sqrt(rt);
    sc->ms_hi_op = rt > a.theta2 * sc->bb ? 1 : 0;
    sc->ms_lo_op = 1 - sc->ms_hi_op;
    bool any = false;
    for (int s = 0; s < a.n; s++)
        any |= st[s].active != 0;
    if (!(rt < INFINITY))
        sc->status = CG_BREAKDOWN;
    else if (!any)
        sc->status = CG_CONVERGED;
    else if (sc->iter >= sc->max_iter)
        sc->status = CG_MAXITER;
    ms_set_condition(sc);
}

// x_s += alpha^s p_s for the shifts active in this iteration, then
// p_s = zeta_{k+1} r + beta^s p_s for those still active
template <int P, int PL>
__global__ void __launch_bounds__(MSB)
ms_p_kernel(Geom g, MsArgs a, const CgScalars *sc, const ShiftState *st) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    // this iteration's solution updates are due unless already applied (a
    // host-driven launch after the solve ended finds them done)
    const int it = sc->iter;
    const bool xdue = sc->ms_xdone != it;
    const bool running = sc->status == CG_RUNNING;
    if (!xdue && !running)
        return;
    const int c = blockIdx.x * MSB + threadIdx.x;
    if (c >= g.Vh)
        return;
    cplx<R> rv[3];
    if (running)
        load_vec<P>((const E *)a.r, g.stride, c, rv);
    for (int s = 0; s < a.n; s++) {
        const bool xs = xdue && st[s].iters == it;   // was active in this iteration
        const bool ps = running && st[s].active;     // still active
        if (!xs && !ps)
            continue;
        cplx<R> pv[3];
        load_vec<P>((const E *)a.p[s], g.stride, c, pv);
        if (xs) {
            // x_s += alpha^s p_s with the direction of this iteration
            const R as = scalar_as<R>(st[s].alpha_s);
            cplx<R> xv[3];
            load_vec<P>((const E *)a.x[s], g.stride, c, xv);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                mac(xv[k].re, as, pv[k].re);
                mac(xv[k].im, as, pv[k].im);
                xv[k].re = rnorm<R>(xv[k].re);
                xv[k].im = rnorm<R>(xv[k].im);
            }
            store_vec<P>((E *)a.x[s], g.stride, c, xv);
        }
        if (!ps)
            continue;
        const R z = scalar_as<R>(st[s].zeta_next);
        const R bs = scalar_as<R>(st[s].beta_s);
        cplx<R> o[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            o[k].re = rzero<R>();
            o[k].im = rzero<R>();
            mac(o[k].re, z, rv[k].re);
            mac(o[k].im, z, rv[k].im);
            mac(o[k].re, bs, pv[k].re);
            mac(o[k].im, bs, pv[k].im);
            o[k].re = rnorm<R>(o[k].re);
            o[k].im = rnorm<R>(o[k].im);
        }
        store_vec<P>((E *)a.p[s], g.stride, c, o);
        if constexpr (PL >= 0) {
            if (s == a.base) {
                // the low-precision copy of the base direction for the Dslash
                using RL = typename Fmt<PL>::R;
                cplx<RL> lv[3];
#pragma unroll
                for (int k = 0; k < 3; k++)
                    lv[k] = cconv<RL, R>(o[k]);
                store_vec<PL>((typename Fmt<PL>::Elem *)a.p_lo, g.stride, c, lv);
            }
        }
    }
}

// y += x (same precision), used to add refinement corrections
template <int P>
__global__ void __launch_bounds__(MSB)
axpy1_kernel(Geom g, const typename Fmt<P>::Elem *x, typename Fmt<P>::Elem *y) {
    using R = typename Fmt<P>::R;
    const int c = blockIdx.x * MSB + threadIdx.x;
    if (c >= g.Vh)
        return;
    cplx<R> xv[3], yv[3];
    load_vec<P>(x, g.stride, c, xv);
    load_vec<P>(y, g.stride, c, yv);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        yv[k].re = radd(yv[k].re, xv[k].re);
        yv[k].im = radd(yv[k].im, xv[k].im);
    }
    store_vec<P>(y, g.stride, c, yv);
}

// out = in converted between precisions
template <int PO, int PI>
__global__ void __launch_bounds__(MSB)
convert_kernel(Geom g, const typename Fmt<PI>::Elem *in, typename Fmt<PO>::Elem *out) {
    using RI = typename Fmt<PI>::R;
    using RO = typename Fmt<PO>::R;
    const int c = blockIdx.x * MSB + threadIdx.x;
    if (c >= g.Vh)
        return;
    cplx<RI> iv[3];
    cplx<RO> ov[3];
    load_vec<PI>(in, g.stride, c, iv);
#pragma unroll
    for (int k = 0; k < 3; k++)
        ov[k] = cconv<RO, RI>(iv[k]);
    store_vec<PO>(out, g.stride, c, ov);
}

#define MS_PREC_SWITCH(prec, ...)                                         \
    switch (prec) {                                                       \
    case P_F64: { constexpr int P = P_F64; __VA_ARGS__; } break;          \
    case P_DF64: { constexpr int P = P_DF64; __VA_ARGS__; } break;        \
    case P_F32: { constexpr int P = P_F32; __VA_ARGS__; } break;          \
    default: return cudaErrorInvalidValue;                                \
    }

// lo: the precision of the Dslash pair (-1: the vectors' own precision);
// mixed precision exists for F64 and DF64 vectors with an FP32 operator
cudaError_t launch_ms_init(int prec, const Geom &g, const MsArgs &a, double *partial, CgScalars *sc,
                           ShiftState *st, cudaStream_t s, int lo) {
    if (lo == P_F32 && (prec == P_F64 || prec == P_DF64)) {
        if (prec == P_F64)
            ms_init_kernel<P_F64, P_F32><<<grid_of(g), MSB, 0, s>>>(g, a, partial, sc, st);
        else
            ms_init_kernel<P_DF64, P_F32><<<grid_of(g), MSB, 0, s>>>(g, a, partial, sc, st);
        return cudaGetLastError();
    }
    if (lo >= 0)
        return cudaErrorInvalidValue;
    MS_PREC_SWITCH(prec, ms_init_kernel<P, -1><<<grid_of(g), MSB, 0, s>>>(g, a, partial, sc, st));
    return cudaGetLastError();
}

cudaError_t launch_ms_update(int prec, const Geom &g, const MsArgs &a, const void *Ap, double *partial,
                             CgScalars *sc, ShiftState *st, cudaStream_t s, int lo) {
    if (lo == P_F32 && (prec == P_F64 || prec == P_DF64)) {
        if (prec == P_F64)
            ms_update_kernel<P_F64, P_F32><<<grid_of(g), MSB, 0, s>>>(g, a, Ap, partial, sc, st);
        else
            ms_update_kernel<P_DF64, P_F32><<<grid_of(g), MSB, 0, s>>>(g, a, Ap, partial, sc, st);
        return cudaGetLastError();
    }
    if (lo >= 0)
        return cudaErrorInvalidValue;
    MS_PREC_SWITCH(prec, ms_update_kernel<P, P><<<grid_of(g), MSB, 0, s>>>(g, a, Ap, partial, sc, st));
    return cudaGetLastError();
}

cudaError_t launch_ms_p(int prec, const Geom &g, const MsArgs &a, const CgScalars *sc,
                        const ShiftState *st, cudaStream_t s, int lo) {
    if (lo == P_F32 && (prec == P_F64 || prec == P_DF64)) {
        if (prec == P_F64)
            ms_p_kernel<P_F64, P_F32><<<grid_of(g), MSB, 0, s>>>(g, a, sc, st);
        else
            ms_p_kernel<P_DF64, P_F32><<<grid_of(g), MSB, 0, s>>>(g, a, sc, st);
        return cudaGetLastError();
    }
    if (lo >= 0)
        return cudaErrorInvalidValue;
    MS_PREC_SWITCH(prec, ms_p_kernel<P, -1><<<grid_of(g), MSB, 0, s>>>(g, a, sc, st));
    return cudaGetLastError();
}

cudaError_t launch_ms_restart(const MsArgs &a, CgScalars *sc, ShiftState *st, cudaStream_t s) {
    ms_restart_kernel<<<1, 32, 0, s>>>(a, sc, st);
    return cudaGetLastError();
}

cudaError_t launch_axpy1(int prec, const Geom &g, const void *x, void *y, cudaStream_t s) {
    MS_PREC_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        axpy1_kernel<P><<<grid_of(g), MSB, 0, s>>>(g, (const E *)x, (E *)y);
    });
    return cudaGetLastError();
}

cudaError_t launch_convert(int prec_out, int prec_in, const Geom &g, const void *in, void *out,
                           cudaStream_t s) {
#define CONV(PO, PI)                                                                             \
    if (prec_out == PO && prec_in == PI) {                                                       \
        convert_kernel<PO, PI><<<grid_of(g), MSB, 0, s>>>(g, (const typename Fmt<PI>::Elem *)in, \
                                                          (typename Fmt<PO>::Elem *)out);        \
        return cudaGetLastError();                                                               \
    }
    CONV(P_F32, P_DF64)
    CONV(P_DF64, P_F32)
    CONV(P_F32, P_F64)
    CONV(P_F64, P_F32)
#undef CONV
    return cudaErrorInvalidValue;
}

}  // namespace stag
