// Kernel templates of the batched CG (batched.cuh describes the layout);
// instantiated per precision in batched_<prec>.cu.
#pragma once
#include "batched.cuh"
#include "kernels.h"

namespace stag {

// which systems of this block's group are still iterating
template <int K>
STAG_D void load_active(const BatchArgs &a, const BatchGroup &G, int *act, bool want_running) {
    if (threadIdx.x < K) {
        const int k = threadIdx.x;
        act[k] = k < G.K && (!want_running || a.sys[G.sys0 + k].status == CG_RUNNING) ? 1 : 0;
    }
    __syncthreads();
}

// multi-RHS Dslash: out_k = D in_k for the active systems of the group;
// EPI_M_PAP: out_k = m_k^2 p_k - D in_k and <p_k, out_k> -> alpha_k;
// EPI_RESID: |b_k - (m_k^2 p_k - D in_k)|^2 -> true_rr_k
template <int P, int EPI, int BLOCK, int K>
__global__ void __launch_bounds__(BLOCK) batch_dslash_kernel(BatchArgs a, int out_par, int src_x) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    __shared__ double smem[32];
    __shared__ int act[K];
    const int gi = group_of(a, blockIdx.x);
    const BatchGroup &G = a.grp[gi];
    // the true-residual passes (D of x, then the residual) cover every system
    load_active<K>(a, G, act, EPI != EPI_RESID && !src_x);
    const int lblk = blockIdx.x - G.block0;
    const int c = lblk * BLOCK + threadIdx.x;
    const Geom &g = G.g;
    const int S = g.stride;
    red_t<R> dot[K];
#pragma unroll
    for (int k = 0; k < K; k++)
        dot[k] = red_zero<red_t<R>>();
    if (c < g.Vh) {
        cplx<R> acc[K][3];
#pragma unroll
        for (int k = 0; k < K; k++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                acc[k][j] = czero<R>();
        const E *Gout = (const E *)G.links[out_par];
        const E *Gin = (const E *)G.links[1 - out_par];
        int x[4];
        cb_coords(g, c, out_par, x);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int s = h ? 3 : 1;
                const int kind = 4 * h + mu;
                const float ls = G.link_scale[h];
#pragma unroll
                for (int dir = 0; dir < 2; dir++) {
                    const int j = cb_hop(g, c, x, mu, dir ? -s : s);
                    const E *Lp = dir ? Gin + kind * 9 * S + j : Gout + kind * 9 * S + c;
                    cplx<R> L[9];
#pragma unroll
                    for (int e = 0; e < 9; e++)
                        L[e] = F::unpack_link(ld_stream(Lp + e * S), ls);
#pragma unroll
                    for (int k = 0; k < K; k++) {
                        if (!act[k])
                            continue;
                        // EPI_NONE: D_oe of p (or of x for the true residual);
                        // otherwise D_eo of the odd t
                        const E *vin = (const E *)(EPI == EPI_NONE ? (src_x ? G.x[k] : G.p[k]) : G.t[k]);
                        cplx<R> v[3];
                        load_vec<P>(vin, S, j, v);
                        if (dir) {
#pragma unroll
                            for (int b = 0; b < 3; b++)
                                v[b] = cneg(v[b]);
#pragma unroll
                            for (int r = 0; r < 3; r++)
#pragma unroll
                                for (int b = 0; b < 3; b++)
                                    cmac_conj(acc[k][r], L[3 * b + r], v[b]);
                        } else {
#pragma unroll
                            for (int r = 0; r < 3; r++)
#pragma unroll
                                for (int b = 0; b < 3; b++)
                                    cmac(acc[k][r], L[3 * r + b], v[b]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (!act[k])
                continue;
            if (EPI == EPI_NONE) {
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    acc[k][r].re = rnorm<R>(acc[k][r].re);
                    acc[k][r].im = rnorm<R>(acc[k][r].im);
                }
                store_vec<P>((E *)G.t[k], S, c, acc[k]);
            } else {
                const R m2 = scalar_as<R>(a.sys[G.sys0 + k].m2);
                cplx<R> pv[3], o[3];
                // EPI_RESID: the vector M acts on is x_k
                load_vec<P>((const E *)(EPI == EPI_RESID ? G.x[k] : G.p[k]), S, c, pv);
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    o[r] = cneg(acc[k][r]);
                    mac(o[r].re, m2, pv[r].re);
                    mac(o[r].im, m2, pv[r].im);
                    o[r].re = rnorm<R>(o[r].re);
                    o[r].im = rnorm<R>(o[r].im);
                }
                if (EPI == EPI_RESID) {
                    cplx<R> bv[3];
                    load_vec<P>((const E *)G.b[k], S, c, bv);
#pragma unroll
                    for (int r = 0; r < 3; r++) {
                        o[r].re = rsub(bv[r].re, o[r].re);
                        o[r].im = rsub(bv[r].im, o[r].im);
                    }
                    dot[k] = re_dot3<R>(o, o);
                } else {
                    store_vec<P>((E *)G.Ap[k], S, c, o);
                    dot[k] = re_dot3<R>(pv, o);
                }
            }
        }
    }
    if (EPI == EPI_M_PAP || EPI == EPI_RESID) {
        double tot[K];
        if (group_sum<BLOCK, K>(dot, G.K, G.partial, lblk, G.nblocks, &a.tickets[gi], smem, tot) &&
            threadIdx.x == 0) {
            for (int k = 0; k < G.K; k++) {
                if (!act[k])
                    continue;
                CgScalars &sc = a.sys[G.sys0 + k];
                if (EPI == EPI_RESID) {
                    sc.true_rr = tot[k];
                } else {
                    sc.pAp = tot[k];
                    if (!(tot[k] > 0.0 && tot[k] < INFINITY))
                        sc.status = CG_BREAKDOWN;
                    sc.alpha = make_dpair(sc.status == CG_RUNNING ? sc.rr / tot[k] : 0.0);
                }
            }
        }
    }
}

// the epilogue of system k at site c of a lane-mapped Dslash: store D psi
// (EPI_NONE), or m_k^2 p_k - D psi and its share of <p_k, Ap_k> (EPI_M_PAP),
// or the share of |b_k - M x_k|^2 (EPI_RESID)
template <int P, int EPI>
STAG_D red_t<typename Fmt<P>::R> batch_lane_epilogue(const BatchArgs &a, const BatchGroup &G, int k, int c,
                                                      cplx<typename Fmt<P>::R> acc[3]) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    const int S = G.g.stride;
    red_t<R> dk = red_zero<red_t<R>>();
    if (EPI == EPI_NONE) {
#pragma unroll
        for (int r = 0; r < 3; r++) {
            acc[r].re = rnorm<R>(acc[r].re);
            acc[r].im = rnorm<R>(acc[r].im);
        }
        store_vec<P>((E *)G.t[k], S, c, acc);
    } else {
        const R m2 = scalar_as<R>(a.sys[G.sys0 + k].m2);
        cplx<R> pv[3], o[3];
        load_vec<P>((const E *)(EPI == EPI_RESID ? G.x[k] : G.p[k]), S, c, pv);
#pragma unroll
        for (int r = 0; r < 3; r++) {
            o[r] = cneg(acc[r]);
            mac(o[r].re, m2, pv[r].re);
            mac(o[r].im, m2, pv[r].im);
            o[r].re = rnorm<R>(o[r].re);
            o[r].im = rnorm<R>(o[r].im);
        }
        if (EPI == EPI_RESID) {
            cplx<R> bv[3];
            load_vec<P>((const E *)G.b[k], S, c, bv);
#pragma unroll
            for (int r = 0; r < 3; r++) {
                o[r].re = rsub(bv[r].re, o[r].re);
                o[r].im = rsub(bv[r].im, o[r].im);
            }
            dk = re_dot3<R>(o, o);
        } else {
            store_vec<P>((E *)G.Ap[k], S, c, o);
            dk = re_dot3<R>(pv, o);
        }
    }
    return dk;
}

// the group's sums of a lane-mapped Dslash and what its last block makes of
// them: alpha_k (EPI_M_PAP) or the true residual (EPI_RESID)
template <int EPI, int BLOCK, int K, class T>
STAG_D void batch_lane_reduce(const BatchArgs &a, int gi, const BatchGroup &G, const int *act, int lblk,
                              const T (&dot)[K], double *smem) {
    if (EPI == EPI_M_PAP || EPI == EPI_RESID) {
        double tot[K];
        if (group_sum<BLOCK, K>(dot, G.K, G.partial, lblk, G.dnblocks, &a.tickets[gi], smem, tot) &&
            threadIdx.x == 0) {
            for (int kk = 0; kk < G.K; kk++) {
                if (!act[kk])
                    continue;
                CgScalars &sc = a.sys[G.sys0 + kk];
                if (EPI == EPI_RESID) {
                    sc.true_rr = tot[kk];
                } else {
                    sc.pAp = tot[kk];
                    if (!(tot[kk] > 0.0 && tot[kk] < INFINITY))
                        sc.status = CG_BREAKDOWN;
                    sc.alpha = make_dpair(sc.status == CG_RUNNING ? sc.rr / tot[kk] : 0.0);
                }
            }
        }
    }
}

// the vector a lane-mapped Dslash reads for system k: D_oe of p (or of x
// for the true residual), or D_eo of the odd t
template <int EPI>
STAG_D const void *batch_lane_input(const BatchGroup &G, int k, int src_x) {
    return EPI == EPI_NONE ? (src_x ? G.x[k] : G.p[k]) : G.t[k];
}

// Lane-mapped multi-RHS Dslash (double-float and FP64): thread t of the
// group's range handles site t / GK for system t % GK (GK = systems in the
// group), with the single-site stencil; epilogues as batch_dslash_kernel.
template <int P, int EPI, int BLOCK, int K>
__global__ void __launch_bounds__(BLOCK) batch_dslash_lanes_kernel(BatchArgs a, int out_par, int src_x) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    __shared__ double smem[32];
    __shared__ int act[K];
    const int gi = group_of_lanes(a, blockIdx.x);
    const BatchGroup &G = a.grp[gi];
    load_active<K>(a, G, act, EPI != EPI_RESID && !src_x);
    const int lblk = blockIdx.x - G.dblock0;
    const int t = lblk * BLOCK + threadIdx.x;
    const int k = t % G.K;
    const int c = t / G.K;
    const Geom &g = G.g;
    red_t<R> dot[K];
#pragma unroll
    for (int kk = 0; kk < K; kk++)
        dot[kk] = red_zero<red_t<R>>();
    if (c < g.Vh && act[k]) {
        DslashArgs da = {};
        da.link_scale[0] = G.link_scale[0];
        da.link_scale[1] = G.link_scale[1];
        cplx<R> acc[3] = {czero<R>(), czero<R>(), czero<R>()};
        dslash_site<P, 0>(g, out_par, c, G.links[out_par], G.links[1 - out_par],
                              (const E *)batch_lane_input<EPI>(G, k, src_x), da, acc);
        const red_t<R> dk = batch_lane_epilogue<P, EPI>(a, G, k, c, acc);
#pragma unroll
        for (int kk = 0; kk < K; kk++)
            if (kk == k)
                dot[kk] = dk;
    }
    batch_lane_reduce<EPI, BLOCK, K>(a, gi, G, act, lblk, dot, smem);
}

// x = 0, r = b, p = b, |b|^2 per system
template <int P, int BLOCK, int K>
__global__ void __launch_bounds__(BLOCK) batch_init_kernel(BatchArgs a) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    __shared__ double smem[32];
    const int gi = group_of(a, blockIdx.x);
    const BatchGroup &G = a.grp[gi];
    const int lblk = blockIdx.x - G.block0;
    const int c = lblk * BLOCK + threadIdx.x;
    const int S = G.g.stride;
    red_t<R> dot[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        dot[k] = red_zero<red_t<R>>();
        if (k < G.K && c < G.g.Vh) {
            cplx<R> bv[3], z[3];
            load_vec<P>((const E *)G.b[k], S, c, bv);
#pragma unroll
            for (int r = 0; r < 3; r++)
                z[r] = czero<R>();
            store_vec<P>((E *)G.x[k], S, c, z);
            store_vec<P>((E *)G.r[k], S, c, bv);
            store_vec<P>((E *)G.p[k], S, c, bv);
            dot[k] = re_dot3<R>(bv, bv);
        }
    }
    double tot[K];
    if (group_sum<BLOCK, K>(dot, G.K, G.partial, lblk, G.nblocks, &a.tickets[gi], smem, tot)) {
        if (threadIdx.x == 0) {
            int running = 0;
            for (int k = 0; k < G.K; k++) {
                CgScalars &sc = a.sys[G.sys0 + k];
                sc.bb = tot[k];
                sc.rr = tot[k];
                sc.true_rr = tot[k];
                sc.rr_stop = sc.tol2 * tot[k];
                sc.iter = 0;
                sc.alpha = make_dpair(0.0);
                sc.beta = make_dpair(0.0);
                if (!(tot[k] < INFINITY))
                    sc.status = CG_BREAKDOWN;
                else if (tot[k] <= sc.rr_stop)
                    sc.status = CG_CONVERGED;
                else if (sc.max_iter <= 0)
                    sc.status = CG_MAXITER;
                else
                    sc.status = CG_RUNNING;
                sc.pad2 = sc.status == CG_RUNNING ? 0 : 1;  // not running: never counted
                running += sc.status == CG_RUNNING;
            }
            atomicAdd(&a.ctl->running, running);
            batch_finish_group(a);
        }
    }
}

// x += alpha p, r -= alpha Ap, |r|^2 -> beta and stopping, per system
template <int P, int BLOCK, int K>
__global__ void __launch_bounds__(BLOCK) batch_update_kernel(BatchArgs a) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    __shared__ double smem[32];
    __shared__ int act[K];
    const int gi = group_of(a, blockIdx.x);
    const BatchGroup &G = a.grp[gi];
    load_active<K>(a, G, act, true);
    const int lblk = blockIdx.x - G.block0;
    const int c = lblk * BLOCK + threadIdx.x;
    const int S = G.g.stride;
    red_t<R> dot[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        dot[k] = red_zero<red_t<R>>();
        if (act[k] && c < G.g.Vh) {
            const R alpha = scalar_as<R>(a.sys[G.sys0 + k].alpha);
            const R malpha = -alpha;
            cplx<R> xv[3], rv[3], pv[3], av[3];
            load_vec<P>((const E *)G.x[k], S, c, xv);
            load_vec<P>((const E *)G.r[k], S, c, rv);
            load_vec<P>((const E *)G.p[k], S, c, pv);
            load_vec<P>((const E *)G.Ap[k], S, c, av);
#pragma unroll
            for (int r = 0; r < 3; r++) {
                mac(xv[r].re, alpha, pv[r].re);
                mac(xv[r].im, alpha, pv[r].im);
                mac(rv[r].re, malpha, av[r].re);
                mac(rv[r].im, malpha, av[r].im);
                xv[r].re = rnorm<R>(xv[r].re);
                xv[r].im = rnorm<R>(xv[r].im);
                rv[r].re = rnorm<R>(rv[r].re);
                rv[r].im = rnorm<R>(rv[r].im);
            }
            store_vec<P>((E *)G.x[k], S, c, xv);
            store_vec<P>((E *)G.r[k], S, c, rv);
            dot[k] = re_dot3<R>(rv, rv);
        }
    }
    double tot[K];
    if (group_sum<BLOCK, K>(dot, G.K, G.partial, lblk, G.nblocks, &a.tickets[gi], smem, tot)) {
        if (threadIdx.x == 0) {
            int stopped = 0;
            for (int k = 0; k < G.K; k++) {
                CgScalars &sc = a.sys[G.sys0 + k];
                if (!act[k]) {
                    // stopped earlier (counted then), or broke down in this
                    // iteration's M: count it once (pad2 marks "counted")
                    if (sc.status != CG_RUNNING && sc.pad2 == 0) {
                        sc.pad2 = 1;
                        stopped++;
                    }
                    continue;
                }
                const double beta = tot[k] / sc.rr;
                sc.beta = make_dpair(beta);
                sc.rr = tot[k];
                sc.iter += 1;
                if (!(tot[k] < INFINITY))
                    sc.status = CG_BREAKDOWN;
                else if (tot[k] <= sc.rr_stop)
                    sc.status = CG_CONVERGED;
                else if (sc.iter >= sc.max_iter)
                    sc.status = CG_MAXITER;
                if (sc.status != CG_RUNNING) {
                    sc.pad2 = 1;
                    stopped++;
                }
            }
            if (stopped)
                atomicSub(&a.ctl->running, stopped);
            batch_finish_group(a);
        }
    }
}

// p = r + beta p per running system
template <int P, int BLOCK, int K>
__global__ void __launch_bounds__(BLOCK) batch_p_kernel(BatchArgs a) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    __shared__ int act[K];
    const int gi = group_of(a, blockIdx.x);
    const BatchGroup &G = a.grp[gi];
    load_active<K>(a, G, act, true);
    const int c = (blockIdx.x - G.block0) * BLOCK + threadIdx.x;
    if (c >= G.g.Vh)
        return;
    const int S = G.g.stride;
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (!act[k])
            continue;
        const R beta = scalar_as<R>(a.sys[G.sys0 + k].beta);
        cplx<R> rv[3], pv[3];
        load_vec<P>((const E *)G.r[k], S, c, rv);
        load_vec<P>((const E *)G.p[k], S, c, pv);
#pragma unroll
        for (int r = 0; r < 3; r++) {
            mac(rv[r].re, beta, pv[r].re);
            mac(rv[r].im, beta, pv[r].im);
            rv[r].re = rnorm<R>(rv[r].re);
            rv[r].im = rnorm<R>(rv[r].im);
        }
        store_vec<P>((E *)G.p[k], S, c, rv);
    }
}

// one launch of kernel `what` for groups of at most K right-hand sides
template <int P, int BLOCK, int K>
cudaError_t launch_batch_pbk(int what, const BatchArgs &a, cudaStream_t s) {
    const int grid = a.nblocks;
    if constexpr (P != P_F32) {
        const int dgrid = a.dnblocks;
        switch (what) {
        case BATCH_DSLASH_OE: batch_dslash_lanes_kernel<P, EPI_NONE, BLOCK, K><<<dgrid, BLOCK, 0, s>>>(a, 1, 0); return cudaGetLastError();
        case BATCH_DSLASH_X: batch_dslash_lanes_kernel<P, EPI_NONE, BLOCK, K><<<dgrid, BLOCK, 0, s>>>(a, 1, 1); return cudaGetLastError();
        case BATCH_M_PAP: batch_dslash_lanes_kernel<P, EPI_M_PAP, BLOCK, K><<<dgrid, BLOCK, 0, s>>>(a, 0, 0); return cudaGetLastError();
        case BATCH_RESID: batch_dslash_lanes_kernel<P, EPI_RESID, BLOCK, K><<<dgrid, BLOCK, 0, s>>>(a, 0, 0); return cudaGetLastError();
        default: break;
        }
    }
    switch (what) {
    case BATCH_INIT: batch_init_kernel<P, BLOCK, K><<<grid, BLOCK, 0, s>>>(a); break;
    case BATCH_DSLASH_OE: batch_dslash_kernel<P, EPI_NONE, BLOCK, K><<<grid, BLOCK, 0, s>>>(a, 1, 0); break;
    case BATCH_DSLASH_X: batch_dslash_kernel<P, EPI_NONE, BLOCK, K><<<grid, BLOCK, 0, s>>>(a, 1, 1); break;
    case BATCH_M_PAP: batch_dslash_kernel<P, EPI_M_PAP, BLOCK, K><<<grid, BLOCK, 0, s>>>(a, 0, 0); break;
    case BATCH_RESID: batch_dslash_kernel<P, EPI_RESID, BLOCK, K><<<grid, BLOCK, 0, s>>>(a, 0, 0); break;
    case BATCH_UPDATE: batch_update_kernel<P, BLOCK, K><<<grid, BLOCK, 0, s>>>(a); break;
    case BATCH_P: batch_p_kernel<P, BLOCK, K><<<grid, BLOCK, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace stag
