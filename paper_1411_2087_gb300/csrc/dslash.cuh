// The improved-staggered Dslash stencil (the paper's Sec. 3 operation):
// for each output site x of one checkerboard,
//
//   out(x) = sum_mu [ U~_mu(x) psi(x+mu)  - U~_mu(x-mu)^+  psi(x-mu)
//                   + N~_mu(x) psi(x+3mu) - N~_mu(x-3mu)^+ psi(x-3mu) ]
//
// with U~, N~ the links with c1/c3, the Kogut-Susskind phases and the
// boundary signs folded in at upload (so the stencil itself has no signs
// beyond the minus of the backward hops).  One thread per output site; the
// 16 link matrices stream from HBM with evict-first loads, the 16 neighbour
// vectors come through L1/L2.
#pragma once
#include "cg_state.cuh"
#include "fields.cuh"
#include "reduce.cuh"

namespace stag {

// epilogues fused into the stencil
enum Epi {
    EPI_NONE = 0,   // out = D in
    EPI_M = 1,      // out = m^2 p - D in                (M p with in = D_oe p)
    EPI_M_PAP = 2,  // as EPI_M, plus <p, out> -> alpha = rr / <p, M p>
    EPI_RESID = 3,  // r = b - (m^2 p - D in), |r|^2 -> true residual (r not stored)
    EPI_RESID_STORE = 4  // as EPI_RESID, and r stored to out
};

struct DslashArgs {
    Geom g;
    int out_par;
    const void *links_out;  // links on sites of the output parity: [8][9][stride]
    const void *links_in;   // links on sites of the input parity
    const void *in;         // input vector, other parity
    void *out;              // output vector
    const void *p;          // EPI_M*: the even vector M acts on
    const void *b;          // EPI_RESID: right-hand side
    double *partial;        // per-block partial sums
    CgScalars *sc;          // device scalars (m2, rr, alpha, ...)
    dpair m2;               // EPI_M: m^2 when m2_in_args, else read from sc
    int m2_in_args;
    int skip_if_done;       // return at once when sc->status is no longer CG_RUNNING
    const int *gate;        // if set, return at once unless *gate != 0 (uniform flag)
    float link_scale[2];    // 16-bit links: value = q * scale (one-link, three-link)
};

// acc += D psi at checkerboard site c of parity par
template <int P>
STAG_D void dslash_site(const Geom &g, int par, int c,
                        const typename Fmt<P>::Elem *__restrict__ Gout,
                        const typename Fmt<P>::Elem *__restrict__ Gin,
                        const typename Fmt<P>::Elem *__restrict__ in,
                        const float link_scale[2], cplx<typename Fmt<P>::R> acc[3]) {
    using F = Fmt<P>;
    using R = typename F::R;
    const int S = g.stride;
    int x[4];
    cb_coords(g, c, par, x);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int s = h ? 3 : 1;
            const int kind = 4 * h + mu;
            const float ls = link_scale[h];
            // forward: + L(x) psi(x + s mu)
            {
                const int j = cb_hop(g, c, x, mu, +s);
                cplx<R> v[3];
                load_vec<P>(in, S, j, v);
                const typename F::Elem *Lp = Gout + kind * 9 * S + c;
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++)
                        cmac(acc[a], F::unpack_link(ld_stream(Lp + (3 * a + b) * S), ls), v[b]);
            }
            // backward: - L(x - s mu)^+ psi(x - s mu)
            {
                const int j = cb_hop(g, c, x, mu, -s);
                cplx<R> v[3];
                load_vec<P>(in, S, j, v);
#pragma unroll
                for (int b = 0; b < 3; b++)
                    v[b] = cneg(v[b]);
                const typename F::Elem *Lp = Gin + kind * 9 * S + j;
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++)
                        cmac_conj(acc[a], F::unpack_link(ld_stream(Lp + (3 * b + a) * S), ls), v[b]);
            }
        }
    }
}

template <class R> STAG_D double re_dot3(const cplx<R> a[3], const cplx<R> b[3]) {
    R s = rzero<R>();
#pragma unroll
    for (int k = 0; k < 3; k++) {
        mac(s, a[k].re, b[k].re);
        mac(s, a[k].im, b[k].im);
    }
    return to_double<R>(rnorm<R>(s));
}

template <int P, int EPI, int BLOCK>
__global__ void __launch_bounds__(BLOCK) dslash_kernel(DslashArgs a) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    __shared__ double smem[32];
    // the status is uniform over the grid: either every block returns here or none
    if (a.skip_if_done && a.sc->status != CG_RUNNING)
        return;
    if (a.gate && *a.gate == 0)
        return;
    const int c = blockIdx.x * BLOCK + threadIdx.x;
    const int S = a.g.stride;
    double dot = 0.0;
    if (c < a.g.Vh) {
        cplx<R> acc[3] = {czero<R>(), czero<R>(), czero<R>()};
        dslash_site<P>(a.g, a.out_par, c, (const E *)a.links_out, (const E *)a.links_in,
                       (const E *)a.in, a.link_scale, acc);
        if (EPI == EPI_NONE) {
#pragma unroll
            for (int k = 0; k < 3; k++) {
                acc[k].re = rnorm<R>(acc[k].re);
                acc[k].im = rnorm<R>(acc[k].im);
            }
            store_vec<P>((E *)a.out, S, c, acc);
        } else {
            const R m2 = scalar_as<R>(a.m2_in_args ? a.m2 : a.sc->m2);
            cplx<R> p[3], o[3];
            load_vec<P>((const E *)a.p, S, c, p);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                o[k] = cneg(acc[k]);
                mac(o[k].re, m2, p[k].re);
                mac(o[k].im, m2, p[k].im);
                o[k].re = rnorm<R>(o[k].re);
                o[k].im = rnorm<R>(o[k].im);
            }
            if (EPI == EPI_RESID || EPI == EPI_RESID_STORE) {
                cplx<R> bb[3];
                load_vec<P>((const E *)a.b, S, c, bb);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    o[k].re = rsub(bb[k].re, o[k].re);
                    o[k].im = rsub(bb[k].im, o[k].im);
                }
                dot = re_dot3<R>(o, o);
                if (EPI == EPI_RESID_STORE)
                    store_vec<P>((E *)a.out, S, c, o);
            } else {
                store_vec<P>((E *)a.out, S, c, o);
                if (EPI == EPI_M_PAP)
                    dot = re_dot3<R>(p, o);
            }
        }
    }
    if (EPI == EPI_M_PAP || EPI == EPI_RESID || EPI == EPI_RESID_STORE) {
        double total;
        if (grid_sum<BLOCK>(dot, a.partial, &a.sc->ticket, smem, total) && threadIdx.x == 0) {
            CgScalars *sc = a.sc;
            if (EPI == EPI_M_PAP) {
                sc->pAp = total;
                if (sc->status == CG_RUNNING && !(total > 0.0 && total < INFINITY))
                    sc->status = CG_BREAKDOWN;
                sc->alpha = make_dpair(sc->status == CG_RUNNING ? sc->rr / total : 0.0);
            } else {
                sc->true_rr = total;
            }
        }
    }
}

}  // namespace stag
