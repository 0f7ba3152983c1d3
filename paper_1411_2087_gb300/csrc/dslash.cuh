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
    EPI_RESID_STORE = 4, // as EPI_RESID, and r stored to out
    EPI_M_PART = 5  // as EPI_M, plus one partial of <p, out> per block (summed by pap_finish)
};

struct DslashArgs {
    Geom g;
    int out_par;
    const void *links_out;  // links on sites of the output parity: 8 kinds (link_kind_offset)
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
    int compressed;         // compression mask (link_kind_offset): 12-real one-link (bit 0), three-link (bit 1)
    int c0, cn;             // output sites c0 .. c0+cn-1 (cn = 0: all Vh)
    int c0b, cnb;           // with cn > 0: also sites c0b .. c0b+cnb-1 (cnb = 0: none)
    float inv_c[2];         // 1/c1, 1/c3: the reconstruction divides by s = c eta b
    int bc_neg[4];          // boundary sign of direction mu is -1
    int regs;               // EPI_NONE, EPI_M_PART: REGS_* (autotuned)
};

// register variant of the stencil (DslashArgs::regs): the launcher's
// measured default, the compiler's free choice, at most 64 registers, or
// (16-bit stencil, EPI_NONE and EPI_M_PART) two sites per thread in packed
// FP32x2 arithmetic with the loads through a shared-memory ring
// (stencil16_pair_async) where pair16_applies, else the default
enum { REGS_DEFAULT = 0, REGS_FREE = 1, REGS_CAPPED = 2, REGS_PAIR = 3 };

// rebuild row 2 of L = s U (U in SU(3)) from rows 0 and 1: conj(r0 x r1) / s
template <class R>
STAG_D void reconstruct_row2(cplx<R> L[9], float inv_s) {
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        // r0_k r1_l - r0_l r1_k
        const float re = L[k].re * L[3 + l].re - L[k].im * L[3 + l].im - (L[l].re * L[3 + k].re - L[l].im * L[3 + k].im);
        const float im = L[k].re * L[3 + l].im + L[k].im * L[3 + l].re - (L[l].re * L[3 + k].im + L[l].im * L[3 + k].re);
        L[6 + j] = cplx<R>{re * inv_s, -im * inv_s};
    }
}

// number of times a hop of s steps from coordinate v wraps (L >= 2, |s| <= 3)
STAG_HD int hop_wraps(int v, int s, int L) {
    int y = v + s, w = 0;
    if (y >= L) { y -= L; w++; }
    if (y >= L) { y -= L; w++; }
    if (y < 0) { y += L; w++; }
    if (y < 0) { y += L; w++; }
    return w;
}

// the nine entries of one link of kind `kind` (compression mask CM): either
// stored whole, or rows 0 and 1 of the 12-real layout with row 2 rebuilt
// (inv_s = 1/(c eta b) of that link)
template <int P, int CM>
STAG_D void load_link(const void *G, int kind, int S, int idx, float ls, float inv_s,
                      cplx<typename Fmt<P>::R> L[9]) {
    using F = Fmt<P>;
    using E = typename F::Elem;
    const E *Lp;
    if constexpr (CM != 0) {
        const char *kb = (const char *)G + link_kind_offset(P, CM, kind, (size_t)S);
        if ((CM >> (kind >> 2)) & 1) {
            C12<P>::load(kb, S, idx, ls, L);
            reconstruct_row2(L, inv_s);
            return;
        }
        Lp = (const E *)kb + idx;
    } else {
        // all kinds full: a 32-bit element offset (72 planes of one parity
        // fit, the lattice checks it).  With the 64-bit byte offset the
        // compiler kept the sixteen links' addresses live and the
        // double-float stencil grew from 80 to 116 registers.
        Lp = (const E *)G + (kind * 9 * S + idx);
    }
#pragma unroll
    for (int e = 0; e < 9; e++)
        L[e] = F::unpack_link(ld_stream(Lp + e * S), ls);
}

}  // namespace stag

#include "stencil16.cuh"

namespace stag {

// acc += D psi at checkerboard site c of parity par (links with compression
// mask CM)
template <int P, int CM = 0>
STAG_D void dslash_site(const Geom &g, int par, int c, const void *__restrict__ Gout,
                        const void *__restrict__ Gin, const typename Fmt<P>::Elem *__restrict__ in,
                        const DslashArgs &a, cplx<typename Fmt<P>::R> acc[3]) {
    using R = typename Fmt<P>::R;
    if constexpr (P == P_F16) {
        // raw integer units (stencil16.cuh)
        stencil16_site<CM>(g, par, c, Gout, Gin, in, a, acc);
        return;
    }
    const int S = g.stride;
    int x[4];
    cb_coords(g, c, par, x);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        // Kogut-Susskind phase of direction mu at x (equal at x - s mu)
        int esum = 0;
#pragma unroll
        for (int nu = 0; nu < mu; nu++)
            esum += x[nu];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int s = h ? 3 : 1;
            const int kind = 4 * h + mu;
            const float ls = a.link_scale[h];
            // forward: + L(x) psi(x + s mu)
            {
                const int j = cb_hop(g, c, x, mu, +s);
                cplx<R> v[3];
                load_vec<P>(in, S, j, v);
                float inv_s = 0.f;
                if ((CM >> h) & 1) {
                    const int flip = (esum + (a.bc_neg[mu] ? hop_wraps(x[mu], s, g.L[mu]) : 0)) & 1;
                    inv_s = flip ? -a.inv_c[h] : a.inv_c[h];
                }
                cplx<R> L[9];
                load_link<P, CM>(Gout, kind, S, c, ls, inv_s, L);
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int b = 0; b < 3; b++)
                        cmac(acc[r], L[3 * r + b], v[b]);
            }
            // backward: - L(x - s mu)^+ psi(x - s mu)
            {
                const int j = cb_hop(g, c, x, mu, -s);
                cplx<R> v[3];
                load_vec<P>(in, S, j, v);
#pragma unroll
                for (int b = 0; b < 3; b++)
                    v[b] = cneg(v[b]);
                float inv_s = 0.f;
                if ((CM >> h) & 1) {
                    const int flip = (esum + (a.bc_neg[mu] ? hop_wraps(x[mu], -s, g.L[mu]) : 0)) & 1;
                    inv_s = flip ? -a.inv_c[h] : a.inv_c[h];
                }
                cplx<R> L[9];
                load_link<P, CM>(Gin, kind, S, j, ls, inv_s, L);
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int b = 0; b < 3; b++)
                        cmac_conj(acc[r], L[3 * b + r], v[b]);
            }
        }
    }
}

// Re <a, b> of one site, in the reduction type of R (FP64 for FP64, else
// double-float: exact for an FP32 sum, the double-float sum itself for DF64)
STAG_D double to_red(double s) { return s; }
STAG_D df to_red(float s) { return df_make(s, 0.f); }
STAG_D df to_red(df s) { return df_norm(s); }

template <class R> STAG_D red_t<R> re_dot3(const cplx<R> a[3], const cplx<R> b[3]) {
    R s = rzero<R>();
#pragma unroll
    for (int k = 0; k < 3; k++) {
        mac(s, a[k].re, b[k].re);
        mac(s, a[k].im, b[k].im);
    }
    return to_red(s);
}

// the epilogue of output site c: store D psi (EPI_NONE) or o = m^2 p - D psi
// (and for the residual forms b - o); returns the site's share of the sum
// the epilogue reduces (<p, o> or |b - o|^2)
template <int P, int EPI>
STAG_D red_t<typename Fmt<P>::R> dslash_epilogue(const DslashArgs &a, int c, cplx<typename Fmt<P>::R> acc[3]) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    const int S = a.g.stride;
    red_t<R> dot = red_zero<red_t<R>>();
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
            if (EPI == EPI_M_PAP || EPI == EPI_M_PART)
                dot = re_dot3<R>(p, o);
        }
    }
    return dot;
}

// the block's (EPI_M_PART) or the grid's (EPI_M_PAP, EPI_RESID*) sum of the
// sites' shares, and what the epilogue makes of it
template <int EPI, int BLOCK, class T>
STAG_D void dslash_reduce(const DslashArgs &a, T dot, double *smem) {
    if (EPI == EPI_M_PART) {
        // no ticket: the block's partial is all this kernel contributes
        const double s = block_sum<BLOCK>(dot, smem);
        if (threadIdx.x == 0)
            a.partial[blockIdx.x] = s;
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

template <int P, int EPI, int BLOCK, int CM>
STAG_D void dslash_body(const DslashArgs &a) {
    using F = Fmt<P>;
    using R = typename F::R;
    using E = typename F::Elem;
    __shared__ double smem[32];
    // the status is uniform over the grid: either every block returns here or none
    if (a.skip_if_done && a.sc->status != CG_RUNNING)
        return;
    if (a.gate && *a.gate == 0)
        return;
    // site i of the launch: the range c0.., then the second range c0b..
    const int i = blockIdx.x * BLOCK + threadIdx.x;
    const int n1 = a.cn ? a.cn : a.g.Vh;
    const int n2 = a.cn ? a.cnb : 0;
    const int c = i < n1 ? a.c0 + i : a.c0b + (i - n1);
    red_t<R> dot = red_zero<red_t<R>>();
    if (i < n1 + n2) {
        cplx<R> acc[3] = {czero<R>(), czero<R>(), czero<R>()};
        dslash_site<P, CM>(a.g, a.out_par, c, a.links_out, a.links_in, (const E *)a.in, a, acc);
        dot = dslash_epilogue<P, EPI>(a, c, acc);
    }
    dslash_reduce<EPI, BLOCK>(a, dot, smem);
}

// The compressed 16-bit stencil on the pair (c, c + Vh/2) per thread
// (stencil16_pair_async: all Vh sites, Lt a multiple of 4 and at least 8);
// block partials of EPI_M_PART cover both sites of each thread.
template <int EPI, int BLOCK, int CM>
STAG_D void pair16_body(const DslashArgs &a) {
    __shared__ double smem[32];
    __shared__ int4 ring[pair16_ring<BLOCK, CM>() * pair16_cells<CM>() * BLOCK];
    if (a.skip_if_done && a.sc->status != CG_RUNNING)
        return;
    if (a.gate && *a.gate == 0)
        return;
    const int H = a.g.Vh >> 1;
    const int c = blockIdx.x * BLOCK + threadIdx.x;
    df dot = df_zero();
    if (c < H) {
        cplx<float2> acc[3];
#pragma unroll
        for (int k = 0; k < 3; k++)
            acc[k] = cplx<float2>{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        stencil16_pair_async<BLOCK, pair16_ring<BLOCK, CM>(), CM>(a.g, a.out_par, c, a.links_out, a.links_in,
                                                                  (const short2 *)a.in, a, ring, acc);
        cplx<float> lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            lo[k] = cplx<float>{acc[k].re.x, acc[k].im.x};
            hi[k] = cplx<float>{acc[k].re.y, acc[k].im.y};
        }
        dot = dslash_epilogue<P_F16, EPI>(a, c, lo);
        dot = red_add(dot, dslash_epilogue<P_F16, EPI>(a, c + H, hi));
    }
    dslash_reduce<EPI, BLOCK>(a, dot, smem);
}

// One launch of the stencil.  The capped form asks for at least 1024 resident
// threads per SM (at most 64 registers).  Left free, the compiler gives the
// uncompressed FP32 kernels so few registers (32-44) that too few loads are
// in flight; the launcher picks the capped form for those and for the
// 16-bit ones (kCapped) and the free one for the rest.
template <int P, int EPI, int BLOCK, int CM = 0>
__global__ void __launch_bounds__(BLOCK) dslash_kernel(DslashArgs a) {
    dslash_body<P, EPI, BLOCK, CM>(a);
}

template <int P, int EPI, int BLOCK, int CM>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) dslash_kernel_capped(DslashArgs a) {
    dslash_body<P, EPI, BLOCK, CM>(a);
}

// whether a launch of precision prec and epilogue epi runs the pair form
STAG_HD bool pair16_used(int prec, int epi, const DslashArgs &a) {
    return prec == P_F16 && a.regs == REGS_PAIR &&
           (epi == EPI_NONE || epi == EPI_M_PART) &&
           a.c0 == 0 && (a.cn == 0 || a.cn == a.g.Vh) && a.cnb == 0 && pair16_applies(a.g);
}
STAG_HD int dslash_pair16_grid(const Geom &g, int block) { return ((g.Vh >> 1) + block - 1) / block; }

// the pair form (REGS_PAIR): at least 768 resident threads per SM, at most
// 85 registers (80 used).  At 48^3x96 this measured 351 us against 381-417
// us with 640 threads and 96 registers (rings of 2 or 4 hops) and 386 us
// with 512 threads and 124 registers.
template <int EPI, int BLOCK, int CM>
__global__ void __launch_bounds__(BLOCK, (768 / BLOCK > 0 ? 768 / BLOCK : 1)) dslash_pair16_kernel(DslashArgs a) {
    pair16_body<EPI, BLOCK, CM>(a);
}

}  // namespace stag
