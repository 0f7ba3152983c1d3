// The 16-bit stencil (16-bit links and colour vectors) in raw integer
// units, written once over a lane type V:
//
//   V = float    one output site per thread
//   V = float2   two output sites per thread, the pair (x, y, z, t) and
//                (x, y, z, t + Lt/2), in Blackwell's packed FP32x2
//                arithmetic (one FFMA2 does the same multiply-add on both)
//
// Both forms run the same IEEE operations in the same order on every lane,
// so they give the same bits.  In the pair form the two sites share their
// coordinates, every x/y/z hop offset and every Kogut-Susskind and boundary
// sign; only the t hops differ (one site of the pair can wrap forward, the
// other backward).  This halves the floating-point instructions per site
// and removes half of the index arithmetic, the two costs that keep the
// one-site form below the memory roof.
//
// Each group of links (one-link, three-link) is either full (nine entries)
// or 12-real, as the compression mask CM says (link_kind_offset).
//
// Units: a link entry is ls q (ls the field's scale), a vector component
// (n / 32767) q (n the site's norm), q the stored integers.  Of a 12-real
// link rows 0 and 1 are stored; with X = row0 x row1 (raw), row 2 of the
// link is conj(X) ls / s (s = c eta b of that link), which the hop's
// coefficients carry.
#pragma once
#include "fields.cuh"

namespace stag {

STAG_D float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
STAG_D float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
STAG_D float vmul(float a, float b) { return __fmul_rn(a, b); }
STAG_D float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
STAG_D float vneg(float a) { return -a; }
STAG_D float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
template <class V> STAG_D V vsplat(float s);
template <> STAG_D float vsplat<float>(float s) { return s; }
template <> STAG_D float2 vsplat<float2>(float s) { return make_float2(s, s); }

// X = row0 x row1 of the raw link (L[0..2] row 0, L[3..5] row 1)
template <class V>
STAG_D void cross01(const cplx<V> L[6], cplx<V> X[3]) {
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        const cplx<V> &ak = L[k], &al = L[l], &bk = L[3 + k], &bl = L[3 + l];
        // ak bl - al bk
        V re = vmul(ak.re, bl.re);
        re = vfma(vneg(ak.im), bl.im, re);
        re = vfma(vneg(al.re), bk.re, re);
        re = vfma(al.im, bk.im, re);
        V im = vmul(ak.re, bl.im);
        im = vfma(ak.im, bl.re, im);
        im = vfma(vneg(al.re), bk.im, im);
        im = vfma(vneg(al.im), bk.re, im);
        X[j] = cplx<V>{re, im};
    }
}

// forward hop: acc_r += cf (L v)_r for rows 0, 1 and acc_2 += cf2 (conj(X) . v)
template <class V>
STAG_D void hop_fwd16(cplx<V> acc[3], const cplx<V> L[6], const cplx<V> v[3], V cf, V cf2) {
#pragma unroll
    for (int r = 0; r < 2; r++) {
        V tr = vmul(L[3 * r].re, v[0].re);
        tr = vfma(vneg(L[3 * r].im), v[0].im, tr);
        V ti = vmul(L[3 * r].re, v[0].im);
        ti = vfma(L[3 * r].im, v[0].re, ti);
#pragma unroll
        for (int b = 1; b < 3; b++) {
            tr = vfma(L[3 * r + b].re, v[b].re, tr);
            tr = vfma(vneg(L[3 * r + b].im), v[b].im, tr);
            ti = vfma(L[3 * r + b].re, v[b].im, ti);
            ti = vfma(L[3 * r + b].im, v[b].re, ti);
        }
        acc[r].re = vfma(cf, tr, acc[r].re);
        acc[r].im = vfma(cf, ti, acc[r].im);
    }
    cplx<V> X[3];
    cross01(L, X);
    V tr = vmul(X[0].re, v[0].re);
    tr = vfma(X[0].im, v[0].im, tr);
    V ti = vmul(X[0].re, v[0].im);
    ti = vfma(vneg(X[0].im), v[0].re, ti);
#pragma unroll
    for (int b = 1; b < 3; b++) {
        tr = vfma(X[b].re, v[b].re, tr);
        tr = vfma(X[b].im, v[b].im, tr);
        ti = vfma(X[b].re, v[b].im, ti);
        ti = vfma(vneg(X[b].im), v[b].re, ti);
    }
    acc[2].re = vfma(cf2, tr, acc[2].re);
    acc[2].im = vfma(cf2, ti, acc[2].im);
}

// backward hop: acc_r += cf (L^+ v)_r, with L^+ v = sum_b conj(L_br) v_b and
// conj(L_2r) = X_r k2 (k2 = ls / s of the link)
template <class V>
STAG_D void hop_bwd16(cplx<V> acc[3], const cplx<V> L[6], const cplx<V> v[3], V cf, V k2) {
    cplx<V> X[3];
    cross01(L, X);
    const cplx<V> w = {vmul(v[2].re, k2), vmul(v[2].im, k2)};
#pragma unroll
    for (int r = 0; r < 3; r++) {
        V tr = vmul(L[r].re, v[0].re);
        tr = vfma(L[r].im, v[0].im, tr);
        tr = vfma(L[3 + r].re, v[1].re, tr);
        tr = vfma(L[3 + r].im, v[1].im, tr);
        tr = vfma(X[r].re, w.re, tr);
        tr = vfma(vneg(X[r].im), w.im, tr);
        V ti = vmul(L[r].re, v[0].im);
        ti = vfma(vneg(L[r].im), v[0].re, ti);
        ti = vfma(L[3 + r].re, v[1].im, ti);
        ti = vfma(vneg(L[3 + r].im), v[1].re, ti);
        ti = vfma(X[r].re, w.im, ti);
        ti = vfma(X[r].im, w.re, ti);
        acc[r].re = vfma(cf, tr, acc[r].re);
        acc[r].im = vfma(cf, ti, acc[r].im);
    }
}

// forward hop, full link: acc_r += cf (L v)_r
template <class V>
STAG_D void hop_fwd16_full(cplx<V> acc[3], const cplx<V> L[9], const cplx<V> v[3], V cf) {
#pragma unroll
    for (int r = 0; r < 3; r++) {
        V tr = vmul(L[3 * r].re, v[0].re);
        tr = vfma(vneg(L[3 * r].im), v[0].im, tr);
        V ti = vmul(L[3 * r].re, v[0].im);
        ti = vfma(L[3 * r].im, v[0].re, ti);
#pragma unroll
        for (int b = 1; b < 3; b++) {
            tr = vfma(L[3 * r + b].re, v[b].re, tr);
            tr = vfma(vneg(L[3 * r + b].im), v[b].im, tr);
            ti = vfma(L[3 * r + b].re, v[b].im, ti);
            ti = vfma(L[3 * r + b].im, v[b].re, ti);
        }
        acc[r].re = vfma(cf, tr, acc[r].re);
        acc[r].im = vfma(cf, ti, acc[r].im);
    }
}

// backward hop, full link: acc_r += cf sum_b conj(L_br) v_b
template <class V>
STAG_D void hop_bwd16_full(cplx<V> acc[3], const cplx<V> L[9], const cplx<V> v[3], V cf) {
#pragma unroll
    for (int r = 0; r < 3; r++) {
        V tr = vmul(L[r].re, v[0].re);
        tr = vfma(L[r].im, v[0].im, tr);
        V ti = vmul(L[r].re, v[0].im);
        ti = vfma(vneg(L[r].im), v[0].re, ti);
#pragma unroll
        for (int b = 1; b < 3; b++) {
            tr = vfma(L[3 * b + r].re, v[b].re, tr);
            tr = vfma(L[3 * b + r].im, v[b].im, tr);
            ti = vfma(L[3 * b + r].re, v[b].im, ti);
            ti = vfma(vneg(L[3 * b + r].im), v[b].re, ti);
        }
        acc[r].re = vfma(cf, tr, acc[r].re);
        acc[r].im = vfma(cf, ti, acc[r].im);
    }
}

// ---- loads: one site (V = float) ----------------------------------------

// raw vector of site j (its 16-byte cell); returns its norm
STAG_D float ld_vec16(const short2 *__restrict__ v, int j, cplx<float> w[3]) {
    const int4 q = ld_cell16(v, j);
    w[0] = cplx<float>{q_lo(q.x), q_hi(q.x)};
    w[1] = cplx<float>{q_lo(q.y), q_hi(q.y)};
    w[2] = cplx<float>{q_lo(q.z), q_hi(q.z)};
    return __int_as_float(q.w);
}

// rows 0, 1 of link idx of one kind (12-real 16-bit layout)
STAG_D void ld_link16(const char *kb, int S, int idx, cplx<float> L[6]) {
    const int4 a = ld_stream((const int4 *)kb + idx);
    const int2 b = ld_stream((const int2 *)(kb + (size_t)16 * S) + idx);
    L[0] = cplx<float>{q_lo(a.x), q_hi(a.x)};
    L[1] = cplx<float>{q_lo(a.y), q_hi(a.y)};
    L[2] = cplx<float>{q_lo(a.z), q_hi(a.z)};
    L[3] = cplx<float>{q_lo(a.w), q_hi(a.w)};
    L[4] = cplx<float>{q_lo(b.x), q_hi(b.x)};
    L[5] = cplx<float>{q_lo(b.y), q_hi(b.y)};
}

// the nine entries of link idx of one full kind
STAG_D void ld_link16_full(const char *kb, int S, int idx, cplx<float> L[9]) {
    int w[9];
    L16::load(kb, (size_t)S, idx, w);
#pragma unroll
    for (int e = 0; e < 9; e++)
        L[e] = cplx<float>{q_lo(w[e]), q_hi(w[e])};
}

// ---- loads: a pair of sites (V = float2, lanes ja, jb) -------------------

STAG_D cplx<float2> q2(int wa, int wb) {
    return cplx<float2>{make_float2(q_lo(wa), q_lo(wb)), make_float2(q_hi(wa), q_hi(wb))};
}

STAG_D float2 ld_vec16(const short2 *__restrict__ v, int ja, int jb, cplx<float2> w[3]) {
    const int4 qa = ld_cell16(v, ja), qb = ld_cell16(v, jb);
    w[0] = q2(qa.x, qb.x);
    w[1] = q2(qa.y, qb.y);
    w[2] = q2(qa.z, qb.z);
    return make_float2(__int_as_float(qa.w), __int_as_float(qb.w));
}

STAG_D void ld_link16(const char *kb, int S, int ia, int ib, cplx<float2> L[6]) {
    const int4 a = ld_stream((const int4 *)kb + ia), c = ld_stream((const int4 *)kb + ib);
    const int2 b = ld_stream((const int2 *)(kb + (size_t)16 * S) + ia);
    const int2 d = ld_stream((const int2 *)(kb + (size_t)16 * S) + ib);
    const int wa[6] = {a.x, a.y, a.z, a.w, b.x, b.y}, wb[6] = {c.x, c.y, c.z, c.w, d.x, d.y};
#pragma unroll
    for (int e = 0; e < 6; e++)
        L[e] = cplx<float2>{make_float2(q_lo(wa[e]), q_lo(wb[e])), make_float2(q_hi(wa[e]), q_hi(wb[e]))};
}

STAG_D void ld_link16_full(const char *kb, int S, int ia, int ib, cplx<float2> L[9]) {
    int wa[9], wb[9];
    L16::load(kb, (size_t)S, ia, wa);
    L16::load(kb, (size_t)S, ib, wb);
#pragma unroll
    for (int e = 0; e < 9; e++)
        L[e] = q2(wa[e], wb[e]);
}

// ---- the site loops -------------------------------------------------------

// acc += D psi at checkerboard site c of parity par (one site)
template <int CM, class A>
STAG_D void stencil16_site(const Geom &g, int par, int c, const void *__restrict__ Gout,
                           const void *__restrict__ Gin, const short2 *__restrict__ in, const A &a,
                           cplx<float> acc[3]) {
    const int S = g.stride;
    int x[4];
    cb_coords(g, c, par, x);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        int esum = 0;
#pragma unroll
        for (int nu = 0; nu < mu; nu++)
            esum += x[nu];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int s = h ? 3 : 1;
            const bool c12 = (CM >> h) & 1;
            const size_t off = link_kind_offset(P_F16, CM, 4 * h + mu, (size_t)S);
            const char *ko = (const char *)Gout + off;
            const char *ki = (const char *)Gin + off;
            const float ls = a.link_scale[h], lsq = ls * (1.f / kQ16);
            {
                const int j = cb_hop(g, c, x, mu, +s);
                cplx<float> v[3];
                const float cf = vmul(ld_vec16(in, j, v), lsq);
                if (c12) {
                    const int flip = (esum + (a.bc_neg[mu] ? hop_wraps(x[mu], s, g.L[mu]) : 0)) & 1;
                    cplx<float> L[6];
                    ld_link16(ko, S, c, L);
                    hop_fwd16(acc, L, v, cf, vmul(cf, ls * (flip ? -a.inv_c[h] : a.inv_c[h])));
                } else {
                    cplx<float> L[9];
                    ld_link16_full(ko, S, c, L);
                    hop_fwd16_full(acc, L, v, cf);
                }
            }
            {
                const int j = cb_hop(g, c, x, mu, -s);
                cplx<float> v[3];
                const float cf = vmul(ld_vec16(in, j, v), -lsq);
                if (c12) {
                    const int flip = (esum + (a.bc_neg[mu] ? hop_wraps(x[mu], -s, g.L[mu]) : 0)) & 1;
                    cplx<float> L[6];
                    ld_link16(ki, S, j, L);
                    hop_bwd16(acc, L, v, cf, ls * (flip ? -a.inv_c[h] : a.inv_c[h]));
                } else {
                    cplx<float> L[9];
                    ld_link16_full(ki, S, j, L);
                    hop_bwd16_full(acc, L, v, cf);
                }
            }
        }
    }
}

// The pair form applies when Lt is a multiple of 4 and at least 8: then
// (x, y, z, t) and (x, y, z, t + Lt/2), t < Lt/2, have the same x (the
// checkerboard offset depends on t through t's parity only), sit H = Vh/2
// apart in the checkerboard index, and a hop of at most 3 along t wraps at
// most one of them (the lower one backward, the upper one forward).
STAG_HD bool pair16_applies(const Geom &g) { return g.L[3] % 4 == 0 && g.L[3] >= 8; }

}  // namespace stag

// ---- the pair form, loads through an asynchronous ring ---------------------
//
// Each thread copies the links and neighbour vectors of hop k + RING into
// shared memory with cp.async while it computes hop k, so that RING hops of
// both sites' loads are in flight without holding registers.  A slot holds,
// per thread, 16-byte cells: 0, 1 entries e0..e3 of site A's and site B's
// link; 2, 3 the two sites' vector cells (three int16 pairs and the norm);
// then, for a 12-real link, 4: both sites' e4, e5; for a full link, 4, 5:
// e4..e7 of A and B, and 6: e8 of A and of B.  Every thread reads only its
// own cells, so no barrier is needed.
namespace stag {

STAG_D void cp_async16(unsigned dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
STAG_D void cp_async8(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
STAG_D void cp_async4(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
STAG_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> STAG_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// cells per slot: 5 when every link is 12-real, 7 when some are full
template <int CM> __host__ __device__ constexpr int pair16_cells() { return CM == 3 ? 5 : 7; }

// ring depth: up to three hops in flight per thread while a block's ring
// stays within 40 KB of shared memory (128-thread blocks: three hops, 30 KB;
// 256: two), fewer beyond; 0: no pair form for this block size.  At 48^3x96
// on 12-real links the 128-thread form took 368 us with three hops against
// 373.5 us with two (four and more measured slower at 768 threads per SM).
template <int BLOCK, int CM> __host__ __device__ constexpr int pair16_ring() {
    return 40960 / (pair16_cells<CM>() * 16 * BLOCK) >= 3 ? 3 : 40960 / (pair16_cells<CM>() * 16 * BLOCK);
}

// the indices of hop k = 4 mu + 2 h + dir (dir 1: backward) of the pair
// (c, c + H): neighbour vectors at ja, jb, links at ia, ib of kind 4h + mu
// in the output parity's (dir 0) or the input parity's field (dir 1)
STAG_D void pair16_hop_index(const Geom &g, int c, const int x[4], int k, int &ja, int &jb, int &ia, int &ib) {
    const int mu = k >> 2, s = ((k >> 1) & 1) ? 3 : 1, dir = k & 1, H = g.Vh >> 1;
    if (mu < 3) {
        ja = cb_hop(g, c, x, mu, dir ? -s : s);
        jb = ja + H;
    } else {
        const int t = x[3], Lh = g.L[3] >> 1, P = g.plane[3];
        if (dir == 0) {
            ja = c + s * P;
            jb = c + H + s * P - (t + s >= Lh ? g.Vh : 0);
        } else {
            ja = c - s * P + (t < s ? g.Vh : 0);
            jb = c + H - s * P;
        }
    }
    ia = dir ? ja : c;
    ib = dir ? jb : c + H;
}

// the row-2 factors ls / s of hop k (12-real links) for the two sites (eta
// b folded)
template <class A>
STAG_D float2 pair16_hop_k2(const Geom &g, const int x[4], int k, const A &a) {
    const int mu = k >> 2, h = (k >> 1) & 1, s = h ? 3 : 1, dir = k & 1;
    int esum = 0;
#pragma unroll
    for (int nu = 0; nu < mu; nu++)
        esum += x[nu];
    const int eta = esum & 1;
    const float kp = a.link_scale[h] * a.inv_c[h];
    if (mu < 3) {
        const int f = (eta + (a.bc_neg[mu] ? hop_wraps(x[mu], dir ? -s : s, g.L[mu]) : 0)) & 1;
        return vsplat<float2>(f ? -kp : kp);
    }
    const int t = x[3], Lh = g.L[3] >> 1, bn = a.bc_neg[3];
    if (dir == 0)
        return make_float2(eta ? -kp : kp, (eta ^ (bn & (t + s >= Lh))) ? -kp : kp);
    return make_float2((eta ^ (bn & (t < s))) ? -kp : kp, eta ? -kp : kp);
}

template <int BLOCK, int CM>
STAG_D void pair16_issue(unsigned cell, const Geom &g, int c, const int x[4], int k, const void *Gout,
                         const void *Gin, const short2 *in) {
    const int S = g.stride;
    int ja, jb, ia, ib;
    pair16_hop_index(g, c, x, k, ja, jb, ia, ib);
    const int mu = k >> 2, h = (k >> 1) & 1, dir = k & 1;
    const char *kb = (const char *)(dir ? Gin : Gout) + link_kind_offset(P_F16, CM, 4 * h + mu, (size_t)S);
    constexpr unsigned R = 16 * BLOCK;  // bytes between a slot's cells
    cp_async16(cell, kb + (size_t)ia * 16);
    cp_async16(cell + R, kb + (size_t)ib * 16);
    if ((CM >> h) & 1) {
        const char *k2 = kb + (size_t)16 * S;
        cp_async8(cell + 4 * R, k2 + (size_t)ia * 8);
        cp_async8(cell + 4 * R + 8, k2 + (size_t)ib * 8);
    } else {
        const char *k2 = kb + (size_t)16 * S, *k3 = kb + (size_t)32 * S;
        cp_async16(cell + 4 * R, k2 + (size_t)ia * 16);
        cp_async16(cell + 5 * R, k2 + (size_t)ib * 16);
        cp_async4(cell + 6 * R, k3 + (size_t)ia * 4);
        cp_async4(cell + 6 * R + 4, k3 + (size_t)ib * 4);
    }
    // the neighbour cells bypass L1 like the links (at 48^3x96 on 12-real
    // links 364 against 367 us with L1-allocating copies): their reuse is
    // across blocks, in L2
    cp_async16(cell + 2 * R, (const int4 *)in + ja);
    cp_async16(cell + 3 * R, (const int4 *)in + jb);
}

// acc += D psi at sites c and c + H (c < H = Vh/2), loads through the ring
// (ring: this block's RING * pair16_cells<CM>() * BLOCK cells of 16 bytes)
template <int BLOCK, int RING, int CM, class A>
STAG_D void stencil16_pair_async(const Geom &g, int par, int c, const void *__restrict__ Gout,
                                 const void *__restrict__ Gin, const short2 *__restrict__ in, const A &a,
                                 int4 *ring, cplx<float2> acc[3]) {
    constexpr int CELLS = pair16_cells<CM>();
    int x[4];
    cb_coords(g, c, par, x);
    const unsigned cell0 = (unsigned)__cvta_generic_to_shared(ring + threadIdx.x);
#pragma unroll
    for (int k = 0; k < RING; k++) {
        pair16_issue<BLOCK, CM>(cell0 + (unsigned)(k * CELLS * BLOCK * 16), g, c, x, k, Gout, Gin, in);
        cp_async_commit();
    }
#pragma unroll
    for (int k = 0; k < 16; k++) {
        cp_async_wait<RING - 1>();
        const int slot = k % RING, h = (k >> 1) & 1, dir = k & 1;
        const int4 *cell = ring + slot * CELLS * BLOCK + threadIdx.x;
        const int4 la = cell[0], lb = cell[BLOCK], va = cell[2 * BLOCK], vb = cell[3 * BLOCK];
        cplx<float2> v[3];
        v[0] = q2(va.x, vb.x);
        v[1] = q2(va.y, vb.y);
        v[2] = q2(va.z, vb.z);
        const float lsq = a.link_scale[h] * (1.f / kQ16);
        const float2 nrm = make_float2(__int_as_float(va.w), __int_as_float(vb.w));
        if ((CM >> h) & 1) {
            const int4 l2 = cell[4 * BLOCK];
            cplx<float2> L[6];
            L[0] = q2(la.x, lb.x);
            L[1] = q2(la.y, lb.y);
            L[2] = q2(la.z, lb.z);
            L[3] = q2(la.w, lb.w);
            L[4] = q2(l2.x, l2.z);
            L[5] = q2(l2.y, l2.w);
            const float2 k2 = pair16_hop_k2(g, x, k, a);
            if (dir == 0) {
                const float2 cf = vmul(nrm, vsplat<float2>(lsq));
                hop_fwd16(acc, L, v, cf, vmul(cf, k2));
            } else {
                hop_bwd16(acc, L, v, vmul(nrm, vsplat<float2>(-lsq)), k2);
            }
        } else {
            const int4 ma = cell[4 * BLOCK], mb = cell[5 * BLOCK], e8 = cell[6 * BLOCK];
            cplx<float2> L[9];
            L[0] = q2(la.x, lb.x);
            L[1] = q2(la.y, lb.y);
            L[2] = q2(la.z, lb.z);
            L[3] = q2(la.w, lb.w);
            L[4] = q2(ma.x, mb.x);
            L[5] = q2(ma.y, mb.y);
            L[6] = q2(ma.z, mb.z);
            L[7] = q2(ma.w, mb.w);
            L[8] = q2(e8.x, e8.y);
            if (dir == 0)
                hop_fwd16_full(acc, L, v, vmul(nrm, vsplat<float2>(lsq)));
            else
                hop_bwd16_full(acc, L, v, vmul(nrm, vsplat<float2>(-lsq)));
        }
        // the slot's cells are in registers now; refill it with hop k + RING
        if (k + RING < 16)
            pair16_issue<BLOCK, CM>(cell0 + (unsigned)(slot * CELLS * BLOCK * 16), g, c, x, k + RING, Gout, Gin,
                                    in);
        cp_async_commit();
    }
}

}  // namespace stag
