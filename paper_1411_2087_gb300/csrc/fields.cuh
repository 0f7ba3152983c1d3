// Storage formats of links and colour vectors, one per precision, and the
// cache-hinted loads/stores the kernels use.
//
// Layout (structure of arrays, one checkerboard):
//   colour vector   Elem v[3][stride]           component a of site c at a*stride + c
//                   16-bit: one 16-byte cell per site instead, the three
//                   components (int16 pairs) and the site's float norm, so
//                   that a gather of one neighbour is one 16-byte load
//   links           G[2][8][...]                [site parity][kind], kind 0..3 =
//                   folded one-link U~_mu, 4..7 = folded three-link N~_mu; a
//                   full kind is Elem [9][stride] ([row*3+col][cb site]), in
//                   16-bit three planes instead (see link_kind_bytes)
// One Elem holds one complex number: a warp loading component j of 32
// consecutive sites touches one contiguous segment.
#pragma once
#include "common.cuh"

namespace stag {

enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_DF64 = 3 };

// cache hints: links stream through once (evict-first); colour vectors are
// gathered 16 times per launch and should stay in L1/L2.
template <class T> STAG_D T ld_stream(const T *p) { return __ldcs(p); }
template <class T> STAG_D T ld_keep(const T *p) { return __ldg(p); }

template <int P> struct Fmt;

template <> struct Fmt<P_F64> {
    using Elem = double2;
    using R = double;
    STAG_D static cplx<R> unpack(double2 e) { return cplx<R>{e.x, e.y}; }
    STAG_D static double2 pack(const cplx<R> &c) { return make_double2(c.re, c.im); }
    STAG_D static cplx<R> make(double re, double im) { return cplx<R>{re, im}; }
    STAG_D static cplx<R> unpack_link(double2 e, float) { return unpack(e); }
    STAG_D static double2 pack_link(double re, double im, float) { return make_double2(re, im); }
};

template <> struct Fmt<P_DF64> {
    using Elem = float4;  // re.hi, re.lo, im.hi, im.lo
    using R = df;
    STAG_D static cplx<R> unpack(float4 e) { return cplx<R>{df_make(e.x, e.y), df_make(e.z, e.w)}; }
    STAG_D static float4 pack(const cplx<R> &c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }
    STAG_D static cplx<R> make(double re, double im) {
        return cplx<R>{df_from_double(re), df_from_double(im)};
    }
    STAG_D static cplx<R> unpack_link(float4 e, float) { return unpack(e); }
    STAG_D static float4 pack_link(double re, double im, float) { return pack(make(re, im)); }
};

template <> struct Fmt<P_F32> {
    using Elem = float2;
    using R = float;
    STAG_D static cplx<R> unpack(float2 e) { return cplx<R>{e.x, e.y}; }
    STAG_D static float2 pack(const cplx<R> &c) { return make_float2(c.re, c.im); }
    STAG_D static cplx<R> make(double re, double im) { return cplx<R>{(float)re, (float)im}; }
    STAG_D static cplx<R> unpack_link(float2 e, float) { return unpack(e); }
    STAG_D static float2 pack_link(double re, double im, float) { return make_float2((float)re, (float)im); }
};

// 16-bit storage: signed fixed point q = round(v / scale * 32767), float
// arithmetic.  Links use one scale per field (the largest |entry| of the
// folded one-link or three-link field); colour vectors one per site (the
// largest |component| at that site), stored in the site's cell after its
// three components.
constexpr float kQ16 = 32767.f;

STAG_D short q16(float v) { return (short)__float2int_rn(fminf(fmaxf(v, -kQ16), kQ16)); }

// the two int16 halves of a 32-bit word (a short2: x low, y high) as floats
// (exact), and the word from two stored values
STAG_D float q_lo(int w) { return (float)(short)(w & 0xffff); }
STAG_D float q_hi(int w) { return (float)(w >> 16); }
STAG_D int q16_pair(float re, float im) {
    return (int)((unsigned)(unsigned short)q16(re) | ((unsigned)(unsigned short)q16(im) << 16));
}

template <> struct Fmt<P_F16> {
    using Elem = short2;
    using R = float;
    STAG_D static cplx<R> make(double re, double im) { return cplx<R>{(float)re, (float)im}; }
    // scale = field max / 32767
    STAG_D static cplx<R> unpack_link(short2 e, float scale) {
        return cplx<R>{(float)e.x * scale, (float)e.y * scale};
    }
    // inv_scale = 32767 / field max
    STAG_D static short2 pack_link(double re, double im, float inv_scale) {
        return make_short2(q16((float)re * inv_scale), q16((float)im * inv_scale));
    }
};

// --------------------------------------------------------------------------
// 12-real ("two-row") compressed links (the paper's gauge compression,
// Sec. 4): rows 0 and 1 of the folded link L = s U, U in SU(3), s = c eta b;
// row 2 = conj(row0 x row1) / s is rebuilt in the kernel.  Per parity and
// kind, entries e0..e5 (row-major rows 0, 1):
//   FP32:   float4 [3][stride], chunk k holds e(2k), e(2k+1)  (48 B per link)
//   16-bit: int4 [stride] (e0..e3) then int2 [stride] (e4, e5) (24 B per link)
// --------------------------------------------------------------------------
template <int P> struct C12;

template <> struct C12<P_F32> {
    STAG_HD static size_t kind_bytes(size_t S) { return 3 * S * 16; }
    STAG_D static void load(const char *kind_base, int S, int idx, float, cplx<float> L[6]) {
        const float4 *p = (const float4 *)kind_base;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float4 v = ld_stream(p + k * S + idx);
            L[2 * k] = cplx<float>{v.x, v.y};
            L[2 * k + 1] = cplx<float>{v.z, v.w};
        }
    }
    STAG_D static void store(char *kind_base, size_t S, size_t idx, int e, double re, double im, float) {
        float2 *p = (float2 *)((float4 *)kind_base + (e / 2) * S + idx) + (e % 2);
        *p = make_float2((float)re, (float)im);
    }
};

template <> struct C12<P_F16> {
    STAG_HD static size_t kind_bytes(size_t S) { return 24 * S; }
    STAG_D static cplx<float> q(int v, float scale) {
        return cplx<float>{(float)(short)(v & 0xffff) * scale, (float)(v >> 16) * scale};
    }
    STAG_D static void load(const char *kind_base, int S, int idx, float scale, cplx<float> L[6]) {
        const int4 a = ld_stream((const int4 *)kind_base + idx);
        const int2 b = ld_stream((const int2 *)(kind_base + (size_t)16 * S) + idx);
        L[0] = q(a.x, scale);
        L[1] = q(a.y, scale);
        L[2] = q(a.z, scale);
        L[3] = q(a.w, scale);
        L[4] = q(b.x, scale);
        L[5] = q(b.y, scale);
    }
    STAG_D static void store(char *kind_base, size_t S, size_t idx, int e, double re, double im, float inv_scale) {
        short2 *p = e < 4 ? (short2 *)kind_base + idx * 4 + e : (short2 *)(kind_base + 16 * S) + idx * 2 + (e - 4);
        *p = make_short2(q16((float)re * inv_scale), q16((float)im * inv_scale));
    }
};

// --------------------------------------------------------------------------
// Link storage by kind.  A full kind is 9 entries per site: Elem [9][stride]
// planes in FP64, double-float and FP32; in 16-bit three planes, int4
// [stride] (entries 0..3), int4 [stride] (entries 4..7) and int [stride]
// (entry 8), each entry an int16 pair, so that a link is three loads.  A
// 12-real kind is C12's layout.  Per parity the one-link kinds 0..3 come
// first, then the three-link kinds 4..7; the bits of a compression mask say
// which group is 12-real (bit 0 one-link, bit 1 three-link).
// --------------------------------------------------------------------------
STAG_HD size_t link_kind_bytes(int p, bool c12, size_t S) {
    if (c12)
        return p == P_F32 ? 48 * S : 24 * S;
    return p == P_F32 ? 72 * S : p == P_F16 ? 36 * S : 144 * S;
}
STAG_HD size_t link_kind_offset(int p, int mask, int kind, size_t S) {
    const size_t k1 = link_kind_bytes(p, mask & 1, S), k3 = link_kind_bytes(p, (mask >> 1) & 1, S);
    return kind < 4 ? (size_t)kind * k1 : 4 * k1 + (size_t)(kind - 4) * k3;
}
STAG_HD size_t link_parity_bytes(int p, int mask, size_t S) { return link_kind_offset(p, mask, 8, S); }

// the full 16-bit kind: where entry e of link idx lives, and its nine raw
// int16 pairs in three loads
struct L16 {
    STAG_D static short2 *slot(char *kb, size_t S, size_t idx, int e) {
        if (e < 4)
            return (short2 *)kb + idx * 4 + e;
        if (e < 8)
            return (short2 *)(kb + 16 * S) + idx * 4 + (e - 4);
        return (short2 *)(kb + 32 * S) + idx;
    }
    STAG_D static void load(const char *kb, size_t S, int idx, int w[9]) {
        const int4 a = ld_stream((const int4 *)kb + idx);
        const int4 b = ld_stream((const int4 *)(kb + 16 * S) + idx);
        w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w;
        w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
        w[8] = ld_stream((const int *)(kb + 32 * S) + idx);
    }
};

inline size_t c12_link_bytes(int p, size_t stride, int mask = 3) {  // both parities, 8 kinds
    return (p == P_F32 || p == P_F16) ? 2 * link_parity_bytes(p, mask, stride) : 0;
}

// bytes of one colour-vector field / one complex link entry
inline size_t prec_vec_bytes(int p, size_t stride) {
    switch (p) {
    case P_F64: return 3 * stride * sizeof(double2);
    case P_DF64: return 3 * stride * sizeof(float4);
    case P_F32: return 3 * stride * sizeof(float2);
    case P_F16: return stride * sizeof(int4);  // one 16-byte cell per site
    default: return 0;
    }
}
// bytes from one site's entry of a colour vector to the next site's (within
// a component plane; a 16-bit field's cell holds all components)
inline size_t vec_site_bytes(int p) { return p == P_F16 ? 16 : prec_vec_bytes(p, 1) / 3; }
inline size_t prec_link_elem_bytes(int p) {
    switch (p) {
    case P_F64: return sizeof(double2);
    case P_DF64: return sizeof(float4);
    case P_F32: return sizeof(float2);
    case P_F16: return sizeof(short2);
    default: return 0;
    }
}

// --------------------------------------------------------------------------
// colour-vector loads and stores (one site, three components)
// --------------------------------------------------------------------------
template <int P>
STAG_D void load_vec(const typename Fmt<P>::Elem *__restrict__ v, int stride, int c,
                     cplx<typename Fmt<P>::R> w[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++)
        w[a] = Fmt<P>::unpack(ld_keep(v + a * stride + c));
}

// the 16-bit cell of site c: components 0..2 as int16 pairs (re low, im
// high) in x, y, z, the norm's bits in w
STAG_D int4 ld_cell16(const short2 *__restrict__ v, int c) { return ld_keep((const int4 *)v + c); }

template <>
STAG_D void load_vec<P_F16>(const short2 *__restrict__ v, int stride, int c, cplx<float> w[3]) {
    (void)stride;
    const int4 q = ld_cell16(v, c);
    const float s = __int_as_float(q.w) * (1.f / kQ16);
    const int qa[3] = {q.x, q.y, q.z};
#pragma unroll
    for (int a = 0; a < 3; a++)
        w[a] = cplx<float>{(float)(short)(qa[a] & 0xffff) * s, (float)(qa[a] >> 16) * s};
}

template <int P>
STAG_D void store_vec(typename Fmt<P>::Elem *__restrict__ v, int stride, int c,
                      const cplx<typename Fmt<P>::R> w[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++)
        __stcs(v + a * stride + c, Fmt<P>::pack(w[a]));
}

template <>
STAG_D void store_vec<P_F16>(short2 *__restrict__ v, int stride, int c, const cplx<float> w[3]) {
    (void)stride;
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++)
        m = fmaxf(m, fmaxf(fabsf(w[a].re), fabsf(w[a].im)));
    const float inv = m > 0.f ? kQ16 / m : 0.f;
    int q[3];
#pragma unroll
    for (int a = 0; a < 3; a++)
        q[a] = q16_pair(w[a].re * inv, w[a].im * inv);
    __stcs((int4 *)v + c, make_int4(q[0], q[1], q[2], __float_as_int(m)));
}

// to/from canonical complex128 for export and the double-valued epilogues
template <class R> STAG_D double to_double(R a);
template <> STAG_D double to_double<double>(double a) { return a; }
template <> STAG_D double to_double<float>(float a) { return (double)a; }
template <> STAG_D double to_double<df>(df a) { return df_to_double(a); }

// convert between arithmetic types (used when one kernel reads two precisions)
template <class RO, class RI> STAG_D RO rconv(RI a);
template <> STAG_D double rconv<double, double>(double a) { return a; }
template <> STAG_D double rconv<double, float>(float a) { return (double)a; }
template <> STAG_D float rconv<float, double>(double a) { return (float)a; }
template <> STAG_D float rconv<float, float>(float a) { return a; }
template <> STAG_D df rconv<df, df>(df a) { return a; }
template <> STAG_D df rconv<df, float>(float a) { return df_make(a, 0.f); }
template <> STAG_D float rconv<float, df>(df a) { return a.hi + a.lo; }

template <class RO, class RI> STAG_D cplx<RO> cconv(const cplx<RI> &a) {
    return cplx<RO>{rconv<RO, RI>(a.re), rconv<RO, RI>(a.im)};
}

}  // namespace stag
