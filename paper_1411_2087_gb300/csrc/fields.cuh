// Storage formats of links and colour vectors, one per precision, and the
// cache-hinted loads/stores the kernels use.
//
// Layout (structure of arrays, one checkerboard):
//   colour vector   Elem v[3][stride]           component a of site c at a*stride + c
//   links           Elem G[2][8][9][stride]     [site parity][kind][row*3+col][cb site]
//                   kind 0..3 = folded one-link U~_mu, 4..7 = folded three-link N~_mu
// One Elem holds one complex number: a warp loading component j of 32
// consecutive sites touches one contiguous 512-byte (16-byte Elem) segment.
#pragma once
#include "common.cuh"

namespace stag {

enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_DF64 = 3 };

// cache hints: links stream through once (evict-first); colour vectors are
// gathered 16 times per launch and should stay in L1/L2.
STAG_D double2 ld_stream(const double2 *p) { return __ldcs(p); }
STAG_D float4 ld_stream(const float4 *p) { return __ldcs(p); }
STAG_D float2 ld_stream(const float2 *p) { return __ldcs(p); }
STAG_D double2 ld_keep(const double2 *p) { return __ldg(p); }
STAG_D float4 ld_keep(const float4 *p) { return __ldg(p); }
STAG_D float2 ld_keep(const float2 *p) { return __ldg(p); }

template <int P> struct Fmt;

template <> struct Fmt<P_F64> {
    using Elem = double2;
    using R = double;
    STAG_D static cplx<R> unpack(double2 e) { return cplx<R>{e.x, e.y}; }
    STAG_D static double2 pack(const cplx<R> &c) { return make_double2(c.re, c.im); }
    STAG_HD static double2 from_double(double re, double im) { return make_double2(re, im); }
};

template <> struct Fmt<P_DF64> {
    using Elem = float4;  // re.hi, re.lo, im.hi, im.lo
    using R = df;
    STAG_D static cplx<R> unpack(float4 e) { return cplx<R>{df_make(e.x, e.y), df_make(e.z, e.w)}; }
    STAG_D static float4 pack(const cplx<R> &c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }
    STAG_HD static float4 from_double(double re, double im) {
        df r = df_from_double(re), i = df_from_double(im);
        return make_float4(r.hi, r.lo, i.hi, i.lo);
    }
};

template <> struct Fmt<P_F32> {
    using Elem = float2;
    using R = float;
    STAG_D static cplx<R> unpack(float2 e) { return cplx<R>{e.x, e.y}; }
    STAG_D static float2 pack(const cplx<R> &c) { return make_float2(c.re, c.im); }
    STAG_HD static float2 from_double(double re, double im) { return make_float2((float)re, (float)im); }
};

template <int P> STAG_HD size_t elem_bytes() { return sizeof(typename Fmt<P>::Elem); }

inline size_t prec_elem_bytes(int p) {
    switch (p) {
    case P_F64: return sizeof(double2);
    case P_DF64: return sizeof(float4);
    case P_F32: return sizeof(float2);
    default: return 0;
    }
}

// to/from canonical complex128 for export and the double-valued epilogues
template <class R> STAG_D double to_double(R a);
template <> STAG_D double to_double<double>(double a) { return a; }
template <> STAG_D double to_double<float>(float a) { return (double)a; }
template <> STAG_D double to_double<df>(df a) { return df_to_double(a); }

}  // namespace stag
