// Shared device-side types: complex numbers over several real types, the
// double-float real type, storage formats of links and colour vectors, and
// lattice geometry.  Everything here is internal to libstag.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#define STAG_HD __host__ __device__ __forceinline__
#define STAG_D __device__ __forceinline__

namespace stag {

// --------------------------------------------------------------------------
// double-float: value = hi + lo, |lo| <= ulp(hi)/2.  Products use the FMA
// error-free transformation, sums Knuth's TwoSum, so that one multiply-add
// keeps about 48 significant bits.  Accumulators may carry an unnormalised
// lo (the sum of all captured rounding errors); df_norm() renormalises.
// The operations use explicitly rounded intrinsics, so that the compiler
// fuses no multiply into a later add (which would break TwoSum's premise
// s = fl(a + b)).
// --------------------------------------------------------------------------
struct df {
    float hi, lo;
};

STAG_HD df df_make(float h, float l) { df r; r.hi = h; r.lo = l; return r; }
STAG_HD df df_zero() { return df_make(0.f, 0.f); }
STAG_HD df operator-(df a) { return df_make(-a.hi, -a.lo); }

// exact split of a double into hi + lo (round to nearest twice)
STAG_HD df df_from_double(double d) {
    float h = (float)d;
    float l = (float)(d - (double)h);
    return df_make(h, l);
}
STAG_HD double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// TwoSum: s + e == a + b exactly
STAG_D void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

STAG_D df df_norm(df a) {
    float s, e;
    two_sum(a.hi, a.lo, s, e);
    return df_make(s, e);
}

// acc += a * b  (acc lo left unnormalised)
STAG_D void df_mac(df &acc, df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

STAG_D df df_add(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_norm(df_make(s, e));
}
STAG_D df df_sub(df a, df b) { return df_add(a, -b); }

STAG_D df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_norm(df_make(p, e));
}

// --------------------------------------------------------------------------
// generic real arithmetic used by the stencil templates
// --------------------------------------------------------------------------
STAG_D void mac(double &acc, double a, double b) { acc = fma(a, b, acc); }
STAG_D void mac(float &acc, float a, float b) { acc = fmaf(a, b, acc); }
STAG_D void mac(df &acc, df a, df b) { df_mac(acc, a, b); }

STAG_D double rsub(double a, double b) { return a - b; }
STAG_D float rsub(float a, float b) { return a - b; }
STAG_D df rsub(df a, df b) { return df_sub(a, b); }
STAG_D double radd(double a, double b) { return a + b; }
STAG_D float radd(float a, float b) { return a + b; }
STAG_D df radd(df a, df b) { return df_add(a, b); }

template <class R> STAG_D R rzero();
template <> STAG_D double rzero<double>() { return 0.0; }
template <> STAG_D float rzero<float>() { return 0.f; }
template <> STAG_D df rzero<df>() { return df_zero(); }

template <class R> STAG_D R rnorm(R a) { return a; }
template <> STAG_D df rnorm<df>(df a) { return df_norm(a); }

template <class R> struct cplx {
    R re, im;
};

template <class R> STAG_D cplx<R> czero() { return cplx<R>{rzero<R>(), rzero<R>()}; }
template <class R> STAG_D cplx<R> cneg(cplx<R> a) { return cplx<R>{-a.re, -a.im}; }

// acc += u * v
template <class R> STAG_D void cmac(cplx<R> &acc, const cplx<R> &u, const cplx<R> &v) {
    mac(acc.re, u.re, v.re);
    mac(acc.re, -u.im, v.im);
    mac(acc.im, u.re, v.im);
    mac(acc.im, u.im, v.re);
}
// acc += conj(u) * v
template <class R> STAG_D void cmac_conj(cplx<R> &acc, const cplx<R> &u, const cplx<R> &v) {
    mac(acc.re, u.re, v.re);
    mac(acc.re, u.im, v.im);
    mac(acc.im, u.re, v.im);
    mac(acc.im, -u.im, v.re);
}

// --------------------------------------------------------------------------
// geometry
// --------------------------------------------------------------------------
// Division by a fixed divisor d as a multiply (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, n / d equals
// (mulhi(m, n) + n) >> l for every 0 <= n < 2^31.
struct FastDiv {
    unsigned m;
    int l;
};
inline FastDiv fastdiv_make(int d) {
    int l = 0;
    while ((1LL << l) < d)
        l++;
    const unsigned long long m = ((1ULL << 32) * ((1ULL << l) - (unsigned long long)d)) / (unsigned long long)d + 1;
    return FastDiv{(unsigned)m, l};
}
STAG_HD int fastdiv(int n, FastDiv f) {
    const unsigned t = (unsigned)(((unsigned long long)f.m * (unsigned)n) >> 32);
    return (int)((t + (unsigned)n) >> f.l);
}

struct Geom {
    int L[4];     // Lx, Ly, Lz, Lt
    int Lxh;      // Lx / 2
    int Vh;       // sites per parity
    int stride;   // elements between colour/component planes (>= Vh, padded)
    int plane[4]; // cb-index step of one hop: 1/2 (x, handled apart), Lx/2, Lx*Ly/2, Lx*Ly*Lz/2
    FastDiv div[3]; // division by Lxh, Ly, Lz (geom_set_div)
};

// the divisors of cb_coords; every Geom is finished with this
inline void geom_set_div(Geom &g) {
    g.div[0] = fastdiv_make(g.Lxh);
    g.div[1] = fastdiv_make(g.L[1]);
    g.div[2] = fastdiv_make(g.L[2]);
}

// coordinates of checkerboard site c of parity par
STAG_HD void cb_coords(const Geom &g, int c, int par, int x[4]) {
    const int r1 = fastdiv(c, g.div[0]);
    const int xh = c - r1 * g.Lxh;
    const int r2 = fastdiv(r1, g.div[1]);
    x[1] = r1 - r2 * g.L[1];
    x[3] = fastdiv(r2, g.div[2]);
    x[2] = r2 - x[3] * g.L[2];
    x[0] = 2 * xh + ((par + x[1] + x[2] + x[3]) & 1);
}

// checkerboard index of the site reached from (c, x) by s steps along mu
// (periodic in index space; the parity flips for odd s)
STAG_HD int cb_hop(const Geom &g, int c, const int x[4], int mu, int s) {
    int L = g.L[mu];
    int y = x[mu] + s;
    // |s| <= 3 and L >= 2: at most two wraps
    if (y >= L) y -= L;
    if (y >= L) y -= L;
    if (y < 0) y += L;
    if (y < 0) y += L;
    if (mu == 0) {
        // full index changes by y - x; cb = floor(full / 2), full parity = x & 1
        return c + (((x[0] & 1) + y - x[0]) >> 1);
    }
    return c + (y - x[mu]) * g.plane[mu];
}

}  // namespace stag
