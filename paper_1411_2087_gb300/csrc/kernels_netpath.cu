// The learned preconditioner evaluated in path form.
//
// The net (three gauge-covariant convolution layers 1 -> C -> C -> 1, no
// nonlinearity; include/stag.h) is linear in its input, and its colour-blind
// weights commute with the link transports.  Each layer applies at most one
// hop, T_0 = 1 or T_d psi(x) = U_mu(x) psi(x+mu) (d = +mu) or
// U_mu(x-mu)^+ psi(x-mu) (d = -mu), so the whole net is a sum over hop
// sequences (d1, d2, d3) of (W3[d3] W2[d2] W1[d1]) T_d3 T_d2 T_d1.  As a
// preconditioner its input r lives on the even sites and only its even
// outputs are kept, which leaves the sequences with zero or two hops:
//
//   z(x) = c0 r(x) + sum_{a,b} C[a][b] (T_a T_b r)(x)          (x even)
//   c0      = W3[0] W2[0] W1[0]
//   C[a][b] = W3[0] W2[a] W1[b] + W3[a] W2[0] W1[b] + W3[a] W2[b] W1[0]
//
// (row . matrix . column products over the channels).  Two kernels evaluate
// it: net_mid_kernel forms chi_a(y) = sum_b C[a][b] (T_b r)(y) on the odd
// sites (eight link transports and an 8 x 8 complex mixing per site), and
// net_out_kernel adds the eight transports T_a chi_a on the even sites.
// That is 16 link matrices and about 1.4k multiply-adds per even site,
// against 27 link loads and about 12k multiply-adds per site for the three
// layers one after another.  Training differentiates the same form: the
// gradient with respect to C[a][b] is <T_b r, T_a^+ g> summed over the odd
// sites (g = dL/dz*), and the chain rule through the products above gives
// the gradient of every layer weight.
#include <type_traits>

#include "kernels.h"
#include "learned.cuh"
#include "reduce.cuh"

namespace stag {

// ---- links -----------------------------------------------------------------
// Net links per parity, the boundary sign of a wrapping forward hop folded
// into the last-slice link.  FP32 (float2): structure of arrays, element e
// (row*3+col) of U_mu at checkerboard site c of parity par at
// ((par*4 + mu)*9 + e)*S + c.  16-bit (short2, value = q * scale): per
// (par, mu) 36 S bytes, an int4 plane with e0..e3, an int4 plane with
// e4..e7 and an int plane with e8, so that a link is three loads.
STAG_D cplx<float> nl_get(float2 v) { return cplx<float>{v.x, v.y}; }

template <class LT>
STAG_D void nl_load(const LT *__restrict__ NL, int S, int par, int mu, int c, cplx<float> U[9]);

template <>
STAG_D void nl_load<float2>(const float2 *__restrict__ NL, int S, int par, int mu, int c, cplx<float> U[9]) {
    const float2 *p = NL + (size_t)((par * 4 + mu) * 9) * S + c;
#pragma unroll
    for (int e = 0; e < 9; e++)
        U[e] = nl_get(ld_stream(p + (size_t)e * S));
}

STAG_D const char *nl16_base(const void *NL, int S, int par, int mu) {
    return (const char *)NL + (size_t)(par * 4 + mu) * 36 * S;
}

template <>
STAG_D void nl_load<short2>(const short2 *__restrict__ NL, int S, int par, int mu, int c, cplx<float> U[9]) {
    const char *base = nl16_base(NL, S, par, mu);
    const int4 a = ld_stream((const int4 *)base + c);
    const int4 b = ld_stream((const int4 *)(base + (size_t)16 * S) + c);
    const int e8 = ld_stream((const int *)(base + (size_t)32 * S) + c);
    const int w[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, e8};
#pragma unroll
    for (int e = 0; e < 9; e++)
        U[e] = cplx<float>{q_lo(w[e]), q_hi(w[e])};
}

// 12-real 16-bit links (special unitary fat links): per (par, mu) an int4
// plane with entries 0..3 and an int2 plane with entries 4, 5 (rows 0 and
// 1); row 2 of V = s U (s = eta b = +-1, U in SU(3)) is s conj(r0 x r1), in
// raw units k2 conj(q0 x q1) with k2 = s * scale
struct L12 {
    int4 v;
};

STAG_D const char *nl12_base(const void *NL, int S, int par, int mu) {
    return (const char *)NL + (size_t)(par * 4 + mu) * 24 * S;
}

STAG_D void nl_load12(const L12 *__restrict__ NL, int S, int par, int mu, int c, float k2, cplx<float> U[9]) {
    const char *base = nl12_base(NL, S, par, mu);
    const int4 a = ld_stream((const int4 *)base + c);
    const int2 b = ld_stream((const int2 *)(base + (size_t)16 * S) + c);
    const int w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
#pragma unroll
    for (int e = 0; e < 6; e++)
        U[e] = cplx<float>{q_lo(w[e]), q_hi(w[e])};
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        // X_j = r0_k r1_l - r0_l r1_k; row 2 entry j = k2 conj(X_j)
        const float re = U[k].re * U[3 + l].re - U[k].im * U[3 + l].im - (U[l].re * U[3 + k].re - U[l].im * U[3 + k].im);
        const float im = U[k].re * U[3 + l].im + U[k].im * U[3 + l].re - (U[l].re * U[3 + k].im + U[l].im * U[3 + k].re);
        U[6 + j] = cplx<float>{k2 * re, -k2 * im};
    }
}

// s = eta_mu(x) b of the link a hop of the net takes from site x: its own
// link (bw = 0; b = -1 when it wraps forward, x_mu = L - 1) or the link of
// x - mu (bw = 1; that link wraps when x_mu = 0); eta_mu(x - mu) = eta_mu(x)
STAG_D float nl_link_sign(const Geom &g, const int x[4], int mu, int bw, int bcneg) {
    int esum = 0;
#pragma unroll
    for (int nu = 0; nu < mu; nu++)
        esum += x[nu];
    const bool wrap = ((bcneg >> mu) & 1) && (bw ? x[mu] == 0 : x[mu] == g.L[mu] - 1);
    return ((esum & 1) ^ (wrap ? 1 : 0)) ? -1.f : 1.f;
}

// link V_mu (or the one the hop bw takes) of any layout, in raw units
template <class LT>
STAG_D void net_link(const LT *__restrict__ NL, int S, int par, int mu, int idx, const Geom &g, const int x[4],
                     int bw, float ls, int bcneg, cplx<float> U[9]) {
    if constexpr (std::is_same<LT, L12>::value)
        nl_load12(NL, S, par, mu, idx, nl_link_sign(g, x, mu, bw, bcneg) * ls, U);
    else
        nl_load(NL, S, par, mu, idx, U);
}

// the address of element e of U_mu at (par, c) in either layout
STAG_D float2 *nl_slot(float2 *NL, int S, int par, int mu, int c, int e) {
    return NL + (size_t)((par * 4 + mu) * 9 + e) * S + c;
}
STAG_D short2 *nl_slot(short2 *NL, int S, int par, int mu, int c, int e) {
    char *base = (char *)nl16_base(NL, S, par, mu);
    if (e < 4)
        return (short2 *)base + (size_t)c * 4 + e;
    if (e < 8)
        return (short2 *)(base + (size_t)16 * S) + (size_t)c * 4 + (e - 4);
    return (short2 *)(base + (size_t)32 * S) + c;
}

// h = U v (adj = false) or U^+ v
STAG_D void nl_apply(const cplx<float> U[9], bool adj, const cplx<float> v[3], cplx<float> h[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cplx<float> t = czero<float>();
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (adj)
                cmac_conj(t, U[3 * b + a], v[b]);
            else
                cmac(t, U[3 * a + b], v[b]);
        }
        h[a] = t;
    }
}

// canonical raw fat links complex128 [4][V][3][3] -> net links of both
// parities, eta_mu(x) b U_mu(x): the Kogut-Susskind phase of the link's site
// and the boundary sign of a wrapping forward hop folded in, no coefficient;
// one thread per (mu, site).  inv_scale: 16-bit only.
//
// The phases make the net's two-hop paths those of the operator: the
// product eta_mu(x) eta_nu(x + mu) of a path that turns from mu to nu
// depends on the site, so with raw links translation-invariant weights
// could only form the paths that keep their direction; with phased links
// they can form D^2 itself, and with it a degree-one polynomial in M.
template <class LT> STAG_D LT nl_pack(double re, double im, float inv_scale);
template <> STAG_D float2 nl_pack<float2>(double re, double im, float) { return make_float2((float)re, (float)im); }
template <> STAG_D short2 nl_pack<short2>(double re, double im, float inv) {
    return make_short2(q16((float)re * inv), q16((float)im * inv));
}

template <class LT>
__global__ void net_links_cb_kernel(Geom g, double bc0, double bc1, double bc2, double bc3,
                                    const double2 *__restrict__ fat, LT *NL, float inv_scale) {
    const long long V = 2LL * g.Vh;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 4 * V)
        return;
    const int mu = (int)(t / V);
    const int i = (int)(t % V);
    int x[4];
    x[0] = i % g.L[0];
    int rr = i / g.L[0];
    x[1] = rr % g.L[1];
    rr /= g.L[1];
    x[2] = rr % g.L[2];
    x[3] = rr / g.L[2];
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const double bc[4] = {bc0, bc1, bc2, bc3};
    int esum = 0;
    for (int nu = 0; nu < mu; nu++)
        esum += x[nu];
    const double sgn = ((x[mu] == g.L[mu] - 1 && bc[mu] < 0) ? -1.0 : 1.0) * ((esum & 1) ? -1.0 : 1.0);
    const int S = g.stride;
#pragma unroll 1
    for (int e = 0; e < 9; e++) {
        const double2 u = fat[((size_t)mu * V + i) * 9 + e];
        *nl_slot(NL, S, par, mu, i >> 1, e) = nl_pack<LT>(sgn * u.x, sgn * u.y, inv_scale);
    }
}

// rows 0 and 1 of eta_mu(x) b U_mu(x) into the 12-real 16-bit planes
__global__ void net_links12_kernel(Geom g, double bc0, double bc1, double bc2, double bc3,
                                   const double2 *__restrict__ fat, char *NL, float inv_scale) {
    const long long V = 2LL * g.Vh;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 4 * V)
        return;
    const int mu = (int)(t / V);
    const int i = (int)(t % V);
    int x[4];
    x[0] = i % g.L[0];
    int rr = i / g.L[0];
    x[1] = rr % g.L[1];
    rr /= g.L[1];
    x[2] = rr % g.L[2];
    x[3] = rr / g.L[2];
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const double bc[4] = {bc0, bc1, bc2, bc3};
    int esum = 0;
    for (int nu = 0; nu < mu; nu++)
        esum += x[nu];
    const double sgn = ((x[mu] == g.L[mu] - 1 && bc[mu] < 0) ? -1.0 : 1.0) * ((esum & 1) ? -1.0 : 1.0);
    const size_t S = (size_t)g.stride;
    char *base = NL + (size_t)(par * 4 + mu) * 24 * S;
    short2 q[6];
    for (int e = 0; e < 6; e++) {
        const double2 u = fat[((size_t)mu * V + i) * 9 + e];
        q[e] = nl_pack<short2>(sgn * u.x, sgn * u.y, inv_scale);
    }
    short2 *p4 = (short2 *)base + (size_t)(i >> 1) * 4;
    for (int e = 0; e < 4; e++)
        p4[e] = q[e];
    short2 *p2 = (short2 *)(base + 16 * S) + (size_t)(i >> 1) * 2;
    p2[0] = q[4];
    p2[1] = q[5];
}

size_t net_links12_bytes(const Geom &g) { return (size_t)2 * 4 * 24 * (size_t)g.stride; }

cudaError_t launch_net_links12(const Geom &g, const double bc[4], const double *fat, void *NL12, float inv_scale16,
                               cudaStream_t s) {
    const long long n = 8LL * g.Vh;
    const unsigned grid = (unsigned)((n + 255) / 256);
    net_links12_kernel<<<grid, 256, 0, s>>>(g, bc[0], bc[1], bc[2], bc[3], (const double2 *)fat, (char *)NL12,
                                            inv_scale16);
    return cudaGetLastError();
}

cudaError_t launch_net_links_cb(const Geom &g, const double bc[4], const double *fat, float2 *NL32, short2 *NL16,
                                float inv_scale16, cudaStream_t s) {
    const long long n = 8LL * g.Vh;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (NL32)
        net_links_cb_kernel<float2><<<grid, 256, 0, s>>>(g, bc[0], bc[1], bc[2], bc[3], (const double2 *)fat,
                                                         NL32, 1.f);
    if (NL16)
        net_links_cb_kernel<short2><<<grid, 256, 0, s>>>(g, bc[0], bc[1], bc[2], bc[3], (const double2 *)fat,
                                                         NL16, inv_scale16);
    return cudaGetLastError();
}

// ---- path coefficients from the layer weights ------------------------------
// w: the weights as FP32 (re, im) pairs, layers at complex offsets off[0..2]
// (W1 [9][C][1], W2 [9][C][C], W3 [9][1][C]); round_half rounds each weight
// through binary16 first (the deployed preconditioner's weight storage).
struct NetW {
    const float2 *w;
    int C, off1, off2, round_half;
    const double2 *sw = nullptr;  // the weights staged in shared memory, if set
    STAG_D double2 load(int k) const {
        float2 v = w[k];
        if (round_half)
            v = make_float2(__half2float(__float2half_rn(v.x)), __half2float(__float2half_rn(v.y)));
        return make_double2((double)v.x, (double)v.y);
    }
    STAG_D double2 get(int k) const { return sw ? sw[k] : load(k); }
    STAG_D double2 w1(int d, int i) const { return get(d * C + i); }
    STAG_D double2 w2(int d, int j, int i) const { return get(off1 + (d * C + j) * C + i); }
    STAG_D double2 w3(int d, int j) const { return get(off2 + d * C + j); }
};

STAG_D double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
STAG_D double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
STAG_D double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// W3[d3] . W2[d2] . W1[d1]
STAG_D double2 triple(const NetW &W, int d3, int d2, int d1) {
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < W.C; j++) {
        double2 t = make_double2(0.0, 0.0);
        for (int i = 0; i < W.C; i++)
            t = zadd(t, zmul(W.w2(d2, j, i), W.w1(d1, i)));
        s = zadd(s, zmul(W.w3(d3, j), t));
    }
    return s;
}

// one block: the weights go to shared memory, then thread a*8+b computes
// C[a][b] and thread 64 c0
constexpr int NET_MAX_W = 9 * (2 * 8 + 8 * 8);

// hermitian: the coefficients of (N + N^+)/2 instead.  T_a^+ = T_abar (abar
// = a ^ 1, the reversed hop), so N^+ has conj(c0) and the coefficient
// conj(C[bbar][abar]) on T_a T_b.
__global__ void net_path_coef_kernel(NetW W, int hermitian, NetPath *out) {
    __shared__ double2 sw[NET_MAX_W];
    __shared__ double2 sc[65];
    const int nw = 9 * (2 * W.C + W.C * W.C);
    for (int k = threadIdx.x; k < nw; k += blockDim.x)
        sw[k] = W.load(k);
    __syncthreads();
    W.sw = sw;
    const int q = threadIdx.x;
    if (q < 64) {
        const int a = q >> 3, b = q & 7;
        sc[q] = zadd(zadd(triple(W, 0, a + 1, b + 1), triple(W, a + 1, 0, b + 1)), triple(W, a + 1, b + 1, 0));
    } else if (q == 64) {
        sc[64] = triple(W, 0, 0, 0);
    }
    __syncthreads();
    if (q < 64) {
        double2 v = sc[q];
        if (hermitian) {
            const int a = q >> 3, b = q & 7;
            const double2 t = sc[(b ^ 1) * 8 + (a ^ 1)];
            v = make_double2(0.5 * (v.x + t.x), 0.5 * (v.y - t.y));
        }
        out->C[q] = make_float2((float)v.x, (float)v.y);
    } else if (q == 64) {
        const double2 v = sc[64];
        out->c0 = make_float2((float)v.x, hermitian ? 0.f : (float)v.y);
    }
}

cudaError_t launch_net_path_coef(int C, const float *w32, const int off[3], int round_half, NetPath *out,
                                 cudaStream_t s, int hermitian) {
    NetW W{(const float2 *)w32, C, off[1], off[2], round_half};
    net_path_coef_kernel<<<1, 96, 0, s>>>(W, hermitian, out);
    return cudaGetLastError();
}

// dL/dW* of every complex weight from G[a*8+b] = dL/dC[a][b]* and G[64] =
// dL/dc0* (C holomorphic in W: dL/dW* = sum conj(dC/dW) dL/dC*); added to grad
__global__ void net_path_chain_kernel(NetW W, int nw, const double2 *__restrict__ G, double2 *grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nw)
        return;
    const int C = W.C;
    const double2 G0 = G[64];
    double2 acc = make_double2(0.0, 0.0);
    auto add = [&](double2 coef, double2 gv) { acc = zadd(acc, zmul(zconj(coef), gv)); };
    if (k < W.off1) {  // W1[d][i]
        const int d = k / C, i = k % C;
        // sum_j W3[d3][j] W2[d2][j][i]
        auto s32 = [&](int d3, int d2) {
            double2 t = make_double2(0.0, 0.0);
            for (int j = 0; j < C; j++)
                t = zadd(t, zmul(W.w3(d3, j), W.w2(d2, j, i)));
            return t;
        };
        if (d == 0) {
            add(s32(0, 0), G0);
            for (int a = 0; a < 8; a++)
                for (int b = 0; b < 8; b++)
                    add(s32(a + 1, b + 1), G[a * 8 + b]);
        } else {
            const int b = d - 1;
            for (int a = 0; a < 8; a++)
                add(zadd(s32(0, a + 1), s32(a + 1, 0)), G[a * 8 + b]);
        }
    } else if (k < W.off2) {  // W2[d][j][i]
        const int q = k - W.off1;
        const int d = q / (C * C), j = (q / C) % C, i = q % C;
        if (d == 0) {
            add(zmul(W.w3(0, j), W.w1(0, i)), G0);
            for (int a = 0; a < 8; a++)
                for (int b = 0; b < 8; b++)
                    add(zmul(W.w3(a + 1, j), W.w1(b + 1, i)), G[a * 8 + b]);
        } else {
            const int e = d - 1;
            for (int b = 0; b < 8; b++)  // W2 as the outer hop, layer 3 idle
                add(zmul(W.w3(0, j), W.w1(b + 1, i)), G[e * 8 + b]);
            for (int a = 0; a < 8; a++)  // W2 as the inner hop, layer 1 idle
                add(zmul(W.w3(a + 1, j), W.w1(0, i)), G[a * 8 + e]);
        }
    } else {  // W3[d][j]
        const int q = k - W.off2;
        const int d = q / C, j = q % C;
        // sum_i W2[d2][j][i] W1[d1][i]
        auto s21 = [&](int d2, int d1) {
            double2 t = make_double2(0.0, 0.0);
            for (int i = 0; i < C; i++)
                t = zadd(t, zmul(W.w2(d2, j, i), W.w1(d1, i)));
            return t;
        };
        if (d == 0) {
            add(s21(0, 0), G0);
            for (int a = 0; a < 8; a++)
                for (int b = 0; b < 8; b++)
                    add(s21(a + 1, b + 1), G[a * 8 + b]);
        } else {
            const int a = d - 1;
            for (int b = 0; b < 8; b++)
                add(zadd(s21(0, b + 1), s21(b + 1, 0)), G[a * 8 + b]);
        }
    }
    grad[k] = zadd(grad[k], acc);
}

cudaError_t launch_net_path_chain(int C, const float *w32, const int off[3], const double2 *G, double2 *grad,
                                  cudaStream_t s) {
    NetW W{(const float2 *)w32, C, off[1], off[2], 0};
    const int nw = 9 * (2 * C + C * C);
    net_path_chain_kernel<<<(nw + 127) / 128, 128, 0, s>>>(W, nw, G, grad);
    return cudaGetLastError();
}

// ---- the two stencil passes --------------------------------------------------
constexpr int NET_BLOCK = 128;

template <class R> STAG_D cplx<float> to_f(const cplx<R> &v) { return cconv<float, R>(v); }

// The odd-site intermediate chi: FP32 (float2 [8][3][S]) with FP32 links,
// and 16-bit with 16-bit links: one 16-byte cell per channel and site,
// int4 [8][S], the three components as int16 pairs and the norm (value =
// q * norm / 32767; the norm is the channel's largest |component| there).
template <class LT> struct Chi;
template <> struct Chi<float2> {
    STAG_D static void store(void *chi, int S, int a, int c, const cplx<float> v[3]) {
        float2 *p = (float2 *)chi;
#pragma unroll
        for (int k = 0; k < 3; k++)
            __stcs(p + (size_t)(a * 3 + k) * S + c, make_float2(v[k].re, v[k].im));
    }
    // v = chi_a at site j; returns the factor that turns v into values
    STAG_D static float load(const void *chi, int S, int a, int j, cplx<float> v[3]) {
        const float2 *p = (const float2 *)chi;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float2 t = __ldcs(p + (size_t)(a * 3 + k) * S + j);
            v[k] = cplx<float>{t.x, t.y};
        }
        return 1.f;
    }
};
template <> struct Chi<short2> {
    STAG_D static void store(void *chi, int S, int a, int c, const cplx<float> v[3]) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++)
            m = fmaxf(m, fmaxf(fabsf(v[k].re), fabsf(v[k].im)));
        const float inv = m > 0.f ? kQ16 / m : 0.f;
        __stcs((int4 *)chi + (size_t)a * S + c,
               make_int4(q16_pair(v[0].re * inv, v[0].im * inv), q16_pair(v[1].re * inv, v[1].im * inv),
                         q16_pair(v[2].re * inv, v[2].im * inv), __float_as_int(m)));
    }
    STAG_D static float load(const void *chi, int S, int a, int j, cplx<float> v[3]) {
        const int4 t = __ldcs((const int4 *)chi + (size_t)a * S + j);
        v[0] = cplx<float>{q_lo(t.x), q_hi(t.x)};
        v[1] = cplx<float>{q_lo(t.y), q_hi(t.y)};
        v[2] = cplx<float>{q_lo(t.z), q_hi(t.z)};
        return __int_as_float(t.w) * (1.f / kQ16);
    }
};
template <> struct Chi<L12> : Chi<short2> {};

// chi_a(y) = sum_b C[a][b] (T_b r)(y) on the odd sites; r even (precision P,
// component stride rs).  Hop index b = 2 mu (+mu) or 2 mu + 1 (-mu).  ls: the
// links' scale (1 for FP32).  The eight transported vectors go to shared
// memory first (each thread reads back only its own), so that the loads of
// the transport phase and the mixing's 48 live values never meet.
// Six resident blocks (at most 80 registers, 24 warps per SM): at eight the
// 16-bit form spills 96 bytes, and measured at 32^3x64 the solver-form net
// application took 0.342 ms against 0.308 ms at six.
constexpr int NET_MID_MINB = 6;

template <int P, class LT>
__global__ void __launch_bounds__(NET_BLOCK, NET_MID_MINB)
net_mid_kernel(Geom g, const LT *__restrict__ NL, float ls, int bcneg, const NetPath *__restrict__ path,
               const typename Fmt<P>::Elem *__restrict__ r, int rs, void *__restrict__ chi, const int *gate) {
    __shared__ cplx<float> sC[64];
    __shared__ float2 sh[8][3][NET_BLOCK];
    if (gate && *gate != CG_RUNNING)
        return;
    if (threadIdx.x < 64) {
        const float2 v = path->C[threadIdx.x];
        sC[threadIdx.x] = cplx<float>{v.x * ls, v.y * ls};
    }
    __syncthreads();
    const int c = blockIdx.x * NET_BLOCK + threadIdx.x;
    if (c >= g.Vh)
        return;
    const int S = g.stride;
    int x[4];
    cb_coords(g, c, 1, x);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
#pragma unroll
        for (int bw = 0; bw < 2; bw++) {
            // +mu: U_mu(y) r(y+mu), the link of this odd site;
            // -mu: U_mu(y-mu)^+ r(y-mu), the link of the even neighbour
            const int j = cb_hop(g, c, x, mu, bw ? -1 : 1);
            cplx<typename Fmt<P>::R> vr[3];
            load_vec<P>(r, rs, j, vr);
            cplx<float> v[3], U[9], h[3];
#pragma unroll
            for (int k = 0; k < 3; k++)
                v[k] = to_f(vr[k]);
            net_link(NL, S, bw ? 0 : 1, mu, bw ? j : c, g, x, bw, ls, bcneg, U);
            nl_apply(U, bw, v, h);
#pragma unroll
            for (int k = 0; k < 3; k++)
                sh[2 * mu + bw][k][threadIdx.x] = make_float2(h[k].re, h[k].im);
        }
    }
    if constexpr (std::is_same<LT, float2>::value) {
        // FP32 links (training): the scalar mixing, channel by channel
        cplx<float> h[8][3];
#pragma unroll
        for (int b = 0; b < 8; b++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float2 t = sh[b][k][threadIdx.x];
                h[b][k] = cplx<float>{t.x, t.y};
            }
#pragma unroll
        for (int a = 0; a < 8; a++) {
            cplx<float> acc[3] = {czero<float>(), czero<float>(), czero<float>()};
#pragma unroll
            for (int b = 0; b < 8; b++) {
                const cplx<float> w = sC[a * 8 + b];
#pragma unroll
                for (int k = 0; k < 3; k++)
                    cmac(acc[k], w, h[b][k]);
            }
            Chi<LT>::store(chi, S, a, c, acc);
        }
        return;
    }
    // 16-bit links (the solver's form): the mixing, four output channels at
    // a time and b outermost:
    // acc[a][k] = sum_b C[a][b] h_b[k] with each accumulator's (re, im) in
    // one packed FP32x2 register pair, so that a complex multiply-add is two
    // packed FMAs, w.re (h.re, h.im) and w.im (-h.im, h.re), in the order of
    // a scalar complex multiply-add
#pragma unroll
    for (int a0 = 0; a0 < 8; a0 += 4) {
        float2 acc[4][3];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++)
                acc[a][k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            float2 hb[3], hs[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                hb[k] = sh[b][k][threadIdx.x];
                hs[k] = make_float2(-hb[k].y, hb[k].x);
            }
#pragma unroll
            for (int a = 0; a < 4; a++) {
                const cplx<float> w = sC[(a0 + a) * 8 + b];
                const float2 wr = make_float2(w.re, w.re), wi = make_float2(w.im, w.im);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    acc[a][k] = __ffma2_rn(wr, hb[k], acc[a][k]);
                    acc[a][k] = __ffma2_rn(wi, hs[k], acc[a][k]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const cplx<float> v[3] = {cplx<float>{acc[a][0].x, acc[a][0].y}, cplx<float>{acc[a][1].x, acc[a][1].y},
                                      cplx<float>{acc[a][2].x, acc[a][2].y}};
            Chi<LT>::store(chi, S, a0 + a, c, v);
        }
    }
}

// z(x) = c0 r(x) + sum_a (T_a chi_a)(x) on the even sites.  NET_OUT_DOTS
// adds per-block partials of Re<z, r> (partial[blk]) and Re<z, Ap>
// (partial[nblk + blk]; 0 without Ap) for the flexible CG.
enum { NET_OUT_PLAIN = 0, NET_OUT_DOTS = 1 };

template <int PI, int PO, class LT, int EPI>
__global__ void __launch_bounds__(NET_BLOCK)
net_out_kernel(Geom g, const LT *__restrict__ NL, float ls, int bcneg, const NetPath *__restrict__ path,
               const void *__restrict__ chi, const typename Fmt<PI>::Elem *__restrict__ r, int rs,
               typename Fmt<PO>::Elem *__restrict__ z, int zs, const typename Fmt<PO>::Elem *__restrict__ Ap,
               double *partial, const int *gate) {
    using RO = typename Fmt<PO>::R;
    __shared__ double smem[32];
    if (gate && *gate != CG_RUNNING)
        return;
    const int c = blockIdx.x * NET_BLOCK + threadIdx.x;
    const int S = g.stride;
    red_t<RO> d0 = red_zero<red_t<RO>>(), d1 = red_zero<red_t<RO>>();
    if (c < g.Vh) {
        int x[4];
        cb_coords(g, c, 0, x);
        cplx<float> acc[3] = {czero<float>(), czero<float>(), czero<float>()};
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
#pragma unroll
            for (int bw = 0; bw < 2; bw++) {
                // +mu: U_mu(x) chi_{+mu}(x+mu); -mu: U_mu(x-mu)^+ chi_{-mu}(x-mu)
                const int j = cb_hop(g, c, x, mu, bw ? -1 : 1);
                cplx<float> v[3], U[9], h[3];
                const float f = Chi<LT>::load(chi, S, 2 * mu + bw, j, v);
                net_link(NL, S, bw ? 1 : 0, mu, bw ? j : c, g, x, bw, ls, bcneg, U);
                nl_apply(U, bw, v, h);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    acc[k].re = fmaf(f, h[k].re, acc[k].re);
                    acc[k].im = fmaf(f, h[k].im, acc[k].im);
                }
            }
        }
        const float2 c0 = path->c0;
        cplx<typename Fmt<PI>::R> rv[3];
        load_vec<PI>(r, rs, c, rv);
        cplx<RO> zo[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const cplx<float> rf = to_f(rv[k]);
            cplx<float> zf = cplx<float>{acc[k].re * ls, acc[k].im * ls};
            cmac(zf, cplx<float>{c0.x, c0.y}, rf);
            zo[k] = cplx<RO>{rconv<RO, float>(zf.re), rconv<RO, float>(zf.im)};
        }
        store_vec<PO>(z, zs, c, zo);
        if (EPI == NET_OUT_DOTS) {
            cplx<RO> ro[3];
#pragma unroll
            for (int k = 0; k < 3; k++)
                ro[k] = cconv<RO, typename Fmt<PI>::R>(rv[k]);
            d0 = re_dot3<RO>(zo, ro);
            if (Ap) {
                cplx<RO> av[3];
                load_vec<PO>(Ap, zs, c, av);
                d1 = re_dot3<RO>(zo, av);
            }
        }
    }
    if (EPI == NET_OUT_DOTS) {
        const double s0 = block_sum<NET_BLOCK>(d0, smem);
        const double s1 = block_sum<NET_BLOCK>(d1, smem);
        if (threadIdx.x == 0) {
            partial[blockIdx.x] = s0;
            partial[gridDim.x + blockIdx.x] = s1;
        }
    }
}

int net_grid(const Geom &g) { return (g.Vh + NET_BLOCK - 1) / NET_BLOCK; }

#define NP_IN_SWITCH(prec, ...)                                            \
    switch (prec) {                                                        \
    case P_F64: { constexpr int P = P_F64; __VA_ARGS__; } break;           \
    case P_DF64: { constexpr int P = P_DF64; __VA_ARGS__; } break;         \
    case P_F32: { constexpr int P = P_F32; __VA_ARGS__; } break;           \
    case P_F16: { constexpr int P = P_F16; __VA_ARGS__; } break;           \
    default: return cudaErrorInvalidValue;                                 \
    }

cudaError_t launch_net_mid(int prec, const Geom &g, const NetLinkSet &nl, const NetPath *path, const void *r,
                           int rs, void *chi, const int *gate, cudaStream_t s) {
    NP_IN_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        if (nl.l12)
            net_mid_kernel<P, L12><<<net_grid(g), NET_BLOCK, 0, s>>>(g, (const L12 *)nl.l12, nl.scale16, nl.bcneg,
                                                                      path, (const E *)r, rs, chi, gate);
        else if (nl.l16)
            net_mid_kernel<P, short2><<<net_grid(g), NET_BLOCK, 0, s>>>(g, nl.l16, nl.scale16, nl.bcneg, path,
                                                                         (const E *)r, rs, chi, gate);
        else
            net_mid_kernel<P, float2><<<net_grid(g), NET_BLOCK, 0, s>>>(g, nl.l32, 1.f, nl.bcneg, path,
                                                                         (const E *)r, rs, chi, gate);
    });
    return cudaGetLastError();
}

template <int PI, int PO, int EPI>
static void net_out_t(const Geom &g, const NetLinkSet &nl, const NetPath *path, const void *chi, const void *r,
                      int rs, void *z, int zs, const void *Ap, double *partial, const int *gate, cudaStream_t s) {
    using EI = typename Fmt<PI>::Elem;
    using EO = typename Fmt<PO>::Elem;
    if (nl.l12)
        net_out_kernel<PI, PO, L12, EPI><<<net_grid(g), NET_BLOCK, 0, s>>>(
            g, (const L12 *)nl.l12, nl.scale16, nl.bcneg, path, chi, (const EI *)r, rs, (EO *)z, zs,
            (const EO *)Ap, partial, gate);
    else if (nl.l16)
        net_out_kernel<PI, PO, short2, EPI><<<net_grid(g), NET_BLOCK, 0, s>>>(
            g, nl.l16, nl.scale16, nl.bcneg, path, chi, (const EI *)r, rs, (EO *)z, zs, (const EO *)Ap, partial,
            gate);
    else
        net_out_kernel<PI, PO, float2, EPI><<<net_grid(g), NET_BLOCK, 0, s>>>(
            g, nl.l32, 1.f, nl.bcneg, path, chi, (const EI *)r, rs, (EO *)z, zs, (const EO *)Ap, partial, gate);
}

// input and output of one precision (the solver's), or FP32 pair input with
// FP32 output (training)
cudaError_t launch_net_out(int prec_in, int prec_out, const Geom &g, const NetLinkSet &nl, const NetPath *path,
                           const void *chi, const void *r, int rs, void *z, int zs, bool dots, const void *Ap,
                           double *partial, const int *gate, cudaStream_t s) {
    if (prec_in != prec_out)
        return cudaErrorInvalidValue;
    NP_IN_SWITCH(prec_in, {
        if (dots)
            net_out_t<P, P, NET_OUT_DOTS>(g, nl, path, chi, r, rs, z, zs, Ap, partial, gate, s);
        else
            net_out_t<P, P, NET_OUT_PLAIN>(g, nl, path, chi, r, rs, z, zs, nullptr, nullptr, gate, s);
    });
    return cudaGetLastError();
}

// ---- training: dL/dC[a][b]* and dL/dc0* ----------------------------------------
// Per odd site y: h_b = (T_b r)(y), k_a = (T_a^+ g)(y); the block gathers a
// tile of NET_BLOCK sites in shared memory (site index fastest) and warp w
// adds the 4 x 4 pairs (a in 4 (w >> 1) .. +3, b in 4 (w & 1) .. +3) of
// conj(h_b) k_a over the tile; each thread also adds conj(r) g of the even
// site with its checkerboard index (the c0 term).  One partial per block and
// pair, in double: partial[blk * 65 + q].
constexpr int GRAD_BLOCKS = 1024;

__global__ void __launch_bounds__(NET_BLOCK)
net_grad_kernel(Geom g, const float2 *__restrict__ NL, const float2 *__restrict__ r, int rs,
                const float2 *__restrict__ gv, int gs, double2 *partial) {
    static_assert(NET_BLOCK == 128, "four warps: one per 4 x 4 block of hop pairs");
    __shared__ float2 H[8][3][NET_BLOCK];
    __shared__ float2 K[8][3][NET_BLOCK];
    const int S = g.stride;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a0 = 4 * (warp >> 1), b0 = 4 * (warp & 1);
    cplx<float> acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            acc[i][j] = czero<float>();
    cplx<float> acc0 = czero<float>();
    for (int base = blockIdx.x * NET_BLOCK; base < g.Vh; base += gridDim.x * NET_BLOCK) {
        const int c = base + threadIdx.x;
        if (c < g.Vh) {
            int x[4];
            cb_coords(g, c, 1, x);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                const int jf = cb_hop(g, c, x, mu, 1), jb = cb_hop(g, c, x, mu, -1);
                cplx<float> Uf[9], Ub[9], v[3], h[3];
                nl_load(NL, S, 1, mu, c, Uf);
                nl_load(NL, S, 0, mu, jb, Ub);
                // h_{+mu} = Uf r(y+mu), h_{-mu} = Ub^+ r(y-mu)
                // k_{+mu} = T_{-mu} g = Ub^+ g(y-mu), k_{-mu} = T_{+mu} g = Uf g(y+mu)
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const bool bwd = q & 1;
                    const float2 *src = q < 2 ? r : gv;
                    const int st = q < 2 ? rs : gs;
                    const int j = ((q == 0) || (q == 3)) ? jf : jb;
                    const bool use_b = (q == 1) || (q == 2);
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const float2 t = __ldg(src + (size_t)k * st + j);
                        v[k] = cplx<float>{t.x, t.y};
                    }
                    nl_apply(use_b ? Ub : Uf, use_b, v, h);
                    // q: 0 h_{+mu}, 1 h_{-mu}, 2 k_{+mu}, 3 k_{-mu}
                    const int idx = 2 * mu + (bwd ? 1 : 0);
                    float2(*dst)[3][NET_BLOCK] = q < 2 ? H : K;
#pragma unroll
                    for (int k = 0; k < 3; k++)
                        dst[idx][k][threadIdx.x] = make_float2(h[k].re, h[k].im);
                }
            }
            // c0 term on the even site with this checkerboard index
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float2 rv = __ldg(r + (size_t)k * rs + c), gg = __ldg(gv + (size_t)k * gs + c);
                cmac_conj(acc0, cplx<float>{rv.x, rv.y}, cplx<float>{gg.x, gg.y});
            }
        } else {
#pragma unroll
            for (int b = 0; b < 8; b++)
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    H[b][k][threadIdx.x] = make_float2(0.f, 0.f);
                    K[b][k][threadIdx.x] = make_float2(0.f, 0.f);
                }
        }
        __syncthreads();
#pragma unroll 1
        for (int s = lane; s < NET_BLOCK; s += 32) {
#pragma unroll
            for (int k = 0; k < 3; k++) {
                cplx<float> hb[4], ka[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const float2 t = H[b0 + i][k][s];
                    hb[i] = cplx<float>{t.x, t.y};
                    const float2 u = K[a0 + i][k][s];
                    ka[i] = cplx<float>{u.x, u.y};
                }
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        cmac_conj(acc[i][j], hb[j], ka[i]);
            }
        }
        __syncthreads();
    }
    // warp sums in double, fixed order; acc[i][j] is the pair (a0 + i, b0 + j)
    double2 *out = partial + (size_t)blockIdx.x * 65;
#pragma unroll 1
    for (int i = 0; i < 4; i++)
#pragma unroll 1
        for (int j = 0; j < 4; j++) {
            double re = acc[i][j].re, im = acc[i][j].im;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_down_sync(0xffffffffu, re, o);
                im += __shfl_down_sync(0xffffffffu, im, o);
            }
            if (lane == 0)
                out[(a0 + i) * 8 + b0 + j] = make_double2(re, im);
        }
    double re0 = acc0.re, im0 = acc0.im;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re0 += __shfl_down_sync(0xffffffffu, re0, o);
        im0 += __shfl_down_sync(0xffffffffu, im0, o);
    }
    // the tile is no longer read (the loop ended with a barrier)
    double2 *red = reinterpret_cast<double2 *>(&H[0][0][0]);
    if (lane == 0)
        red[warp] = make_double2(re0, im0);
    __syncthreads();
    if (threadIdx.x == 0)
        out[64] = make_double2((red[0].x + red[1].x) + (red[2].x + red[3].x),
                               (red[0].y + red[1].y) + (red[2].y + red[3].y));
}

// G[q] += sum over blocks of partial[blk * 65 + q]: block q sums its
// coefficient, thread t the blocks t, t + 256, ... in order, then the block
// tree (a fixed order, so the sum is the same on every run).  One thread per
// coefficient summing all blocks serially took 160 us per call at 32^3x64.
constexpr int GRAD_FINISH_BLOCK = 256;

__global__ void __launch_bounds__(GRAD_FINISH_BLOCK)
net_grad_finish_kernel(const double2 *__restrict__ partial, int nblk, double2 *G) {
    __shared__ double smem[32];
    const int q = blockIdx.x;
    double tx = 0.0, ty = 0.0;
    for (int b = threadIdx.x; b < nblk; b += GRAD_FINISH_BLOCK) {
        const double2 v = partial[(size_t)b * 65 + q];
        tx += v.x;
        ty += v.y;
    }
    tx = block_sum<GRAD_FINISH_BLOCK>(tx, smem);
    ty = block_sum<GRAD_FINISH_BLOCK>(ty, smem);
    if (threadIdx.x == 0) {
        G[q].x += tx;
        G[q].y += ty;
    }
}

int net_grad_blocks(const Geom &g) {
    const int need = (g.Vh + NET_BLOCK - 1) / NET_BLOCK;
    return need < GRAD_BLOCKS ? need : GRAD_BLOCKS;
}

cudaError_t launch_net_grad(const Geom &g, const float2 *NL32, const float2 *r, int rs, const float2 *gv, int gs,
                            double2 *partial, double2 *G, cudaStream_t s) {
    const int nb = net_grad_blocks(g);
    net_grad_kernel<<<nb, NET_BLOCK, 0, s>>>(g, NL32, r, rs, gv, gs, partial);
    net_grad_finish_kernel<<<65, GRAD_FINISH_BLOCK, 0, s>>>(partial, nb, G);
    return cudaGetLastError();
}

// ---- losses on the even sites (FP32) -----------------------------------------
// error loss: g = (z - e) / |e|^2, *loss += |z - e|^2 / |e|^2 (z, g: stride zs;
// e: stride es)
// Loss and dot sums: each site's six products are summed in FP32, the sites
// of a thread and the block tree in double float (FP32 pipe), one FP64
// value and one atomic per block.  Accumulated in FP64 per element, with one
// atomic per warp, these kernels took 66-73 us per call at 32^3x64, bound by
// the FP64 pipe (1/64 of the FP32 rate).
constexpr int NET_SUM_BLOCK = 256;

__global__ void __launch_bounds__(NET_SUM_BLOCK)
net_error_loss_kernel(int Vh, const float2 *__restrict__ z, int zs, const float2 *__restrict__ e, int es,
                      const double *enorm2, float2 *gv, double *loss) {
    __shared__ double smem[32];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const double n2 = *enorm2;
    float part = 0.f;
    if (c < Vh) {
        // a pair with e = 0 carries no information: no loss, no gradient
        const float inv = n2 > 0.0 ? (float)(1.0 / n2) : 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float2 zv = z[(size_t)k * zs + c], ev = e[(size_t)k * es + c];
            const float2 d = make_float2(zv.x - ev.x, zv.y - ev.y);
            part = fmaf(d.x, d.x, fmaf(d.y, d.y, part));
            gv[(size_t)k * zs + c] = make_float2(d.x * inv, d.y * inv);
        }
    }
    const double tot = block_sum<NET_SUM_BLOCK>(df_make(part, 0.f), smem);
    if (threadIdx.x == 0 && tot != 0.0 && n2 > 0.0)
        atomicAdd(loss, tot / n2);
}

// residual loss: q = (Mz - r) / |r|^2 written over mz, *loss += |Mz - r|^2 / |r|^2
__global__ void __launch_bounds__(NET_SUM_BLOCK)
net_resid_loss_kernel(int Vh, float2 *mz, int ms, const float2 *__restrict__ r, int rs,
                      const double *rnorm2, double *loss) {
    __shared__ double smem[32];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const double n2 = *rnorm2;
    float part = 0.f;
    if (c < Vh) {
        const float inv = n2 > 0.0 ? (float)(1.0 / n2) : 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float2 m = mz[(size_t)k * ms + c], rv = r[(size_t)k * rs + c];
            const float2 q = make_float2(m.x - rv.x, m.y - rv.y);
            part = fmaf(q.x, q.x, fmaf(q.y, q.y, part));
            mz[(size_t)k * ms + c] = make_float2(q.x * inv, q.y * inv);
        }
    }
    const double tot = block_sum<NET_SUM_BLOCK>(df_make(part, 0.f), smem);
    if (threadIdx.x == 0 && tot != 0.0 && n2 > 0.0)
        atomicAdd(loss, tot / n2);
}

// out[0] += Re<a, b>, out[1] += |a|^2 (even FP32 vectors of strides as, bs)
__global__ void __launch_bounds__(NET_SUM_BLOCK)
net_dot2_kernel(int Vh, const float2 *__restrict__ a, int as, const float2 *__restrict__ b, int bs, double *out) {
    __shared__ double smem[32];
    df p0 = df_zero(), p1 = df_zero();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < Vh; c += gridDim.x * blockDim.x) {
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float2 x = a[(size_t)k * as + c], y = b[(size_t)k * bs + c];
            s0 = fmaf(x.x, y.x, fmaf(x.y, y.y, s0));
            s1 = fmaf(x.x, x.x, fmaf(x.y, x.y, s1));
        }
        p0 = df_add(p0, df_make(s0, 0.f));
        p1 = df_add(p1, df_make(s1, 0.f));
    }
    const double t0 = block_sum<NET_SUM_BLOCK>(p0, smem);
    const double t1 = block_sum<NET_SUM_BLOCK>(p1, smem);
    if (threadIdx.x == 0) {
        atomicAdd(out, t0);
        atomicAdd(out + 1, t1);
    }
}

cudaError_t launch_net_error_loss(int Vh, const float2 *z, int zs, const float2 *e, int es, const double *enorm2,
                                  float2 *gv, double *loss, cudaStream_t s) {
    net_error_loss_kernel<<<(Vh + NET_SUM_BLOCK - 1) / NET_SUM_BLOCK, NET_SUM_BLOCK, 0, s>>>(Vh, z, zs, e, es,
                                                                                         enorm2, gv, loss);
    return cudaGetLastError();
}

cudaError_t launch_net_resid_loss(int Vh, float2 *mz, int ms, const float2 *r, int rs, const double *rnorm2,
                                  double *loss, cudaStream_t s) {
    net_resid_loss_kernel<<<(Vh + NET_SUM_BLOCK - 1) / NET_SUM_BLOCK, NET_SUM_BLOCK, 0, s>>>(Vh, mz, ms, r, rs,
                                                                                         rnorm2, loss);
    return cudaGetLastError();
}

cudaError_t launch_net_dot2(int Vh, const float2 *a, int as, const float2 *b, int bs, double *out, cudaStream_t s) {
    net_dot2_kernel<<<4 * 152, NET_SUM_BLOCK, 0, s>>>(Vh, a, as, b, bs, out);
    return cudaGetLastError();
}

// ---- flexible CG ---------------------------------------------------------------
// After z = N(r) with the partials of Re<z, r> and Re<z, Ap> (net_out_kernel
// NET_OUT_DOTS or fcg_copy_dots_kernel): beta (Polak-Ribiere,
// <z_new, r_new - r_old> / <z_old, r_old> with r_new - r_old = -alpha Ap; or
// Fletcher-Reeves <z_new, r_new> / <z_old, r_old> after a reliable update,
// where r_new is the recomputed residual; 0 on the first step), rr = <z, r>.
constexpr int FCG_FINISH = 1024;

__global__ void __launch_bounds__(FCG_FINISH)
fcg_finish_kernel(const double *__restrict__ partial, int n, CgScalars *sc, int first) {
    __shared__ double smem[32];
    if (sc->status != CG_RUNNING)
        return;
    // two independent sums per value and thread over a fixed assignment
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    int i = threadIdx.x;
    for (; i + FCG_FINISH < n; i += 2 * FCG_FINISH) {
        a0 += partial[i];
        a1 += partial[i + FCG_FINISH];
        b0 += partial[n + i];
        b1 += partial[n + i + FCG_FINISH];
    }
    if (i < n) {
        a0 += partial[i];
        b0 += partial[n + i];
    }
    const double zr = block_sum<FCG_FINISH>(a0 + a1, smem);
    const double zap = block_sum<FCG_FINISH>(b0 + b1, smem);
    if (threadIdx.x == 0) {
        double beta = 0.0;
        if (!first)
            beta = sc->reliable ? zr / sc->rr : -sc->alpha.d * zap / sc->rr;
        sc->beta = make_dpair(beta);
        sc->rr = zr;
        if (!(zr > 0.0 && zr < INFINITY)) {
            // the preconditioned residual lost positivity
            sc->status = CG_BREAKDOWN;
            if (sc->has_cond)
                cudaGraphSetConditional(sc->cond, 0u);
        }
    }
}

cudaError_t launch_fcg_finish(const double *partial, int n, CgScalars *sc, int first, cudaStream_t s) {
    fcg_finish_kernel<<<1, FCG_FINISH, 0, s>>>(partial, n, sc, first);
    return cudaGetLastError();
}

// z = r with the partials of Re<z, r> and Re<z, Ap> (the flexible CG without
// the net: plain CG)
template <int P>
__global__ void __launch_bounds__(NET_BLOCK)
fcg_copy_dots_kernel(Geom g, const typename Fmt<P>::Elem *__restrict__ r, typename Fmt<P>::Elem *__restrict__ z,
                     const typename Fmt<P>::Elem *__restrict__ Ap, double *partial, const int *gate) {
    using R = typename Fmt<P>::R;
    __shared__ double smem[32];
    if (gate && *gate != CG_RUNNING)
        return;
    const int c = blockIdx.x * NET_BLOCK + threadIdx.x;
    red_t<R> d0 = red_zero<red_t<R>>(), d1 = red_zero<red_t<R>>();
    if (c < g.Vh) {
        cplx<R> rv[3], av[3];
        load_vec<P>(r, g.stride, c, rv);
        store_vec<P>(z, g.stride, c, rv);
        d0 = re_dot3<R>(rv, rv);
        if (Ap) {
            load_vec<P>(Ap, g.stride, c, av);
            d1 = re_dot3<R>(rv, av);
        }
    }
    const double s0 = block_sum<NET_BLOCK>(d0, smem);
    const double s1 = block_sum<NET_BLOCK>(d1, smem);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s0;
        partial[gridDim.x + blockIdx.x] = s1;
    }
}

cudaError_t launch_fcg_copy_dots(int prec, const Geom &g, const void *r, void *z, const void *Ap, double *partial,
                                 const int *gate, cudaStream_t s) {
    NP_IN_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        fcg_copy_dots_kernel<P><<<net_grid(g), NET_BLOCK, 0, s>>>(g, (const E *)r, (E *)z, (const E *)Ap, partial,
                                                                   gate);
    });
    return cudaGetLastError();
}

}  // namespace stag
