// Learned gauge-covariant preconditioner: convolution layers, their
// gradients, the training loss and optimiser, and the vector kernels of the
// flexible CG that applies it.  The paper has no learned preconditioner; the
// layer is a gauge-equivariant convolution (Lehner & Wettig's preconditioner
// networks for lattice QCD):
//
//   y_o(x) = sum_i [ W[0][o][i] psi_i(x)
//                    + sum_mu ( W[1+2mu][o][i] U_mu(x) psi_i(x+mu)
//                             + W[2+2mu][o][i] U_mu(x-mu)^+ psi_i(x-mu) ) ]
//
// on the full lattice with raw links U (the boundary sign of a wrapping hop
// folded into the last-slice links), complex colour-blind weights, channels
// as float2 planes [C][3][V] indexed by the lexicographic site.
#include "learned.cuh"
#include "kernels.h"

namespace stag {

STAG_D void net_coords(const NetGeom &g, int i, int x[4]) {
    x[0] = i % g.L[0];
    int r = i / g.L[0];
    x[1] = r % g.L[1];
    r /= g.L[1];
    x[2] = r % g.L[2];
    x[3] = r / g.L[2];
}

// full-lattice index of the neighbour one step along +-mu
STAG_D int net_hop(const NetGeom &g, int i, const int x[4], int mu, int s) {
    int d = s;
    const int y = x[mu] + s;
    if (y >= g.L[mu])
        d -= g.L[mu];
    else if (y < 0)
        d += g.L[mu];
    return i + d * g.step[mu];
}

// acc += w h (complex, four FMAs)
STAG_D void cmacf(float2 &acc, float2 w, float2 h) {
    acc.x = fmaf(w.x, h.x, acc.x);
    acc.x = fmaf(-w.y, h.y, acc.x);
    acc.y = fmaf(w.x, h.y, acc.y);
    acc.y = fmaf(w.y, h.x, acc.y);
}

// the link of one hop, U at Lp[e * V]
STAG_D void load_link9(const float2 *__restrict__ Lp, int V, float2 U[9]) {
#pragma unroll
    for (int e = 0; e < 9; e++)
        U[e] = __ldg(Lp + (size_t)e * V);
}

// h = U v (fwd) or U^+ v
STAG_D void apply_link(const float2 U[9], bool adj, const float2 v[3], float2 h[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const float2 u = adj ? make_float2(U[3 * b + a].x, -U[3 * b + a].y) : U[3 * a + b];
            re = fmaf(u.x, v[b].x, fmaf(-u.y, v[b].y, re));
            im = fmaf(u.x, v[b].y, fmaf(u.y, v[b].x, im));
        }
        h[a] = make_float2(re, im);
    }
}

// one layer; weights [9][COUT][CIN] rounded through binary16 when
// round_half (the FP16 weight storage of the deployed preconditioner)
// in_par >= 0: the input is zero off that parity, so a site of that parity
// needs only its own term and a site of the other parity only the hops;
// out_par >= 0: only sites of that parity are computed (one thread each)
template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
covconv_kernel(NetGeom g, const float2 *__restrict__ NL, const float2 *__restrict__ W, int round_half,
               const float2 *__restrict__ in, float2 *__restrict__ out, const int *gate, int in_par,
               int out_par) {
    __shared__ float2 sw[9 * COUT * CIN];
    if (gate && *gate != CG_RUNNING)
        return;
    for (int k = threadIdx.x; k < 9 * COUT * CIN; k += blockDim.x) {
        float2 w = W[k];
        if (round_half)
            w = make_float2(__half2float(__float2half_rn(w.x)), __half2float(__float2half_rn(w.y)));
        sw[k] = w;
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int V = g.V;
    int x[4], i;
    if (out_par < 0) {
        i = t;
        if (i >= V)
            return;
        net_coords(g, i, x);
    } else {
        if (t >= V / 2)
            return;
        // site t of parity out_par in checkerboard order
        const int lxh = g.L[0] / 2;
        const int xh = t % lxh;
        int r = t / lxh;
        x[1] = r % g.L[1];
        r /= g.L[1];
        x[2] = r % g.L[2];
        x[3] = r / g.L[2];
        x[0] = 2 * xh + ((out_par + x[1] + x[2] + x[3]) & 1);
        i = x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]));
    }
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const bool do_self = in_par < 0 || par == in_par;
    const bool do_hops = in_par < 0 || par != in_par;
    float2 acc[COUT][3];
#pragma unroll
    for (int o = 0; o < COUT; o++)
#pragma unroll
        for (int a = 0; a < 3; a++)
            acc[o][a] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int d = 0; d < 9; d++) {
        if (d == 0 ? !do_self : !do_hops)
            continue;
        const int mu = (d - 1) >> 1;
        const bool bwd = d > 0 && ((d - 1) & 1);
        const int j = d == 0 ? i : net_hop(g, i, x, mu, bwd ? -1 : 1);
        // the hop's link, loaded once for all channels
        float2 U[9];
        if (d > 0)
            load_link9(NL + (size_t)mu * 9 * V + (bwd ? j : i), V, U);
        if constexpr (COUT < CIN) {
            // transports commute with the colour-blind weights: mix the
            // input channels at the neighbour, then move COUT vectors
            float2 m[COUT][3];
#pragma unroll
            for (int o = 0; o < COUT; o++)
#pragma unroll
                for (int a = 0; a < 3; a++)
                    m[o][a] = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < CIN; c++) {
                float2 v[3];
#pragma unroll
                for (int a = 0; a < 3; a++)
                    v[a] = __ldg(in + ((size_t)c * 3 + a) * V + j);
#pragma unroll
                for (int o = 0; o < COUT; o++) {
                    const float2 w = sw[(d * COUT + o) * CIN + c];
#pragma unroll
                    for (int a = 0; a < 3; a++)
                        cmacf(m[o][a], w, v[a]);
                }
            }
#pragma unroll
            for (int o = 0; o < COUT; o++) {
                float2 h[3];
                if (d == 0) {
#pragma unroll
                    for (int a = 0; a < 3; a++)
                        h[a] = m[o][a];
                } else {
                    apply_link(U, bwd, m[o], h);
                }
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    acc[o][a].x += h[a].x;
                    acc[o][a].y += h[a].y;
                }
            }
        } else {
            // move each input channel, then mix into the outputs
#pragma unroll
            for (int c = 0; c < CIN; c++) {
                float2 v[3], h[3];
#pragma unroll
                for (int a = 0; a < 3; a++)
                    v[a] = __ldg(in + ((size_t)c * 3 + a) * V + j);
                if (d == 0) {
#pragma unroll
                    for (int a = 0; a < 3; a++)
                        h[a] = v[a];
                } else {
                    apply_link(U, bwd, v, h);
                }
#pragma unroll
                for (int o = 0; o < COUT; o++) {
                    const float2 w = sw[(d * COUT + o) * CIN + c];
#pragma unroll
                    for (int a = 0; a < 3; a++)
                        cmacf(acc[o][a], w, h[a]);
                }
            }
        }
    }
#pragma unroll
    for (int o = 0; o < COUT; o++)
#pragma unroll
        for (int a = 0; a < 3; a++)
            out[((size_t)o * 3 + a) * V + i] = acc[o][a];
}

// The same sum for layers with few channel pairs (one of CIN, COUT is 1):
// each thread keeps OB x CIN complex sums over a grid-stride loop of sites,
// the OB outputs of blockIdx.y's slice; per-block partial sums in double
template <int CIN, int COUT, int OB>
__global__ void __launch_bounds__(128)
covconv_wgrad_reg_kernel(NetGeom g, const float2 *__restrict__ NL, const float2 *__restrict__ in,
                     const float2 *__restrict__ gout, double2 *partial) {
    constexpr int NOB = (COUT + OB - 1) / OB;
    const int d = blockIdx.y / NOB;
    const int o0 = (blockIdx.y % NOB) * OB;
    const int V = g.V;
    const int mu = (d - 1) >> 1;
    const bool bwd = d > 0 && ((d - 1) & 1);
    float2 acc[OB][CIN];
#pragma unroll
    for (int o = 0; o < OB; o++)
#pragma unroll
        for (int c = 0; c < CIN; c++)
            acc[o][c] = make_float2(0.f, 0.f);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
        int x[4];
        net_coords(g, i, x);
        const int j = d == 0 ? i : net_hop(g, i, x, mu, bwd ? -1 : 1);
        float2 gv[OB][3];
#pragma unroll
        for (int o = 0; o < OB; o++)
#pragma unroll
            for (int a = 0; a < 3; a++)
                gv[o][a] = o0 + o < COUT ? __ldg(gout + ((size_t)(o0 + o) * 3 + a) * V + i) : make_float2(0.f, 0.f);
        float2 U[9];
        if (d > 0)
            load_link9(NL + (size_t)mu * 9 * V + (bwd ? j : i), V, U);
#pragma unroll
        for (int c = 0; c < CIN; c++) {
            float2 v[3], h[3];
#pragma unroll
            for (int a = 0; a < 3; a++)
                v[a] = __ldg(in + ((size_t)c * 3 + a) * V + j);
            if (d == 0) {
#pragma unroll
                for (int a = 0; a < 3; a++)
                    h[a] = v[a];
            } else {
                apply_link(U, bwd, v, h);
            }
#pragma unroll
            for (int o = 0; o < OB; o++)
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    // conj(h) * g
                    acc[o][c].x += h[a].x * gv[o][a].x + h[a].y * gv[o][a].y;
                    acc[o][c].y += h[a].x * gv[o][a].y - h[a].y * gv[o][a].x;
                }
        }
    }
    // block reduction of every accumulator, fixed order
    __shared__ float2 red[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
    for (int o = 0; o < OB; o++) {
#pragma unroll 1
        for (int c = 0; c < CIN; c++) {
            float2 v = acc[o][c];
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                v.x += __shfl_down_sync(0xffffffffu, v.x, s);
                v.y += __shfl_down_sync(0xffffffffu, v.y, s);
            }
            if (lane == 0)
                red[warp] = v;
            __syncthreads();
            if (threadIdx.x == 0 && o0 + o < COUT) {
                double2 t = make_double2(0.0, 0.0);
                for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
                    t.x += red[w].x;
                    t.y += red[w].y;
                }
                partial[((size_t)blockIdx.x * 9 + d) * COUT * CIN + (o0 + o) * CIN + c] = t;
            }
            __syncthreads();
        }
    }
}

// dL/dW*[d][o][i] = sum_x <T_d in_i (x), gout_o(x)>, hop d = blockIdx.y;
// per-block partial sums in double.  The sites are taken in tiles of
// WG_THREADS: each thread moves the CIN input channels of its site along the
// hop (the link loaded once) and loads the COUT output gradients there, into
// shared memory; then the CIN * COUT pairs (o, i), each taken by
// WG_THREADS / (CIN * COUT) threads, add their products over the tile.  A
// thread keeps one complex sum: the tile's in FP32, the running one in FP64.
constexpr int WG_THREADS = 128;

template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS)
covconv_wgrad_kernel(NetGeom g, const float2 *__restrict__ NL, const float2 *__restrict__ in,
                     const float2 *__restrict__ gout, double2 *partial) {
    constexpr int NP = CIN * COUT;
    static_assert(WG_THREADS % NP == 0, "pairs must divide the block");
    constexpr int NG = WG_THREADS / NP;  // threads per pair
    __shared__ float2 T[WG_THREADS][3][CIN];
    __shared__ float2 G[WG_THREADS][3][COUT];
    __shared__ double2 red[WG_THREADS];
    const int d = blockIdx.y;
    const int V = g.V;
    const int mu = (d - 1) >> 1;
    const bool bwd = d > 0 && ((d - 1) & 1);
    const int q = threadIdx.x % NP, grp = threadIdx.x / NP;
    const int o = q / CIN, ci = q % CIN;
    double2 sum = make_double2(0.0, 0.0);
    for (int base = blockIdx.x * WG_THREADS; base < V; base += gridDim.x * WG_THREADS) {
        // this thread's site: the moved inputs and the output gradients
        const int i = base + threadIdx.x;
        if (i < V) {
            int x[4];
            net_coords(g, i, x);
            const int j = d == 0 ? i : net_hop(g, i, x, mu, bwd ? -1 : 1);
            float2 U[9];
            if (d > 0)
                load_link9(NL + (size_t)mu * 9 * V + (bwd ? j : i), V, U);
#pragma unroll
            for (int c = 0; c < CIN; c++) {
                float2 v[3], h[3];
#pragma unroll
                for (int a = 0; a < 3; a++)
                    v[a] = __ldg(in + ((size_t)c * 3 + a) * V + j);
                if (d == 0) {
#pragma unroll
                    for (int a = 0; a < 3; a++)
                        h[a] = v[a];
                } else {
                    apply_link(U, bwd, v, h);
                }
#pragma unroll
                for (int a = 0; a < 3; a++)
                    T[threadIdx.x][a][c] = h[a];
            }
#pragma unroll
            for (int oo = 0; oo < COUT; oo++)
#pragma unroll
                for (int a = 0; a < 3; a++)
                    G[threadIdx.x][a][oo] = __ldg(gout + ((size_t)oo * 3 + a) * V + i);
        } else {
#pragma unroll
            for (int a = 0; a < 3; a++) {
#pragma unroll
                for (int c = 0; c < CIN; c++)
                    T[threadIdx.x][a][c] = make_float2(0.f, 0.f);
#pragma unroll
                for (int oo = 0; oo < COUT; oo++)
                    G[threadIdx.x][a][oo] = make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
        // pair (o, ci) over this thread's share of the tile: conj(h) g
        float2 t = make_float2(0.f, 0.f);
        for (int sidx = grp; sidx < WG_THREADS; sidx += NG) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float2 h = T[sidx][a][ci], gv = G[sidx][a][o];
                t.x = fmaf(h.x, gv.x, fmaf(h.y, gv.y, t.x));
                t.y = fmaf(h.x, gv.y, fmaf(-h.y, gv.x, t.y));
            }
        }
        sum.x += t.x;
        sum.y += t.y;
        __syncthreads();
    }
    // the NG threads of each pair, added in thread order
    red[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x < NP) {
        double2 tot = make_double2(0.0, 0.0);
#pragma unroll 1
        for (int k = 0; k < NG; k++) {
            const double2 v = red[k * NP + threadIdx.x];
            tot.x += v.x;
            tot.y += v.y;
        }
        partial[((size_t)blockIdx.x * 9 + d) * NP + o * CIN + ci] = tot;
    }
}

// grad[k] += sum over blocks of partial[b][k] (k over 9*COUT*CIN), fixed order
__global__ void wgrad_finish_kernel(const double2 *partial, int nblocks, int n, double2 *grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    double2 t = make_double2(0.0, 0.0);
    for (int b = 0; b < nblocks; b++) {
        const double2 v = partial[(size_t)b * n + k];
        t.x += v.x;
        t.y += v.y;
    }
    grad[k].x += t.x;
    grad[k].y += t.y;
}

// even checkerboard FP32 pair vector [3][Vh] (stride Vh) -> full lattice
// [3][V] with zeros on odd sites, and back
__global__ void pair_to_full_kernel(NetGeom g, const float2 *__restrict__ ev, float2 *__restrict__ full) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V)
        return;
    int x[4];
    net_coords(g, i, x);
    const bool even = ((x[0] + x[1] + x[2] + x[3]) & 1) == 0;
    const int Vh = g.V / 2;
#pragma unroll
    for (int a = 0; a < 3; a++)
        full[(size_t)a * g.V + i] = even ? ev[(size_t)a * Vh + (i >> 1)] : make_float2(0.f, 0.f);
}

// loss of one pair: y (full, [3][V]) against e (even, [3][Vh]);
// gout = (y - e) / |e|^2 on even sites, 0 on odd; *loss += |y - e|^2 / |e|^2
__global__ void pair_loss_kernel(NetGeom g, const float2 *__restrict__ y, const float2 *__restrict__ e,
                                 const double *enorm2, float2 *__restrict__ gout, double *loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (i < g.V) {
        int x[4];
        net_coords(g, i, x);
        const bool even = ((x[0] + x[1] + x[2] + x[3]) & 1) == 0;
        const int Vh = g.V / 2;
        // a pair with e = 0 carries no information: no loss, no gradient
        const float inv = *enorm2 > 0.0 ? (float)(1.0 / *enorm2) : 0.f;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float2 d = make_float2(0.f, 0.f);
            if (even) {
                const float2 yv = y[(size_t)a * g.V + i];
                const float2 ev = e[(size_t)a * Vh + (i >> 1)];
                d = make_float2(yv.x - ev.x, yv.y - ev.y);
                part += (double)d.x * d.x + (double)d.y * d.y;
            }
            gout[(size_t)a * g.V + i] = make_float2(d.x * inv, d.y * inv);
        }
        part *= *enorm2 > 0.0 ? 1.0 / *enorm2 : 0.0;
    }
    for (int s = 16; s > 0; s >>= 1)
        part += __shfl_down_sync(0xffffffffu, part, s);
    if ((threadIdx.x & 31) == 0 && part != 0.0)
        atomicAdd(loss, part);
}

// residual loss of one pair: q = M z - r on even sites (mz, r full [3][V]),
// *loss += |q|^2 / |r|^2, q written over mz (odd sites zero)
__global__ void resid_loss_kernel(NetGeom g, float2 *mz, const float2 *__restrict__ r, const double *rnorm2,
                                  double *loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (i < g.V) {
        int x[4];
        net_coords(g, i, x);
        const bool even = ((x[0] + x[1] + x[2] + x[3]) & 1) == 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float2 q = make_float2(0.f, 0.f);
            if (even) {
                const float2 m = mz[(size_t)a * g.V + i], rv = r[(size_t)a * g.V + i];
                q = make_float2(m.x - rv.x, m.y - rv.y);
                part += (double)q.x * q.x + (double)q.y * q.y;
            }
            mz[(size_t)a * g.V + i] = q;
        }
        part *= *rnorm2 > 0.0 ? 1.0 / *rnorm2 : 0.0;
    }
    for (int s = 16; s > 0; s >>= 1)
        part += __shfl_down_sync(0xffffffffu, part, s);
    if ((threadIdx.x & 31) == 0 && part != 0.0)
        atomicAdd(loss, part);
}

// out[0] += Re<a, b>, out[1] += |a|^2 over full [3][V] vectors
__global__ void dot2_full_kernel(int n, const float2 *__restrict__ a, const float2 *__restrict__ b, double *out) {
    double p0 = 0.0, p1 = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float2 x = a[k], y = b[k];
        p0 += (double)x.x * y.x + (double)x.y * y.y;
        p1 += (double)x.x * x.x + (double)x.y * x.y;
    }
    for (int s = 16; s > 0; s >>= 1) {
        p0 += __shfl_down_sync(0xffffffffu, p0, s);
        p1 += __shfl_down_sync(0xffffffffu, p1, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, p0);
        atomicAdd(out + 1, p1);
    }
}

cudaError_t launch_dot2_full(int n, const float2 *a, const float2 *b, double *out, cudaStream_t s) {
    dot2_full_kernel<<<256, 256, 0, s>>>(n, a, b, out);
    return cudaGetLastError();
}

// v *= 1 / *n2 (full [3][V])
__global__ void scale_full_kernel(NetGeom g, float2 *v, const double *n2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * g.V)
        return;
    const float f = *n2 > 0.0 ? (float)(1.0 / *n2) : 0.f;
    v[k] = make_float2(v[k].x * f, v[k].y * f);
}

cudaError_t launch_resid_loss(const NetGeom &g, float2 *mz, const float2 *r, const double *rnorm2, double *loss,
                              cudaStream_t s) {
    resid_loss_kernel<<<(g.V + 255) / 256, 256, 0, s>>>(g, mz, r, rnorm2, loss);
    return cudaGetLastError();
}

cudaError_t launch_scale_full(const NetGeom &g, float2 *v, const double *n2, cudaStream_t s) {
    scale_full_kernel<<<(3 * g.V + 255) / 256, 256, 0, s>>>(g, v, n2);
    return cudaGetLastError();
}

// |v|^2 of an even FP32 pair vector into *out (atomic; monitoring only)
__global__ void pair_norm2_kernel(int n, const float2 *__restrict__ v, double *out) {
    double part = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float2 t = v[k];
        part += (double)t.x * t.x + (double)t.y * t.y;
    }
    for (int s = 16; s > 0; s >>= 1)
        part += __shfl_down_sync(0xffffffffu, part, s);
    if ((threadIdx.x & 31) == 0)
        atomicAdd(out, part);
}

// Adam on the real parameters (re, im of every weight); grad holds
// dL/dW*, so dL/d(re, im) = 2 (re, im) of it
__global__ void adam_kernel(int n, double *w, const double *grad, double *m, double *v, double lr, double b1,
                            double b2, double eps, int t, float *w32) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    const double gk = 2.0 * grad[k];
    m[k] = b1 * m[k] + (1 - b1) * gk;
    v[k] = b2 * v[k] + (1 - b2) * gk * gk;
    const double mh = m[k] / (1 - pow(b1, (double)t));
    const double vh = v[k] / (1 - pow(b2, (double)t));
    w[k] -= lr * mh / (sqrt(vh) + eps);
    w32[k] = (float)w[k];
}

// ---- vectors between the solver's layout and the net's ----------------
// even solver field (any precision, stride layout) -> full float2 [3][V]
template <int P>
__global__ void solver_to_full_kernel(NetGeom g, Geom sg, const typename Fmt<P>::Elem *f, float2 *full,
                                      const int *gate) {
    if (gate && *gate != CG_RUNNING)
        return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V)
        return;
    int x[4];
    net_coords(g, i, x);
    const bool even = ((x[0] + x[1] + x[2] + x[3]) & 1) == 0;
    cplx<typename Fmt<P>::R> w[3];
    if (even)
        load_vec<P>(f, sg.stride, i >> 1, w);
#pragma unroll
    for (int a = 0; a < 3; a++)
        full[(size_t)a * g.V + i] =
            even ? make_float2(rconv<float>(w[a].re), rconv<float>(w[a].im)) : make_float2(0.f, 0.f);
}

// full float2 [3][V] -> even solver field
template <int P>
__global__ void full_to_solver_kernel(NetGeom g, Geom sg, const float2 *full, typename Fmt<P>::Elem *f,
                                      const int *gate) {
    using R = typename Fmt<P>::R;
    if (gate && *gate != CG_RUNNING)
        return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= sg.Vh)
        return;
    // the even site with checkerboard index c
    int x[4];
    cb_coords(sg, c, 0, x);
    const int i = x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]));
    cplx<R> w[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float2 v = full[(size_t)a * g.V + i];
        w[a] = cplx<R>{rconv<R, float>(v.x), rconv<R, float>(v.y)};
    }
    store_vec<P>(f, sg.stride, c, w);
}

// even solver field (any precision) -> even FP32 pair vector [3][Vh]
template <int P>
__global__ void solver_to_pair_kernel(Geom sg, const typename Fmt<P>::Elem *f, const typename Fmt<P>::Elem *sub,
                                      float2 *pair) {
    using R = typename Fmt<P>::R;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= sg.Vh)
        return;
    cplx<R> w[3], s[3];
    load_vec<P>(f, sg.stride, c, w);
    if (sub)
        load_vec<P>(sub, sg.stride, c, s);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        R re = w[a].re, im = w[a].im;
        if (sub) {
            re = rsub(re, s[a].re);
            im = rsub(im, s[a].im);
        }
        pair[(size_t)a * sg.Vh + c] = make_float2(rconv<float>(re), rconv<float>(im));
    }
}

// ---- flexible CG vector kernels ----------------------------------------
// x += alpha p; r_old = r; r -= alpha Ap; |r|^2 -> stopping test
template <int P, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
fcg_update_kernel(Geom g, typename Fmt<P>::Elem *x, typename Fmt<P>::Elem *r, typename Fmt<P>::Elem *r_old,
                  const typename Fmt<P>::Elem *p, const typename Fmt<P>::Elem *Ap, double *partial,
                  CgScalars *sc) {
    using R = typename Fmt<P>::R;
    __shared__ double smem[32];
    const bool run = sc->status == CG_RUNNING;
    const int c = blockIdx.x * BLOCK + threadIdx.x;
    red_t<R> dot = red_zero<red_t<R>>();
    if (run && c < g.Vh) {
        const R alpha = scalar_as<R>(sc->alpha);
        const R malpha = -alpha;
        cplx<R> xv[3], rv[3], pv[3], av[3];
        load_vec<P>(x, g.stride, c, xv);
        load_vec<P>(r, g.stride, c, rv);
        load_vec<P>(p, g.stride, c, pv);
        load_vec<P>(Ap, g.stride, c, av);
        store_vec<P>(r_old, g.stride, c, rv);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            mac(xv[k].re, alpha, pv[k].re);
            mac(xv[k].im, alpha, pv[k].im);
            mac(rv[k].re, malpha, av[k].re);
            mac(rv[k].im, malpha, av[k].im);
            xv[k].re = rnorm<R>(xv[k].re);
            xv[k].im = rnorm<R>(xv[k].im);
            rv[k].re = rnorm<R>(rv[k].re);
            rv[k].im = rnorm<R>(rv[k].im);
        }
        store_vec<P>(x, g.stride, c, xv);
        store_vec<P>(r, g.stride, c, rv);
        dot = re_dot3<R>(rv, rv);
    }
    double total;
    if (grid_sum<BLOCK>(dot, partial, &sc->ticket, smem, total) && threadIdx.x == 0) {
        if (sc->status == CG_RUNNING) {
            sc->fcg_rr = total;
            sc->iter += 1;
            if (!(total < INFINITY))
                sc->status = CG_BREAKDOWN;
            else if (total <= sc->rr_stop)
                sc->status = CG_CONVERGED;
            else if (sc->iter >= sc->max_iter)
                sc->status = CG_MAXITER;
        }
    }
}

// <z, r> and <z, r_old> (real parts) -> beta (Polak-Ribiere), rr = <z, r>
template <int P, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
fcg_beta_kernel(Geom g, const typename Fmt<P>::Elem *z, const typename Fmt<P>::Elem *r,
                const typename Fmt<P>::Elem *r_old, double *partial, CgScalars *sc, int first) {
    using R = typename Fmt<P>::R;
    __shared__ double smem[32];
    if (sc->status != CG_RUNNING)
        return;
    const int c = blockIdx.x * BLOCK + threadIdx.x;
    red_t<R> d0 = red_zero<red_t<R>>(), d1 = red_zero<red_t<R>>();
    if (c < g.Vh) {
        cplx<R> zv[3], rv[3], ov[3];
        load_vec<P>(z, g.stride, c, zv);
        load_vec<P>(r, g.stride, c, rv);
        d0 = re_dot3<R>(zv, rv);
        if (!first) {
            load_vec<P>(r_old, g.stride, c, ov);
            d1 = re_dot3<R>(zv, ov);
        }
    }
    double zr, zro;
    if (grid_sum2<BLOCK>(d0, d1, partial, &sc->ticket, smem, zr, zro) && threadIdx.x == 0) {
        const double beta = first ? 0.0 : (zr - zro) / sc->rr;
        sc->beta = make_dpair(beta);
        sc->rr = zr;
        if (!(zr > 0.0 && zr < INFINITY))
            sc->status = CG_BREAKDOWN;  // the preconditioned residual lost positivity
    }
}

// ---- launchers -----------------------------------------------------------
template <int CIN, int COUT>
static cudaError_t conv_t(const NetGeom &g, const float2 *NL, const float2 *W, int round_half, const float2 *in,
                          float2 *out, const int *gate, int in_par, int out_par, cudaStream_t s) {
    const int n = out_par < 0 ? g.V : g.V / 2;
    covconv_kernel<CIN, COUT><<<(n + 127) / 128, 128, 0, s>>>(g, NL, W, round_half, in, out, gate, in_par, out_par);
    return cudaGetLastError();
}

cudaError_t launch_covconv(int cin, int cout, const NetGeom &g, const float2 *NL, const float2 *W, int round_half,
                           const float2 *in, float2 *out, const int *gate, cudaStream_t s, int in_par,
                           int out_par) {
#define CC(A, B) \
    if (cin == A && cout == B) return conv_t<A, B>(g, NL, W, round_half, in, out, gate, in_par, out_par, s);
    CC(1, 4) CC(4, 4) CC(4, 1) CC(1, 8) CC(8, 8) CC(8, 1) CC(1, 2) CC(2, 2) CC(2, 1) CC(1, 1)
#undef CC
    return cudaErrorInvalidValue;
}

constexpr int WG_BLOCKS = 512;

int wgrad_partial_blocks() { return WG_BLOCKS; }

template <int CIN, int COUT>
static cudaError_t wgrad_t(const NetGeom &g, const float2 *NL, const float2 *in, const float2 *gout,
                           double2 *partial, double2 *grad, cudaStream_t s) {
    if constexpr (CIN > 1 && COUT > 1) {
        // square layers: the shared-memory tile (measured at 8 x 8 channels,
        // 32^3x64: 3.3 ms against 5.5 ms for the per-thread sums)
        covconv_wgrad_kernel<CIN, COUT><<<dim3(WG_BLOCKS, 9), WG_THREADS, 0, s>>>(g, NL, in, gout, partial);
    } else {
        // narrow layers: per-thread sums (measured at 1 x 8 and 8 x 1
        // channels: 0.9-1.0 ms against 1.25-1.3 ms for the tile)
        constexpr int OB = COUT < 4 ? COUT : 4;
        constexpr int NOB = (COUT + OB - 1) / OB;
        covconv_wgrad_reg_kernel<CIN, COUT, OB><<<dim3(WG_BLOCKS, 9 * NOB), 128, 0, s>>>(g, NL, in, gout, partial);
    }
    const int n = 9 * COUT * CIN;
    wgrad_finish_kernel<<<(n + 127) / 128, 128, 0, s>>>(partial, WG_BLOCKS, n, grad);
    return cudaGetLastError();
}

cudaError_t launch_covconv_wgrad(int cin, int cout, const NetGeom &g, const float2 *NL, const float2 *in,
                                 const float2 *gout, double2 *partial, double2 *grad, cudaStream_t s) {
#define CW(A, B) \
    if (cin == A && cout == B) return wgrad_t<A, B>(g, NL, in, gout, partial, grad, s);
    CW(1, 4) CW(4, 4) CW(4, 1) CW(1, 8) CW(8, 8) CW(8, 1) CW(1, 2) CW(2, 2) CW(2, 1) CW(1, 1)
#undef CW
    return cudaErrorInvalidValue;
}

cudaError_t launch_pair_to_full(const NetGeom &g, const float2 *ev, float2 *full, cudaStream_t s) {
    pair_to_full_kernel<<<(g.V + 255) / 256, 256, 0, s>>>(g, ev, full);
    return cudaGetLastError();
}

cudaError_t launch_pair_loss(const NetGeom &g, const float2 *y, const float2 *e, const double *enorm2,
                             float2 *gout, double *loss, cudaStream_t s) {
    pair_loss_kernel<<<(g.V + 255) / 256, 256, 0, s>>>(g, y, e, enorm2, gout, loss);
    return cudaGetLastError();
}

cudaError_t launch_pair_norm2(int n, const float2 *v, double *out, cudaStream_t s) {
    pair_norm2_kernel<<<256, 256, 0, s>>>(n, v, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(int n, double *w, const double *grad, double *m, double *v, double lr, int t, float *w32,
                        cudaStream_t s) {
    adam_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, w, grad, m, v, lr, 0.9, 0.999, 1e-8, t, w32);
    return cudaGetLastError();
}

#define NP_SWITCH(prec, ...)                                                \
    switch (prec) {                                                         \
    case P_F64: { constexpr int P = P_F64; __VA_ARGS__; } break;            \
    case P_DF64: { constexpr int P = P_DF64; __VA_ARGS__; } break;          \
    case P_F32: { constexpr int P = P_F32; __VA_ARGS__; } break;            \
    default: return cudaErrorInvalidValue;                                  \
    }

cudaError_t launch_solver_to_full(int prec, const NetGeom &g, const Geom &sg, const void *f, float2 *full,
                                  const int *gate, cudaStream_t s) {
    NP_SWITCH(prec, solver_to_full_kernel<P><<<(g.V + 255) / 256, 256, 0, s>>>(
                        g, sg, (const typename Fmt<P>::Elem *)f, full, gate));
    return cudaGetLastError();
}

cudaError_t launch_full_to_solver(int prec, const NetGeom &g, const Geom &sg, const float2 *full, void *f,
                                  const int *gate, cudaStream_t s) {
    NP_SWITCH(prec, full_to_solver_kernel<P><<<(sg.Vh + 255) / 256, 256, 0, s>>>(
                        g, sg, full, (typename Fmt<P>::Elem *)f, gate));
    return cudaGetLastError();
}

cudaError_t launch_solver_to_pair(int prec, const Geom &sg, const void *f, const void *sub, float2 *pair,
                                  cudaStream_t s) {
    NP_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        solver_to_pair_kernel<P><<<(sg.Vh + 255) / 256, 256, 0, s>>>(sg, (const E *)f, (const E *)sub, pair);
    });
    return cudaGetLastError();
}

constexpr int FB = 256;

cudaError_t launch_fcg_update(int prec, const Geom &g, void *x, void *r, void *r_old, const void *p,
                              const void *Ap, double *partial, CgScalars *sc, cudaStream_t s) {
    NP_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        fcg_update_kernel<P, FB><<<(g.Vh + FB - 1) / FB, FB, 0, s>>>(g, (E *)x, (E *)r, (E *)r_old,
                                                                     (const E *)p, (const E *)Ap, partial, sc);
    });
    return cudaGetLastError();
}

cudaError_t launch_fcg_beta(int prec, const Geom &g, const void *z, const void *r, const void *r_old,
                            double *partial, CgScalars *sc, int first, cudaStream_t s) {
    NP_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        fcg_beta_kernel<P, FB><<<(g.Vh + FB - 1) / FB, FB, 0, s>>>(g, (const E *)z, (const E *)r,
                                                                   (const E *)r_old, partial, sc, first);
    });
    return cudaGetLastError();
}

}  // namespace stag

namespace stag {

// raw fat links (canonical complex128 [4][V][3][3]) -> net links
// float2 [4][9][V], the boundary sign of the forward hop folded into the
// last-slice link (so the backward hop, which uses the link of x - mu,
// carries the same sign)
__global__ void net_links_kernel(NetGeom g, double bc0, double bc1, double bc2, double bc3,
                                 const double2 *__restrict__ fat, float2 *NL) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 4LL * g.V)
        return;
    const int mu = (int)(t / g.V);
    const int i = (int)(t % g.V);
    int x[4];
    net_coords(g, i, x);
    const double bc[4] = {bc0, bc1, bc2, bc3};
    const double sgn = (x[mu] == g.L[mu] - 1 && bc[mu] < 0) ? -1.0 : 1.0;
    for (int e = 0; e < 9; e++) {
        const double2 u = fat[((size_t)mu * g.V + i) * 9 + e];
        NL[((size_t)mu * 9 + e) * g.V + i] = make_float2((float)(sgn * u.x), (float)(sgn * u.y));
    }
}

cudaError_t launch_net_links(const NetGeom &g, const double bc[4], const double *fat, float2 *NL, cudaStream_t s) {
    const long long n = 4LL * g.V;
    net_links_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, bc[0], bc[1], bc[2], bc[3],
                                                                 (const double2 *)fat, NL);
    return cudaGetLastError();
}

// WT[dbar][i][o] = conj(W[d][o][i]), dbar the reversed hop: the weights of
// the adjoint layer (input gradient of the backward pass)
__global__ void net_adjoint_kernel(int cin, int cout, const float2 *W, float2 *WT) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 9 * cin * cout)
        return;
    const int d = k / (cout * cin);
    const int o = (k / cin) % cout;
    const int i = k % cin;
    const int db = d == 0 ? 0 : (((d - 1) & 1) ? d - 1 : d + 1);
    const float2 w = W[k];
    WT[(db * cin + i) * cout + o] = make_float2(w.x, -w.y);
}

cudaError_t launch_net_adjoint(int cin, int cout, const float2 *W, float2 *WT, cudaStream_t s) {
    const int n = 9 * cin * cout;
    net_adjoint_kernel<<<(n + 127) / 128, 128, 0, s>>>(cin, cout, W, WT);
    return cudaGetLastError();
}

}  // namespace stag
