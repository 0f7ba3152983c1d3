// Learned preconditioner: the training-pair and optimiser kernels and the
// vector update of the flexible CG that applies it.  The paper has no learned
// preconditioner; the net and its path-form kernels are described in
// kernels_netpath.cu.
#include "learned.cuh"
#include "kernels.h"

namespace stag {

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

// ---- vectors between the solver's layout and the training pairs -------
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

// ---- flexible CG vector kernel ------------------------------------------
// x += alpha p; r -= alpha Ap; |r|^2 -> stopping test
template <int P, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
fcg_update_kernel(Geom g, typename Fmt<P>::Elem *x, typename Fmt<P>::Elem *r,
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

#define NP_SWITCH(prec, ...)                                                \
    switch (prec) {                                                         \
    case P_F64: { constexpr int P = P_F64; __VA_ARGS__; } break;            \
    case P_DF64: { constexpr int P = P_DF64; __VA_ARGS__; } break;          \
    case P_F32: { constexpr int P = P_F32; __VA_ARGS__; } break;            \
    default: return cudaErrorInvalidValue;                                  \
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

cudaError_t launch_solver_to_pair(int prec, const Geom &sg, const void *f, const void *sub, float2 *pair,
                                  cudaStream_t s) {
    NP_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        solver_to_pair_kernel<P><<<(sg.Vh + 255) / 256, 256, 0, s>>>(sg, (const E *)f, (const E *)sub, pair);
    });
    return cudaGetLastError();
}

constexpr int FB = 256;

cudaError_t launch_fcg_update(int prec, const Geom &g, void *x, void *r, const void *p, const void *Ap,
                              double *partial, CgScalars *sc, cudaStream_t s) {
    NP_SWITCH(prec, {
        using E = typename Fmt<P>::Elem;
        fcg_update_kernel<P, FB><<<(g.Vh + FB - 1) / FB, FB, 0, s>>>(g, (E *)x, (E *)r, (const E *)p,
                                                                     (const E *)Ap, partial, sc);
    });
    return cudaGetLastError();
}

}  // namespace stag
