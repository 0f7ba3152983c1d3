// Shared declarations of the learned preconditioner (kernels_learned.cu,
// kernels_netpath.cu, learned.cu): path coefficients, link sets and kernel
// launchers.
#pragma once
#include "dslash.cuh"

namespace stag {

// The net's action on even fields as a two-hop path sum (kernels_netpath.cu):
// z = c0 r + sum_{a,b} C[a*8+b] T_a T_b r, hop index 2 mu (+mu) or 2 mu + 1 (-mu)
struct NetPath {
    float2 C[64];
    float2 c0;
};

// the net's link copies: FP32, and optionally 16-bit (used when l16 or l12
// is set; l12 first)
struct NetLinkSet {
    const float2 *l32 = nullptr;
    const short2 *l16 = nullptr;
    const void *l12 = nullptr;  // 16-bit, rows 0 and 1 only (special unitary links)
    float scale16 = 0.f;        // 16-bit value = q * scale16
    int bcneg = 0;              // bit mu: the boundary sign of direction mu is -1
};

cudaError_t launch_net_links_cb(const Geom &g, const double bc[4], const double *fat, float2 *NL32, short2 *NL16,
                                float inv_scale16, cudaStream_t s);
// rows 0 and 1 of the net links in 16-bit: per (parity, mu) an int4 plane
// (entries 0..3) and an int2 plane (entries 4, 5), 24 stride bytes
cudaError_t launch_net_links12(const Geom &g, const double bc[4], const double *fat, void *NL12, float inv_scale16,
                               cudaStream_t s);
size_t net_links12_bytes(const Geom &g);
// hermitian: the coefficients of the net's Hermitian part (N + N^+)/2
cudaError_t launch_net_path_coef(int C, const float *w32, const int off[3], int round_half, NetPath *out,
                                 cudaStream_t s, int hermitian = 0);
cudaError_t launch_net_path_chain(int C, const float *w32, const int off[3], const double2 *G, double2 *grad,
                                  cudaStream_t s);
// chi (odd sites; FP32 [8][3][stride] with FP32 links, 16-bit [8][3][stride]
// plus float norms [8][stride] with 16-bit links) from the even input r
// (precision prec, stride rs)
cudaError_t launch_net_mid(int prec, const Geom &g, const NetLinkSet &nl, const NetPath *path, const void *r,
                           int rs, void *chi, const int *gate, cudaStream_t s);
// z = c0 r + sum_a T_a chi_a (even); dots adds the per-block partials of
// Re<z, r> and Re<z, Ap> (0 without Ap): 2 * net_grid doubles
cudaError_t launch_net_out(int prec_in, int prec_out, const Geom &g, const NetLinkSet &nl, const NetPath *path,
                           const void *chi, const void *r, int rs, void *z, int zs, bool dots, const void *Ap,
                           double *partial, const int *gate, cudaStream_t s);
int net_grid(const Geom &g);
int net_grad_blocks(const Geom &g);
// G[0..63] += dL/dC*, G[64] += dL/dc0* for input r and output gradient g (FP32)
cudaError_t launch_net_grad(const Geom &g, const float2 *NL32, const float2 *r, int rs, const float2 *gv, int gs,
                            double2 *partial, double2 *G, cudaStream_t s);
cudaError_t launch_net_error_loss(int Vh, const float2 *z, int zs, const float2 *e, int es, const double *enorm2,
                                  float2 *gv, double *loss, cudaStream_t s);
cudaError_t launch_net_resid_loss(int Vh, float2 *mz, int ms, const float2 *r, int rs, const double *rnorm2,
                                  double *loss, cudaStream_t s);
cudaError_t launch_net_dot2(int Vh, const float2 *a, int as, const float2 *b, int bs, double *out, cudaStream_t s);
cudaError_t launch_fcg_finish(const double *partial, int n, CgScalars *sc, int first, cudaStream_t s);
cudaError_t launch_fcg_copy_dots(int prec, const Geom &g, const void *r, void *z, const void *Ap, double *partial,
                                 const int *gate, cudaStream_t s);

// kernels_learned.cu
cudaError_t launch_pair_norm2(int n, const float2 *v, double *out, cudaStream_t s);
cudaError_t launch_adam(int n, double *w, const double *grad, double *m, double *v, double lr, int t, float *w32,
                        cudaStream_t s);
cudaError_t launch_solver_to_pair(int prec, const Geom &sg, const void *f, const void *sub, float2 *pair,
                                  cudaStream_t s);
cudaError_t launch_fcg_update(int prec, const Geom &g, void *x, void *r, const void *p, const void *Ap,
                              double *partial, CgScalars *sc, cudaStream_t s);

}  // namespace stag
