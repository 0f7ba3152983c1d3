// Shared declarations of the learned preconditioner (kernels_learned.cu,
// learned.cu): full-lattice geometry and kernel launchers.
#pragma once
#include "dslash.cuh"

namespace stag {

struct NetGeom {
    int L[4];
    int V;        // sites of the full lattice
    int step[4];  // lexicographic index step of one hop: 1, Lx, Lx*Ly, Lx*Ly*Lz
};

// in_par / out_par: parity where the input is non-zero / of the outputs
// needed (-1: all sites)
cudaError_t launch_covconv(int cin, int cout, const NetGeom &g, const float2 *NL, const float2 *W, int round_half,
                           const float2 *in, float2 *out, const int *gate, cudaStream_t s, int in_par = -1,
                           int out_par = -1);
cudaError_t launch_covconv_wgrad(int cin, int cout, const NetGeom &g, const float2 *NL, const float2 *in,
                                 const float2 *gout, double2 *partial, double2 *grad, cudaStream_t s);
int wgrad_partial_blocks();
cudaError_t launch_pair_to_full(const NetGeom &g, const float2 *ev, float2 *full, cudaStream_t s);
cudaError_t launch_pair_loss(const NetGeom &g, const float2 *y, const float2 *e, const double *enorm2,
                             float2 *gout, double *loss, cudaStream_t s);
cudaError_t launch_pair_norm2(int n, const float2 *v, double *out, cudaStream_t s);
cudaError_t launch_adam(int n, double *w, const double *grad, double *m, double *v, double lr, int t, float *w32,
                        cudaStream_t s);
cudaError_t launch_solver_to_full(int prec, const NetGeom &g, const Geom &sg, const void *f, float2 *full,
                                  const int *gate, cudaStream_t s);
cudaError_t launch_full_to_solver(int prec, const NetGeom &g, const Geom &sg, const float2 *full, void *f,
                                  const int *gate, cudaStream_t s);
cudaError_t launch_solver_to_pair(int prec, const Geom &sg, const void *f, const void *sub, float2 *pair,
                                  cudaStream_t s);
cudaError_t launch_fcg_update(int prec, const Geom &g, void *x, void *r, void *r_old, const void *p,
                              const void *Ap, double *partial, CgScalars *sc, cudaStream_t s);
cudaError_t launch_fcg_beta(int prec, const Geom &g, const void *z, const void *r, const void *r_old,
                            double *partial, CgScalars *sc, int first, cudaStream_t s);
cudaError_t launch_resid_loss(const NetGeom &g, float2 *mz, const float2 *r, const double *rnorm2, double *loss,
                              cudaStream_t s);
cudaError_t launch_dot2_full(int n, const float2 *a, const float2 *b, double *out, cudaStream_t s);
cudaError_t launch_scale_full(const NetGeom &g, float2 *v, const double *n2, cudaStream_t s);
cudaError_t launch_net_links(const NetGeom &g, const double bc[4], const double *fat, float2 *NL, cudaStream_t s);
cudaError_t launch_net_adjoint(int cin, int cout, const float2 *W, float2 *WT, cudaStream_t s);

}  // namespace stag
