// Host-side launchers of the libstag kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include "cg_state.cuh"
#include "common.cuh"

namespace stag {

struct DslashArgs;

// Dslash with epilogue `epi` (Epi enum) in precision `prec`; block = 0 picks
// the default block size.
cudaError_t launch_dslash(int prec, int epi, const DslashArgs &a, int block, cudaStream_t s);
int dslash_default_block(int prec);
int dslash_grid(const Geom &g, int block);

// CG vector kernels (grid = ceil(Vh / CG_BLOCK))
constexpr int CG_BLOCK = 256;
cudaError_t launch_cg_init(int prec, const Geom &g, void *x, void *r, void *p, const void *b,
                           double *partial, CgScalars *sc, cudaStream_t s);
cudaError_t launch_cg_update(int prec, const Geom &g, void *x, void *r, const void *p,
                             const void *Ap, double *partial, CgScalars *sc, cudaStream_t s);
cudaError_t launch_cg_p_update(int prec, const Geom &g, const void *r, void *p,
                               const CgScalars *sc, cudaStream_t s);
// <p, M p> from the n block partials of a Dslash with EPI_M_PART, summed in
// block order; then alpha = |r|^2 / <p, M p> and the breakdown test (as the
// EPI_M_PAP epilogue).  Returns at once when skip_if_done and the solve has
// stopped.
// gate (may be NULL): return at once while *gate == 0
cudaError_t launch_pap_finish(const double *partial, int n, CgScalars *sc, bool skip_if_done, cudaStream_t s,
                              const int *gate = nullptr);

// canonical complex128 [Vh][3] (device) <-> internal field layout
cudaError_t launch_import(int prec, const Geom &g, const double *canon, void *field, cudaStream_t s);
cudaError_t launch_export(int prec, const Geom &g, const void *field, double *canon, cudaStream_t s);

// fold c1/c3, Kogut-Susskind phases and boundary signs into the canonical
// fat/long links (device, complex128 [4][V][3][3]) and lay them out per parity
// (inv_scale: 16-bit links only, 32767 / largest |entry| of the folded
// one-link and three-link fields; ignored otherwise)
cudaError_t launch_fold_links(int prec, const Geom &g, const double bc[4], double c1, double c3,
                              const double *fat, const double *lng, void *links,
                              const float inv_scale[2], cudaStream_t s);

// fold into the 12-real layout (FP32 or 16-bit; see C12 in fields.cuh)
cudaError_t launch_fold_links_c12(int prec, const Geom &g, const double bc[4], double c1, double c3,
                                  const double *fat, const double *lng, void *links, const float inv_scale[2],
                                  int mask, cudaStream_t s);
// largest deviation from SU(3) over nlinks canonical 3x3 complex128
// matrices, as float bits in *out (device)
cudaError_t launch_su3_deviation(const double *U, long long nlinks, unsigned *out, cudaStream_t s);

// largest |re| / |im| over n doubles, as float bits in *out (device); a
// NaN, an infinity or a value beyond the FP32 range gives +infinity
cudaError_t launch_absmax(const double *a, long long n, unsigned *out, cudaStream_t s);

// *flag = 1 if a finite entry of n doubles lies beyond the FP32 range (device)
cudaError_t launch_finite_overflow(const double *a, long long n, unsigned *flag, cudaStream_t s);

// largest |component| of a field (F64, DF64: hi parts, F32) as float bits in
// *out (device); v *= 2^e exactly (results in the normal range)
cudaError_t launch_field_absmax(int prec, const Geom &g, const void *v, unsigned *out, cudaStream_t s);
cudaError_t launch_field_ldexp(int prec, const Geom &g, void *v, int e, cudaStream_t s);

// three-link products N_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu), canonical layout
cudaError_t launch_long_links(const Geom &g, const double *fat, double *lng, cudaStream_t s);

// mixed-precision CG with reliable updates: hi = F64 or DF64 (x, r, b),
// lo = F32 or F16 (p, Ap, r_sloppy), x_sloppy always F32
cudaError_t launch_mixed_init(int hi, int lo, const Geom &g, void *x, void *r, const void *b, float *xs,
                              void *rs, void *p, double *partial, CgScalars *sc, cudaStream_t s);
cudaError_t launch_mixed_update(int lo, const Geom &g, float *xs, void *rs, const void *p, const void *Ap,
                                double *partial, CgScalars *sc, cudaStream_t s);
cudaError_t launch_mixed_accum(int hi, const Geom &g, void *x, float *xs, const CgScalars *sc,
                               cudaStream_t s);
cudaError_t launch_mixed_restart(int hi, int lo, const Geom &g, const void *r, void *rs, CgScalars *sc,
                                 cudaStream_t s);

// multi-shift CG (kernels_multishift.cu) and vector helpers
// lo >= 0: mixed precision (vectors in prec, the Dslash pair in lo = FP32)
cudaError_t launch_ms_init(int prec, const Geom &g, const MsArgs &a, double *partial, CgScalars *sc,
                           ShiftState *st, cudaStream_t s, int lo = -1);
cudaError_t launch_ms_update(int prec, const Geom &g, const MsArgs &a, const void *Ap, double *partial,
                             CgScalars *sc, ShiftState *st, cudaStream_t s, int lo = -1);
cudaError_t launch_ms_p(int prec, const Geom &g, const MsArgs &a, const CgScalars *sc,
                        const ShiftState *st, cudaStream_t s, int lo = -1);
// after a reliable update of the base residual (gated on sc->reliable)
cudaError_t launch_ms_restart(const MsArgs &a, CgScalars *sc, ShiftState *st, cudaStream_t s);
cudaError_t launch_axpy1(int prec, const Geom &g, const void *x, void *y, cudaStream_t s);
cudaError_t launch_convert(int prec_out, int prec_in, const Geom &g, const void *in, void *out,
                           cudaStream_t s);

// batched CG (batched.cuh, kernels_batched.cu): `what` is a BatchKernel
struct BatchArgs;
cudaError_t launch_batch(int prec, int what, const BatchArgs &a, int block, cudaStream_t s);
int batch_max_k(int prec);
int batch_min_k(int prec);

// record the calling thread's last error message (read back by
// stag_last_error_message) and return `code`
int set_error(int code, const char *fmt, ...);

}  // namespace stag
