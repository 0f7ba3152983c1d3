/*
 * stag.h — C ABI of the GB300 improved-staggered (Naik) Dslash and even-odd
 * conjugate-gradient library.
 *
 * The operation is the one Li & Gottlieb benchmark ("Staggered Dslash
 * Performance on Intel Xeon Phi Architecture", Lattice 2014, Sec. 3): for every
 * site of one checkerboard, 16 SU(3) matrix x colour-vector products over the
 * 8 forward/backward directions, with the one-link (fat) and three-link (Naik,
 * long) matrices, summed into one colour vector; and the CG solver that calls
 * it twice per iteration.  Written out:
 *
 *   (D psi)(x) = sum_mu eta_mu(x) { c1 [ b U_mu(x) psi(x+mu)  - b U_mu(x-mu)^+ psi(x-mu)  ]
 *                                 + c3 [ b N_mu(x) psi(x+3mu) - b N_mu(x-3mu)^+ psi(x-3mu) ] }
 *
 *   eta_mu(x) = (-1)^(x_0+...+x_{mu-1})   Kogut-Susskind phases (Sec. 4: "absorbed
 *                                          into the gauge fields")
 *   b = bc_mu^w, w = number of times the hop wraps around direction mu
 *   M = m^2 - D_eo D_oe on the even checkerboard (no factor 1/2 in D; MILC's
 *       4m^2 - D D convention is this one with m_MILC = m/2).
 *
 * Conventions shared by every call:
 *   - dims[4] = {Lx, Ly, Lz, Lt}; every extent even and >= 2; V = product,
 *     Vh = V/2 sites per parity.  Site i = x + Lx*(y + Ly*(z + Lz*t));
 *     parity (x+y+z+t) & 1 (0 = even).
 *   - A gauge field in canonical layout is complex128 [4][V][3][3] (direction,
 *     site, row, column; (re, im) interleaved doubles).
 *   - A colour field on one parity in canonical layout is complex128 [Vh][3],
 *     site i of that parity at position i/2 ("checkerboard order").
 *   - Host pointers (STAG_PTR_HOST) are ordinary host memory (pinned memory
 *     makes copies faster); device pointers (STAG_PTR_DEVICE) must be device
 *     memory of the lattice's device.  Gauge uploads and long-link builds
 *     from device pointers synchronize the device first, so the source may
 *     have been written on any stream; field imports from device pointers
 *     read on the lattice stream, so the caller must have finished writing
 *     the source (or written it on that stream).  The caller keeps ownership of every
 *     buffer it passes; the library copies what it needs before returning
 *     (or, for asynchronous calls on device pointers, before the work it
 *     enqueued completes).
 *   - Every function returns STAG_OK (0) or a negative STAG_ERR_* code; no
 *     exception crosses the ABI.  stag_last_error_message() gives a
 *     human-readable reason for the last failure on the calling thread.
 *   - Work is enqueued on the lattice's CUDA stream.  Dslash calls are
 *     asynchronous; field import/export and the solvers return after their
 *     work is complete.  One lattice must not be used by two host threads at
 *     the same time.
 */
#ifndef STAG_H
#define STAG_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
    STAG_OK = 0,
    STAG_ERR_ARG = -1,           /* null pointer, bad dims, size or enum value          */
    STAG_ERR_STATE = -2,         /* no gauge field uploaded, parity/precision mismatch  */
    STAG_ERR_CUDA = -3,          /* a CUDA call failed (message has the CUDA error)     */
    STAG_ERR_NOT_CONVERGED = -4, /* solver hit max_iter; x holds the last iterate       */
    STAG_ERR_BREAKDOWN = -5,     /* <p, M p> not positive or not finite                 */
    STAG_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up                  */
    STAG_ERR_NOMEM = -7          /* device or host allocation failed                    */
};

/* ---- precisions ---------------------------------------------------------
 * STAG_F64   IEEE double storage and double arithmetic.
 * STAG_DF64  "double-float": each real stored as a pair of floats (hi, lo)
 *            with hi + lo the value (about 48 significant bits, float
 *            exponent range); arithmetic in error-free float operations.
 *            GB300's FP64 pipe is far narrower than its FP32 pipes, and this
 *            form keeps FP64-level accuracy at FP32 throughput.
 *            Range: imports into DF64, F32 and F16 fields refuse finite
 *            entries beyond the FP32 range (STAG_ERR_ARG, field unchanged);
 *            entries below about 1e-30 lose relative precision in DF64 (the
 *            low float of the pair leaves the normal range).  Every solver
 *            on DF64 or F32 fields first checks the exponent k of b's largest
 *            entry: when |k| > 16 it solves with a copy b 2^-k (allocated for
 *            the call) and multiplies the solutions by 2^k, both exact, so
 *            the scale of b does not matter within that range.
 * STAG_F32   float storage and arithmetic.
 * STAG_F16   16-bit storage ("half" in the lattice-QCD sense): signed
 *            fixed point, links with one scale per field (the largest folded
 *            entry), colour vectors with one float norm per site (a site's
 *            three components and its norm share one 16-byte cell); float
 *            arithmetic.  1/32767 of the scale per entry.
 */
enum { STAG_F64 = 0, STAG_F32 = 1, STAG_F16 = 2, STAG_DF64 = 3 };
#define STAG_PREC_BIT(p) (1u << (p))
#define STAG_COMPRESS12 (1u << 16)
#define STAG_COMPRESS12_LONG (1u << 17)

enum { STAG_EVEN = 0, STAG_ODD = 1 };
enum { STAG_PTR_HOST = 0, STAG_PTR_DEVICE = 1 };

typedef struct stag_lattice_s *stag_lattice;
typedef struct stag_field_s *stag_field;

/* ---- lattice ------------------------------------------------------------ */

/* Create a lattice on CUDA device `device`.
 * dims: {Lx, Ly, Lz, Lt}, each even and >= 2, V <= 2^31 - 2.
 * bc:   boundary sign per direction, each +1 (periodic) or -1 (antiperiodic);
 *       NULL means {+1, +1, +1, -1}.
 * cuda_stream: a cudaStream_t of that device to enqueue all work on, or NULL
 *       for a stream owned by the lattice.
 * Errors: STAG_ERR_ARG (argument checks run before any CUDA call),
 *         STAG_ERR_CUDA, STAG_ERR_NOMEM. */
int stag_lattice_create(stag_lattice *out, const int dims[4], const double bc[4],
                        int device, void *cuda_stream);

/* Free every device buffer the lattice owns.  Fields created on the lattice
 * must be destroyed first (STAG_ERR_STATE otherwise). NULL is accepted. */
int stag_lattice_destroy(stag_lattice lat);

/* Sizes: V, Vh.  Pure host queries. */
int stag_lattice_volume(const stag_lattice lat, long long *V, long long *Vh);

/* How stag_cg_solve drives its iterations.
 * STAG_CG_LAUNCH_GRAPH (default): one CUDA graph per solve whose loop is a
 *   conditional WHILE node; the last kernel of each iteration sets the loop
 *   condition on the device, so the host waits once per solve.
 * STAG_CG_LAUNCH_HOST: the same kernels launched individually; the host
 *   reads the solver status every `chunk` iterations (1..4096) and kernels
 *   of iterations past convergence return at once.  For drivers or tools
 *   that cannot run or inspect conditional graph nodes (e.g. per-kernel
 *   profiling).  Results are identical in both modes. */
enum { STAG_CG_LAUNCH_GRAPH = 0, STAG_CG_LAUNCH_HOST = 1 };
int stag_lattice_set_cg_launch(stag_lattice lat, int mode, int chunk);

/* ---- gauge field ---------------------------------------------------------
 * Upload the fat (one-link) field and the long (three-link, Naik) field,
 * both canonical complex128 [4][V][3][3], with Naik coefficients c1 (one-link)
 * and c3 (three-link), e.g. 9/8 and -1/24.  lng == NULL builds the long links
 * on the GPU as the three-link products N_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu)
 * of the raw fat links (Sec. 4 "three-link products").
 * The library folds c1, c3, the Kogut-Susskind phases and the boundary signs
 * into its own copies and re-lays them out per parity (structure of arrays).
 * prec_mask: OR of STAG_PREC_BIT(p) for each precision to build a copy for
 *            (0 means F64 | DF64), optionally with STAG_COMPRESS12: the F32
 *            and F16 Dslash then read "two-row" 12-real links (the paper's
 *            gauge compression, Sec. 4) and rebuild row 3 as
 *            conj(row1 x row2) / (c eta b): 2/3 of the link bytes and wider
 *            loads.  Only valid for special unitary links (checked: a link
 *            deviating from SU(3) by more than 1e-6 gives STAG_ERR_ARG, e.g.
 *            smeared fat links, which the paper notes are not in SU(3));
 *            the full copies are kept for the batched solver.  With
 *            STAG_COMPRESS12_LONG instead only the three-link field is
 *            compressed and checked (the paper's suggestion for smeared fat
 *            links, Sec. 4): 5/6 of the link bytes.
 *            A later upload replaces all copies.
 * Links holding a NaN, an infinity or an entry beyond the FP32 range give
 * STAG_ERR_ARG (the lattice then has no gauge field).
 * Blocks until the copies are built. */
int stag_gauge_upload(stag_lattice lat, const double *fat, const double *lng,
                      double c1, double c3, int ptr_kind, unsigned prec_mask);

/* Compute the three-link products N_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu)
 * (Sec. 4 "three-link products") of the raw fat links `fat` on the GPU and
 * write them to `lng`, both canonical complex128 [4][V][3][3] (periodic
 * indexing, no coefficient, phase or boundary sign).  FP64 arithmetic.
 * Blocks until `lng` is written.  Does not change the uploaded gauge field. */
int stag_long_links_build(stag_lattice lat, const double *fat, double *lng, int ptr_kind);

/* ---- colour fields (one parity, internal layout, owned by the library) -- */
int stag_field_create(stag_lattice lat, int parity, int prec, stag_field *out);
int stag_field_destroy(stag_field f);
/* Import/export canonical complex128 [Vh][3] (host or device memory per
 * ptr_kind; the caller owns src/dst); blocks until complete.  A device source
 * is read after all work already queued on the device has finished, so a
 * buffer just written on another stream may be passed directly. */
int stag_field_import(stag_field f, const double *src, int ptr_kind);
int stag_field_export(const stag_field f, double *dst, int ptr_kind);
/* Set a field to zero (asynchronous). */
int stag_field_zero(stag_field f);
/* Device address and size in bytes of the field's internal storage (for
 * zero-copy views; layout is internal). */
int stag_field_storage(const stag_field f, void **dev_ptr, unsigned long long *bytes);
/* Bytes of one field of precision `prec` on this lattice (the size that
 * stag_field_wrap needs). */
int stag_field_bytes(stag_lattice lat, int prec, unsigned long long *bytes);
/* A field that views caller-owned device memory (e.g. a torch tensor) in the
 * library's internal layout, for zero-copy use: `dev_ptr` must be device (or
 * managed) memory of the lattice's device, 16-byte aligned, with at least
 * stag_field_bytes bytes; its contents are used as they are.  The caller
 * keeps ownership: stag_field_destroy releases the view, not the memory, and
 * the memory must outlive the view.  Bad pointer, size or alignment:
 * STAG_ERR_ARG. */
int stag_field_wrap(stag_lattice lat, int parity, int prec, void *dev_ptr, unsigned long long bytes,
                    stag_field *out);

/* ---- Dslash --------------------------------------------------------------
 * out = D_eo in  (out even, in odd)    stag_dslash_eo
 * out = D_oe in  (out odd,  in even)   stag_dslash_oe
 * Both fields must have the same precision, and a gauge copy of that
 * precision must have been uploaded.  Asynchronous on the lattice stream. */
int stag_dslash_eo(stag_lattice lat, stag_field out_even, const stag_field in_odd);
int stag_dslash_oe(stag_lattice lat, stag_field out_odd, const stag_field in_even);

/* out = M in = m^2 in - D_eo D_oe in, both even.  Asynchronous. */
int stag_apply_M(stag_lattice lat, stag_field out_even, const stag_field in_even,
                 double mass);

/* ---- solvers ------------------------------------------------------------- */
typedef struct {
    int iters;             /* CG iterations performed                          */
    int status;            /* STAG_OK, STAG_ERR_NOT_CONVERGED or _BREAKDOWN    */
    double true_rel_resid; /* |b - M x| / |b| recomputed at exit in the        */
                           /* solve's outer precision (FP64 or DF64)           */
    double iter_rel_resid; /* sqrt(|r|^2 / |b|^2) of the recursive residual     */
    double seconds;        /* wall time of the solve on the device             */
    double gflops;         /* model flops / seconds                            */
    double gbs;            /* model bytes / seconds                            */
    int restarts;          /* reliable updates (mixed precision) or 0          */
    int reserved;
} stag_solve_info;

/* Solve M x = b by conjugate gradient from x0 = 0 (Hestenes-Stiefel),
 * stopping when |r| <= rel_tol |b| or after max_iter iterations.  x and b are
 * even fields of the same precision (F64 or DF64), mass > 0.  The iteration
 * runs as one CUDA graph with a device-side loop condition; the host waits
 * once, at the end.  Returns STAG_OK, STAG_ERR_NOT_CONVERGED (x holds the last
 * iterate) or STAG_ERR_BREAKDOWN; info (may be NULL) is filled in all cases. */
int stag_cg_solve(stag_lattice lat, stag_field x_even, const stag_field b_even,
                  double mass, double rel_tol, int max_iter, stag_solve_info *info);

/* stag_cg_solve with a record of the iteration: trace[3k + 0..2] receives
 * alpha_k = |r_k|^2 / <p_k, M p_k>, beta_k = |r_{k+1}|^2 / |r_k|^2 and
 * |r_{k+1}|^2 for k < min(iterations, trace_len) (host memory, caller-owned,
 * 3 * trace_len doubles; entries past the last iteration are not written).
 * The first trace_len iterations run host-driven, one launch sequence and
 * one host wait each, so that the device scalars can be read between them;
 * the arithmetic is that of stag_cg_solve.  This exposes the CG's scalar
 * recurrence for checking against an independent implementation.
 * trace NULL or trace_len < 0: STAG_ERR_ARG.  Otherwise as stag_cg_solve. */
int stag_cg_solve_traced(stag_lattice lat, stag_field x_even, const stag_field b_even,
                         double mass, double rel_tol, int max_iter, double *trace, int trace_len,
                         stag_solve_info *info);

/* Mixed-precision CG with reliable updates (Sleijpen & van der Vorst;
 * Clark et al. for lattice QCD): the iteration runs in `inner_prec`
 * (STAG_F32, or STAG_F16 = 16-bit fixed-point storage with float arithmetic),
 * and whenever the iterated residual has dropped below `delta` times its
 * largest value since the last update (e.g. delta = 0.1), or claims
 * convergence, the accumulated correction is added to x and the true
 * residual b - M x is recomputed in the precision of x and b (F64 or DF64).
 * Convergence (|b - M x| <= rel_tol |b|) is only declared on such a
 * recomputed residual, so info->true_rel_resid is the residual of the
 * returned x.  Needs gauge copies of both precisions.  info->iters counts
 * inner iterations, info->restarts the reliable updates.  Dot products and
 * the scalars of the iteration are accumulated in FP64.  Same return values
 * as stag_cg_solve. */
int stag_cg_solve_mixed(stag_lattice lat, stag_field x_even, const stag_field b_even,
                        double mass, double rel_tol, int max_iter, int inner_prec,
                        double delta, stag_solve_info *info);

/* Multi-shift CG (Jegerlehner's shifted Krylov method; the paper's Sec. 3
 * benchmarks MILC's HISQ multishift solver with 9 or 11 shifts): solves
 * (M + shifts[s]) xs[s] = b for s = 0..n-1 (1 <= n <= 32, shifts >= 0, any
 * order) with one Dslash pair per iteration, all systems sharing the Krylov
 * space of the smallest shift.  A shifted system stops updating once its
 * residual zeta_s |r| meets rel_tol |b|; the solve ends when all have.
 * xs[s] and b: distinct even fields of one precision (F64, DF64 or F32) with
 * a gauge copy of that precision.  infos (may be NULL) receives n entries:
 * per shift the iterations until it met the tolerance and the recomputed
 * true residual |b - (M + shifts[s]) xs[s]| / |b|; infos[0] also carries the
 * model GB/s and GFLOP/s of the whole solve. */
int stag_cg_multishift(stag_lattice lat, stag_field *xs, const double *shifts, int n,
                       const stag_field b, double mass, double rel_tol, int max_iter,
                       stag_solve_info *infos);

/* Mixed-precision multi-shift CG.  Phase 1: the multi-shift iteration with
 * every vector (x_s, p_s, r) in the precision of xs and b (F64 or DF64) and
 * the Dslash pair in FP32, with reliable updates (delta, as in
 * stag_cg_solve_mixed) that recompute the base system's residual in the high
 * precision; convergence is declared on such a residual.  The shifted
 * residuals cannot be recomputed inside the shared Krylov space, so phase 2
 * refines every shift whose recomputed residual misses rel_tol with
 * reliable-update CG (inner_prec F32 or F16, delta) on its own residual, the
 * correction added in the high precision.  Needs gauge copies of that
 * precision, F32 and inner_prec.  infos[s]: iters = multi-shift iterations,
 * restarts = refinement iterations, iter_rel_resid = residual after phase 1,
 * true_rel_resid = final recomputed residual, seconds = wall time of the
 * whole call. */
int stag_cg_multishift_mixed(stag_lattice lat, stag_field *xs, const double *shifts, int n,
                             const stag_field b, double mass, double rel_tol, int max_iter,
                             int inner_prec, double delta, stag_solve_info *infos);

/* Batched CG: n systems M_i x_i = b_i (1 <= n <= 64), possibly on several
 * lattices of different sizes on one device, iterate in lock step inside
 * one CUDA graph launch.  Systems on the same lattice (which must be
 * consecutive in the arrays) share every link load: the multi-right-hand-side
 * Dslash streams each link matrix once per site and applies it to up to 8
 * (FP32: one thread per site) or 4 (F64/DF64: one thread per site and
 * system, the threads of a site loading the link in one coalesced request)
 * vectors.  Each system has its own mass, scalars and
 * stopping test; the loop ends when none is running.  All fields have one
 * precision (F64, DF64 or F32) with gauge copies of it on every lattice.
 * Work runs on lats[0]'s stream (the others' streams are synchronized
 * first).  infos (may be NULL): one entry per system; infos[0].gbs/gflops
 * are the rates of the whole batch counted as if every system had been
 * solved alone. */
int stag_cg_solve_batched(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs,
                          const double *masses, double rel_tol, int max_iter,
                          stag_solve_info *infos);

/* Batched CG in FP32 to max(rel_tol, 1e-5) for all systems in one graph,
 * then every system refined to rel_tol by reliable-update CG (inner_prec F32
 * or F16, delta) on its own residual, in the precision of xs and bs (F64 or
 * DF64).  Every lattice needs gauge copies of that precision, F32 and
 * inner_prec.  infos[i]: iters = batched FP32 iterations, restarts =
 * refinement iterations, iter_rel_resid = residual after the FP32 phase,
 * true_rel_resid = final recomputed residual, seconds = wall time of the
 * call. */
int stag_cg_solve_batched_mixed(int n, stag_lattice *lats, stag_field *xs, const stag_field *bs,
                                const double *masses, double rel_tol, int max_iter, int inner_prec,
                                double delta, stag_solve_info *infos);

/* Autotuner.  Candidates, in precision `prec` on this lattice (10 launches
 * each after 2 warm-ups, CUDA events on the lattice stream):
 *   STAG_TUNE_DSLASH  the Dslash: block 64, 128, 256 or 512 threads, in two
 *                     register variants (regs 1: the compiler's choice,
 *                     2: at most 64 registers, 1024 resident threads per SM)
 *                     and, for STAG_F16 on 12-real links with Lt a multiple
 *                     of 4 and at least 8, regs 3: two sites (x, y, z, t)
 *                     and (x, y, z, t + Lt/2) per thread in packed FP32x2
 *                     arithmetic (the same bits as the one-site forms), the
 *                     next hop's loads in flight through a shared-memory
 *                     ring of cp.async copies
 *   STAG_TUNE_M       the solvers' M Dslash (m^2 p - D t with one <p, Mp>
 *                     partial per block): the same candidates
 *   STAG_TUNE_BATCH   the batched multi-right-hand-side Dslash: block 128 or
 *                     256, and the right-hand sides sharing one link load
 *                     (group: FP32 4 or 8, F64/DF64 2 or 4; decided by the
 *                     time per right-hand side); none in 16-bit storage
 * The fastest of each kind is kept for every later call on the lattice and
 * cached for the process per (dims, precision, link layout, device); when
 * the environment variable STAG_TUNE_CACHE names a file, the cache is read
 * from it at the first call and every new choice appended to it.  Every
 * candidate computes the same numbers (the block size only changes the order
 * of the solvers' partial sums).  Needs a gauge copy of `prec`; overwrites
 * the lattice's internal work vectors. */
typedef struct {
    int kernel;    /* STAG_TUNE_DSLASH, STAG_TUNE_M or STAG_TUNE_BATCH          */
    int block;     /* threads per block                                        */
    int regs;      /* Dslash: 1 free, 2 capped, 3 site pairs; batched 0      */
    int group;     /* batched: right-hand sides per group; others 0            */
    double us;     /* microseconds per launch; 0 for a choice from the cache    */
    int chosen;    /* 1 for the configuration kept                             */
} stag_tune_result;
enum { STAG_TUNE_DSLASH = 0, STAG_TUNE_M = 1, STAG_TUNE_BATCH = 2 };
enum { STAG_TUNE_FORCE = 1 };  /* time again even if the cache holds a choice */

/* Tune (or take the cached choice, *cached = 1: then only the chosen
 * configurations are reported, untimed).  out: up to cap results; *n the
 * number written.  flags: 0 or STAG_TUNE_FORCE.  n, cached may be NULL. */
int stag_lattice_autotune_all(stag_lattice lat, int prec, unsigned flags, stag_tune_result *out, int cap,
                              int *n, int *cached);

/* Set one kind's configuration by hand (regs 0 = the library's default
 * variant, 1..3 as above, 3 falling back to the default where the pair
 * form does not apply; group 0 = the largest).  Bad values: STAG_ERR_ARG. */
int stag_lattice_set_tuning(stag_lattice lat, int prec, int kernel, int block, int regs, int group);

/* The autotuner, timed again (STAG_TUNE_FORCE): dslash_us[2] and batch_us[2]
 * (may be NULL) receive, for blocks of 128 and 256 threads, the fastest
 * Dslash candidate's microseconds per launch and the batched Dslash's time
 * for one launch over the largest group at its fastest group size (0 for
 * STAG_F16). */
int stag_lattice_autotune(stag_lattice lat, int prec, double *dslash_us, double *batch_us);

/* ---- learned preconditioner ------------------------------------------------
 * The paper has no learned preconditioner; this one is a small
 * gauge-equivariant convolutional network (in the manner of Lehner and
 * Wettig's preconditioner networks for lattice QCD) trained on the GPU by
 * the library's own forward and backward kernels and applied inside
 * flexible CG.  Layers 1 -> C -> C -> 1 channels of colour vectors on the
 * full lattice, no nonlinearity:
 *
 *   y_o(x) = sum_i [ W[0][o][i] psi_i(x)
 *                    + sum_mu ( W[1+2mu][o][i] V_mu(x) psi_i(x+mu)
 *                             + W[2+2mu][o][i] V_mu(x-mu)^+ psi_i(x-mu) ) ]
 *
 * with V_mu(x) = eta_mu(x) U_mu(x), the fat links with the Kogut-Susskind
 * phases eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) and the lattice's boundary
 * sign on wrapping hops (no coefficients), and complex colour-blind
 * weights, so the net is gauge covariant.  The phases let the net's
 * translation-invariant weights form the operator's own two-hop paths
 * (D^2 = sum over hop pairs with constant coefficients on phased links),
 * and with them a degree-one polynomial in M; on raw links the paths that
 * turn from one direction to another carry site-dependent signs, and the
 * trained net cut CG iterations 1.42x instead of 1.80x (32^3x64, m = 0.005).  As a preconditioner it maps an even residual r
 * (zero on odd sites) to z = N(r) restricted to the even sites.  Weights:
 * (re, im) doubles, layer 1 [9][C][1], layer 2 [9][C][C], layer 3 [9][1][C],
 * concatenated (9 * (2C + C^2) complex numbers).
 *
 * Evaluation.  The net is linear and its weights commute with the
 * transports, so on an even input with even outputs kept it equals the
 * two-hop path sum
 *   z(x) = c0 r(x) + sum_{a,b} C[a][b] T_a T_b r(x),  T_d one hop d (or 1),
 *   c0 = W3[0] W2[0] W1[0],
 *   C[a][b] = W3[0] W2[a] W1[b] + W3[a] W2[0] W1[b] + W3[a] W2[b] W1[0]
 * (products over the channels).  The library evaluates the net in that form
 * (two stencil kernels: 16 link matrices and about 1.4k multiply-adds per
 * even site) and trains the layer weights through it (the chain rule from
 * dL/dC* to dL/dW*).  FP32 arithmetic; inside the solver the weights are
 * rounded to binary16 and the links read from a 16-bit copy (fixed point,
 * one scale for the field).  When the fat links are special unitary (within
 * 1e-6, checked at creation) that copy keeps rows 0 and 1 only and the
 * kernels rebuild row 2 as s conj(row 0 x row 1), s = eta b the link's phase
 * and boundary sign (the paper's 12-real compression, Sec. 4); otherwise
 * all nine entries. */
typedef struct stag_net_s *stag_net;

/* Create a net with C = channels (1, 2, 4 or 8) on `lat` from the raw fat
 * links (canonical complex128 [4][V][3][3]; a NaN, an infinity or an entry
 * beyond the FP32 range gives STAG_ERR_ARG).  Initial weights: the identity
 * map plus seeded noise; with C = 8 layer 1 puts each hop in a channel of
 * its own and layer 3 reads the identity path (noise N(0, 1e-3)), so that
 * layer 3's hop weights set the two-hop paths linearly; with fewer channels
 * the identity through every channel (noise N(0, 1e-2)).  Counts as a live object of the
 * lattice: destroy nets before their lattice. */
int stag_net_create(stag_lattice lat, const double *fat, int ptr_kind, int channels, unsigned seed,
                    stag_net *out);
int stag_net_destroy(stag_net n);
int stag_net_num_weights(const stag_net n, int *count);  /* complex weights */
int stag_net_set_weights(stag_net n, const double *w);   /* resets the optimiser state */
int stag_net_get_weights(const stag_net n, double *w);

/* out = N(in) on distinct even fields of one precision (F64, DF64 or F32)
 * of the net's lattice.  flags: 0, or an OR of STAG_NET_FP16_WEIGHTS (round
 * the weights to binary16 first), STAG_NET_LINKS16 (read the 16-bit link
 * copy) and STAG_NET_HERMITIAN (apply the Hermitian part (N + N^+)/2
 * instead); the three together are the form the learned solvers apply.
 * Other bits give STAG_ERR_ARG.  Asynchronous. */
enum { STAG_NET_FP16_WEIGHTS = 1, STAG_NET_LINKS16 = 2, STAG_NET_HERMITIAN = 4 };
int stag_net_apply(stag_net n, stag_field out_even, const stag_field in_even, int flags);

/* Training pairs from the plain CG: solve M x* = b to rel_tol, then rerun
 * the same iteration and, every `stride` iterations (at most max_pairs
 * times), store the pair (r_k, e_k = x* - x_k) in FP32 on the device.
 * b is an even field with a gauge copy of its precision; *collected receives
 * the number of pairs added.  Pairs accumulate over calls. */
int stag_net_collect_pairs(stag_net n, const stag_field b, double mass, double rel_tol, int stride,
                           int max_pairs, int *collected);
int stag_net_num_pairs(const stag_net n, int *count);
/* Copy pair k to the host as canonical complex128 [Vh][3] (r and e, FP32
 * values widened). */
int stag_net_get_pair(const stag_net n, int k, double *r, double *e);

/* Training objective.
 * STAG_NET_LOSS_ERROR (default): sum over pairs of |N(r) - e|^2 / |e|^2.
 * STAG_NET_LOSS_RESIDUAL: sum over pairs of |M N(r) - r|^2 / |r|^2 with M at
 *   the mass the pairs were collected with, differentiated through M (FP32
 *   Dslash; needs an F32 gauge copy).  It weights the upper spectrum, where a
 *   local operator can compress the condition number of N M. */
enum { STAG_NET_LOSS_ERROR = 0, STAG_NET_LOSS_RESIDUAL = 1 };
int stag_net_set_loss(stag_net n, int kind);

/* Loss (the objective above) summed over pairs [first, first+count), and its
 * gradient dL/dW* (the Wirtinger derivative with respect to the conjugate
 * weights; dL/dRe W = 2 Re, dL/dIm W = 2 Im of it), same layout as the
 * weights.  loss or grad may be NULL. */
int stag_net_loss_grad(stag_net n, int first, int count, double *loss, double *grad);

/* Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the mean loss over mini-batches
 * of `batch` pairs for `epochs` passes over the collected pairs, shuffled
 * with `seed`; the step size decays from lr to lr/10 (cosine) over the
 * epochs, and over the net's first 100 Adam steps it ramps up linearly from
 * lr/100 (so that a short run leaves the net near its start instead of
 * throwing every weight by about lr per step).  With the residual loss, the
 * first training call first rescales
 * the last layer by the least-squares optimal factor for the pairs.
 * epoch_loss (may be NULL) receives the mean loss per epoch. */
int stag_net_train(stag_net n, int epochs, int batch, double lr, unsigned seed, double *epoch_loss);

/* Flexible CG (Notay; Polak-Ribiere beta on real inner products) for
 * M x = b with z = N_h(r) as the preconditioner, N_h = (N + N^+)/2 the
 * Hermitian part of the net (binary16 weights, 16-bit links; CG's
 * recurrences assume a Hermitian preconditioner, and a briefly trained net
 * is far from Hermitian: at 32^3x64 its Hermitian part needed 229 CG
 * iterations where the net itself needed 635), from x0 = 0.  A run that
 * claims convergence is checked against the recomputed residual and
 * restarted if they drifted apart; after a breakdown (<r, z> <= 0), or the
 * iteration limit, plain CG (z = r) continues from the current x.
 * Convergence means |b - M x| <= rel_tol |b| recomputed in the precision of
 * x and b (F64 or DF64 for an FP64-accurate result).  info->iters counts all
 * iterations, info->restarts the fallbacks to plain CG, info->seconds is
 * wall time. */
int stag_cg_solve_learned(stag_net n, stag_field x_even, const stag_field b_even, double mass,
                          double rel_tol, int max_iter, stag_solve_info *info);

/* Mixed-precision flexible CG with the net: the iteration of
 * stag_cg_solve_mixed (inner_prec STAG_F32 or STAG_F16 storage, reliable
 * updates at `delta` in the precision of x and b, F64 or DF64) with
 * z = N(r_s) as the preconditioner, applied in inner_prec (binary16 weights,
 * 16-bit links), Polak-Ribiere beta, and Fletcher-Reeves beta after a
 * reliable update (r_s replaced by the recomputed residual).  Convergence is
 * declared on a recomputed true residual, as in stag_cg_solve_mixed.  Needs
 * gauge copies of x's precision and inner_prec.  If the flexible iteration
 * breaks down or does not converge, stag_cg_solve_mixed runs from x = 0;
 * info->iters and info->restarts then count both runs.  info->seconds is
 * wall time. */
int stag_cg_solve_learned_mixed(stag_net n, stag_field x_even, const stag_field b_even, double mass,
                                double rel_tol, int max_iter, int inner_prec, double delta,
                                stag_solve_info *info);

/* ---- allocation-free M ---------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code invoked while its caller captures
 * a CUDA graph, services that hand out fixed device buffers up front, or
 * programs whose own allocator owns all device memory.  Creating a lattice
 * allocates, so such callers cannot use stag_apply_M.
 *
 * out_even = m^2 in_even - D_eo D_oe in_even, computed on the caller's
 * buffers in the canonical layouts (no lattice handle, no upload):
 *   fat, lng   complex128 [4][V][3][3] raw links (c1, c3, phases and
 *              boundary signs are applied by the kernel)
 *   in_even    complex128 [Vh][3], out_even complex128 [Vh][3] (distinct)
 * All four must be device memory of the current CUDA device; dims and bc as
 * for stag_lattice_create (bc NULL = {+1,+1,+1,-1}).  FP64 arithmetic.
 *
 * Limit: Vh = V/2 <= 65536 (e.g. 16^4, 16^3 x 32); larger lattices return
 * STAG_ERR_ARG.  The odd intermediate D_oe in_even lives in a 3 MiB array
 * compiled into the library (held on every GPU that loads it until the
 * process exits); every call overwrites all of the part it reads, so nothing
 * needs clearing between calls, but two calls that overlap on the GPU (on
 * different streams or devices sharing a context) race on that array.
 * The first call on a device looks up the array's device address (set-up
 * done once per device, with that device current); make that first call
 * before any stream capture.  Calls no allocating CUDA routine.  Asynchronous
 * on `cuda_stream` (NULL = legacy default stream). */
int stag_apply_M_noalloc(const int dims[4], const double bc[4], double c1, double c3,
                         const double *fat, const double *lng, double mass,
                         const double *in_even, double *out_even, void *cuda_stream);

/* ---- domain decomposition, emulated on one GPU ---------------------------
 * The paper's multi-node runs (Sec. 2 and 3) split the lattice over ranks,
 * each applying Dslash to its part after exchanging the boundary sites of
 * the input with its neighbours.  These calls reproduce that data movement
 * on one device: the t direction is cut into `ndomains` slabs of
 * Lt / ndomains slices (the first Lt % ndomains slabs one more); each slab's
 * Dslash reads a private copy of the input that holds the slab and the three
 * slices on either side (the reach of the three-link term), filled by
 * device-to-device copies as a halo exchange would, and writes the outputs
 * of its slab only.  The global sums of the CG are per-slab partial sums
 * added on the host in slab order, as an allreduce would.  The results equal
 * the single-domain calls up to the order of the summation.
 * Each slab also reads its links from a private copy holding only its own
 * link slices and the three below it (the exchange a multi-GPU upload does
 * once).  1 <= ndomains <= Lt, else STAG_ERR_ARG.  Each call allocates one
 * field and one link copy per slab on the device and frees them before
 * returning. */

/* out = D in, as stag_dslash_eo / stag_dslash_oe (out's parity selects
 * which), computed slab by slab.  Fields of opposite parity, one precision
 * (any), with a gauge copy of that precision; synchronous. */
int stag_dd_dslash(stag_lattice lat, int ndomains, stag_field out, const stag_field in);

/* stag_cg_solve computed slab by slab with host-reduced inner products (one
 * host round trip per reduction: a model of the multi-node solver's data
 * flow, not a fast path).  Same fields, arguments and return values as
 * stag_cg_solve; info->seconds is wall time, gflops and gbs are 0. */
int stag_dd_cg_solve(stag_lattice lat, int ndomains, stag_field x_even, const stag_field b_even,
                     double mass, double rel_tol, int max_iter, stag_solve_info *info);

/* ---- domain decomposition over ranks ----------------------------------------
 * The paper's multi-node MILC runs (Sec. 2 and 3) split the lattice over MPI
 * ranks that exchange the boundary sites of the vector Dslash acts on and sum
 * the CG's inner products globally.  Here the t direction is cut into `size`
 * slabs, one per rank, as for stag_dd_* (rank r owns slices [t0, t0 + nt),
 * nt = Lt / size, the first Lt % size ranks one more; every nt must be >= 3).
 * Each rank holds a full-size lattice on its own GPU with the whole gauge
 * field uploaded: a rank reads the links of its slab and of the three slices
 * below it, and the upload is their exchange.  Fields on a rank carry values
 * on its slab; the library overwrites the three slices on either side (the
 * halo) of every vector it applies Dslash to, and leaves the rest alone.
 * Before each Dslash a rank sends the three lowest slices of the input to
 * rank - 1 and the three highest to rank + 1 (periodically) and receives its
 * halo from them; the CG's global sums (|b|^2, <p, Mp>, |r|^2) are the slab
 * sums added by the communicator's allreduce.
 *
 * The communicator is the caller's (MPI, a torch.distributed group, NCCL
 * through stag_comm_nccl_create, ...).  A message is the three slices of one
 * parity in the field's internal layout: component plane by component plane,
 * each 3 * Lx*Ly*Lz/2 entries (16-bit fields: one plane of 16-byte cells,
 * the site's three components and its norm). */
typedef struct {
    void *ctx;           /* passed back to the callbacks                          */
    int rank, size;      /* 0 <= rank < size                                      */
    int device_buffers;  /* 0: exchange gets host memory and completes before it
                            returns; 1: device memory of the rank's device, and it
                            may enqueue the transfer on `stream` (the lattice's)   */
    /* send `bytes` of to_prev to rank - 1 and of to_next to rank + 1 (mod size);
     * receive from rank - 1 into from_prev and from rank + 1 into from_next.
     * With size 1 both neighbours are the rank itself.  Returns 0 on success. */
    int (*exchange)(void *ctx, const void *to_prev, const void *to_next, void *from_prev, void *from_next,
                    unsigned long long bytes, void *stream);
    /* sum n doubles (host memory) over all ranks, in place; the same result on
     * every rank.  Returns 0 on success. */
    int (*allreduce)(void *ctx, double *vals, int n);
    /* optional (NULL if absent; needs device_buffers = 1): the same sum of n
     * doubles in device memory, enqueued on `stream` without waiting.  With
     * it the CG's sums stay on the device and the host waits once every
     * eight iterations instead of twice per iteration. */
    int (*allreduce_dev)(void *ctx, double *dev_vals, int n, void *stream);
} stag_comm;

typedef struct stag_ddr_s *stag_ddr;

/* The slab of rank `rank` of `size` on a lattice `dims`: t0 and nt.  Host
 * only; STAG_ERR_ARG for bad dims or a slab thinner than 3 slices. */
int stag_ddr_layout(const int dims[4], int size, int rank, int *t0, int *nt);

/* The halo exchange of one parity field held in host memory in the
 * canonical layout (complex128 [Vh][3], full size): the halo slices of
 * `field` are filled from the neighbours' boundary slices through `comm`
 * (whose device_buffers must be 0), with the messages the device path sends
 * (converted to complex128).  Host only: it lets a test on machines without
 * a GPU drive the protocol.  Errors: STAG_ERR_ARG, or STAG_ERR_STATE when a
 * callback fails. */
int stag_ddr_exchange_host(const int dims[4], int parity, const stag_comm *comm, double *field);

/* A rank's view of a decomposed lattice: `lat` is the rank's full-size
 * lattice (gauge uploaded in the precisions used), `comm` is copied. */
int stag_ddr_create(stag_lattice lat, const stag_comm *comm, stag_ddr *out);
int stag_ddr_destroy(stag_ddr d);

/* out = D in on the rank's slab (out's parity selects D_eo or D_oe), after
 * exchanging in's halo; fields of opposite parity and one precision with a
 * gauge copy of it.  Synchronous. */
int stag_ddr_dslash(stag_ddr d, stag_field out, stag_field in);

/* CG for M x = b over all ranks (every rank calls it with its slab of b);
 * the rank's slab of x receives its part of the solution.  F64 or DF64
 * fields.  Per iteration: two halo exchanges, each overlapped with the
 * stencil on the slab's interior (slices more than three from a face; slabs
 * of at least 7 slices), and two allreduces of one value each.  alpha, beta
 * and the stopping test are computed on the device from the global sums, so
 * every rank takes the same decisions; with comm->allreduce_dev the iteration
 * is enqueued in chunks of eight with one host wait per chunk (iterations
 * after the stop do nothing but the exchanges), else the host waits for each
 * allreduce.  info->true_rel_resid is |b - M x| / |b| over the whole lattice
 * (one more exchange and allreduce).  Same return values as stag_cg_solve,
 * the same on every rank. */
int stag_ddr_cg_solve(stag_ddr d, stag_field x, const stag_field b, double mass, double rel_tol, int max_iter,
                      stag_solve_info *info);

/* NCCL as the communicator: device-buffer exchange (grouped ncclSend/ncclRecv
 * on the stream it is given), allreduce (ncclAllReduce of the doubles through
 * a device buffer) and the device allreduce (ncclAllReduce in place on the
 * stream).  stag_comm_nccl_id writes a new 128-byte unique id on one
 * rank, which the caller distributes; every rank then calls
 * stag_comm_nccl_create with it, its rank and the device it uses (a
 * collective call).  STAG_ERR_STATE if the library was built without NCCL. */
int stag_comm_nccl_id(unsigned char id[128]);
int stag_comm_nccl_create(int rank, int size, const unsigned char id[128], int device, stag_comm *out);
int stag_comm_nccl_destroy(stag_comm *c);

/* ---- diagnostics ----------------------------------------------------------
 * The neighbour arithmetic of the Dslash kernels, run on the host: the
 * checkerboard index of the site reached from site `cb` of parity `parity`
 * by `steps` (+-1 or +-3) hops along direction mu (0..3 = x, y, z, t) on a
 * lattice `dims` (each even, >= 2), periodic in index space, and the number
 * of times that hop wraps around the lattice (the exponent of the boundary
 * sign).  Site order: full index i = x + Lx (y + Ly (z + Lz t)), cb = i / 2
 * within a parity, parity = (x + y + z + t) mod 2.  Lets a test check every
 * hop the kernels take against a brute-force table without a GPU.  The paper
 * has no counterpart.  Bad arguments: STAG_ERR_ARG. */
int stag_cb_neighbor(const int dims[4], int parity, long long cb, int mu, int steps,
                     long long *out_cb, int *out_wraps);

/* ---- errors -------------------------------------------------------------- */
const char *stag_strerror(int status);
const char *stag_last_error_message(void);

/* Library version, e.g. "0.1.0". */
const char *stag_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STAG_H */
