// Device-resident scalars of one CG solve.  The kernels of the iteration read
// and write them directly, so the host is not involved until the solve ends.
#pragma once
#include "common.cuh"

namespace stag {

// A scalar kept both as a double and as its double-float split, so that
// kernels of every precision can read it without FP64 conversions.
struct dpair {
    double d;
    float hi, lo;
};

STAG_HD dpair make_dpair(double v) {
    dpair p;
    p.d = v;
    p.hi = (float)v;
    p.lo = (float)(v - (double)p.hi);
    return p;
}

template <class R> STAG_D R scalar_as(const dpair &p);
template <> STAG_D double scalar_as<double>(const dpair &p) { return p.d; }
template <> STAG_D float scalar_as<float>(const dpair &p) { return p.hi; }
template <> STAG_D df scalar_as<df>(const dpair &p) { return df_make(p.hi, p.lo); }

enum CgStatus { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXITER = 2, CG_BREAKDOWN = 3 };

struct CgScalars {
    // inputs, set by the host before each solve
    dpair m2;        // mass^2
    double tol2;     // rel_tol^2
    int max_iter;
    int pad0;
    // state
    double bb;       // |b|^2
    double rr;       // |r_k|^2
    double rr_stop;  // tol^2 |b|^2
    double pAp;      // <p, M p>
    double true_rr;  // |b - M x|^2 at exit
    dpair alpha, beta;
    int iter;
    int status;      // CgStatus
    unsigned ticket; // grid-reduction ticket, zero between kernels
    unsigned pad1;
    cudaGraphConditionalHandle cond;  // loop condition of the solve graph
    int has_cond;
    int pad2;
    // mixed precision with reliable updates
    double delta;    // update when |r_sloppy| < delta * rmax
    double rmax;     // largest |r_sloppy| since the last update
    int reliable;    // this iteration ends with a reliable update
    int restarts;    // reliable updates so far
    // multi-shift CG: the base CG's previous alpha and beta
    double alpha_prev, beta_prev;
    // flexible CG: |r|^2 (rr holds <r, z> there)
    double fcg_rr;
    // mixed precision in a graph: condition of the reliable-update branch
    cudaGraphConditionalHandle rel_cond;
    int has_rel_cond;
    // multi-shift CG: the iteration whose solution updates have been applied
    int ms_xdone;
    // mixed precision with a flexible preconditioner: rr holds <r_s, z> and
    // beta comes from the preconditioner step, not from |r_s|^2
    int fcg;
    // mixed multi-shift: this iteration's Dslash pair in the high precision
    // (hi_op) or the low one (lo_op = !hi_op), the gates of the two paths
    int ms_hi_op, ms_lo_op;
};

// multi-shift CG
constexpr int MS_MAX = 32;

struct ShiftState {
    double zeta_prev, zeta;        // zeta_{k-1}, zeta_k
    dpair zeta_next;               // zeta_{k+1}, read by the direction update
    dpair alpha_s, beta_s;         // alpha^s_k, beta^s_k
    int active;                    // still iterating
    int iters;                     // iterations until this shift met the tolerance
};

struct MsArgs {
    int n;                         // number of shifts
    int base;                      // index of the smallest shift
    double delta[MS_MAX];          // sigma_s - sigma_base >= 0
    void *x[MS_MAX];               // solutions
    void *p[MS_MAX];               // search directions
    const void *b;                 // right-hand side
    void *r;                       // residual of the base system
    void *p_lo;                    // mixed precision: low-precision copy of the base direction
    const void *Ap_hi;             // mixed precision: M p from the high-precision path
    double theta2;                 // the high-precision path runs while |r|^2 > theta2 |b|^2
};

}  // namespace stag
