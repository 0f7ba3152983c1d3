/*
 * Plain FP64 CPU oracle for the improved-staggered (Naik) Dslash and the
 * even-odd preconditioned conjugate-gradient solve of Li & Gottlieb,
 * "Staggered Dslash Performance on Intel Xeon Phi Architecture" (Lattice 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call
 * this code: only the tests, the package's smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA path.
 *
 * It is written to be checked by eye, not to be fast: one output site per
 * loop iteration, coefficients, Kogut-Susskind phases and boundary signs
 * applied explicitly at every hop (nothing folded into the links), complex
 * arithmetic through C99 <complex.h>, serial dot products in site order.
 * The only concession to speed is an OpenMP loop over output sites, which
 * does not change any result (each site is computed independently).
 *
 * Layouts (complex128, C order):
 *   gauge  U[mu][i][a][b], mu = 0..3 = x,y,z,t, site i = x + Lx*(y + Ly*(z + Lz*t))
 *   full-lattice colour field  psi[i][a]
 *   one-parity colour field    psi[cb][a], cb = i / 2 for the sites of that
 *                              parity, parity = (x+y+z+t) mod 2 (0 = even).
 *
 * The operator (the paper's Sec. 3 describes it in words: 16 SU(3)
 * matrix-vector products over the 8 forward/backward directions, with 1-link
 * and 3-link matrices, summed into one colour vector per site):
 *
 *   (D psi)(x) = sum_mu eta_mu(x) { c1 [ b(x,+1) U_mu(x) psi(x+mu)
 *                                       - b(x,-1) U_mu(x-mu)^+ psi(x-mu) ]
 *                                 + c3 [ b(x,+3) N_mu(x) psi(x+3mu)
 *                                       - b(x,-3) N_mu(x-3mu)^+ psi(x-3mu) ] }
 *
 * Readings where the paper is silent (it prints no equations):
 *   - eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}), the Kogut-Susskind phases the
 *     paper says are absorbed into the gauge fields (Sec. 4);
 *   - b(x,s) = bc_mu^w with w = floor((x_mu + s) / L_mu), the number of times
 *     the hop wraps around the lattice (bc_mu = +1 periodic, -1 antiperiodic);
 *   - N_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu), the "three-link products" of
 *     Sec. 4, built from the raw (unphased, unscaled) links with periodic
 *     indexing;
 *   - no factor 1/2 in D; M = m^2 - D_eo D_oe acts on even sites;
 *   - hops that land on the same site (lattices shorter than 7 in a
 *     direction) all contribute: their terms add.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

static long volume_of(const int L[4])
{
    return (long)L[0] * L[1] * L[2] * L[3];
}

/* coordinates of site i, x fastest */
static void coords_of(const int L[4], long i, int x[4])
{
    for (int mu = 0; mu < 4; mu++) {
        x[mu] = (int)(i % L[mu]);
        i /= L[mu];
    }
}

static long site_of(const int L[4], const int x[4])
{
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

static int parity_of(const int x[4])
{
    return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* Kogut-Susskind phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) */
static double eta_of(const int x[4], int mu)
{
    int s = 0;
    for (int nu = 0; nu < mu; nu++)
        s += x[nu];
    return (s & 1) ? -1.0 : 1.0;
}

/* The site reached from x by s steps along mu (periodic in index space);
 * *sign receives bc_mu^w where w counts how often the hop wrapped. */
static long hop(const int L[4], const double bc[4], const int x[4], int mu, int s,
                double *sign)
{
    int y[4] = {x[0], x[1], x[2], x[3]};
    int w = 0;
    y[mu] += s;
    while (y[mu] >= L[mu]) {
        y[mu] -= L[mu];
        w++;
    }
    while (y[mu] < 0) {
        y[mu] += L[mu];
        w--;
    }
    *sign = pow(bc[mu], (double)w);
    return site_of(L, y);
}

/* ------------------------------------------------------------------ */
/* 3x3 complex linear algebra                                          */
/* ------------------------------------------------------------------ */

static const cplx *link_at(const cplx *G, long V, int mu, long i)
{
    return G + ((long)mu * V + i) * 9;
}

/* y += s * A v */
static void add_mat_vec(cplx y[3], double s, const cplx *A, const cplx *v)
{
    for (int a = 0; a < 3; a++) {
        cplx t = 0;
        for (int b = 0; b < 3; b++)
            t += A[a * 3 + b] * v[b];
        y[a] += s * t;
    }
}

/* y += s * A^+ v, A^+ the Hermitian conjugate */
static void add_adj_mat_vec(cplx y[3], double s, const cplx *A, const cplx *v)
{
    for (int a = 0; a < 3; a++) {
        cplx t = 0;
        for (int b = 0; b < 3; b++)
            t += conj(A[b * 3 + a]) * v[b];
        y[a] += s * t;
    }
}

/* C = A B */
static void mat_mul(cplx *C, const cplx *A, const cplx *B)
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            cplx t = 0;
            for (int c = 0; c < 3; c++)
                t += A[a * 3 + c] * B[c * 3 + b];
            C[a * 3 + b] = t;
        }
}

/* ------------------------------------------------------------------ */
/* long links: the three-link products of Sec. 4                       */
/* ------------------------------------------------------------------ */

/* N_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu), periodic indexing, no signs. */
void orc_long_links(const int L[4], const cplx *U, cplx *N)
{
    const long V = volume_of(L);
    const double periodic[4] = {1.0, 1.0, 1.0, 1.0};
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {
        int x[4];
        coords_of(L, i, x);
        for (int mu = 0; mu < 4; mu++) {
            double unused;
            long j1 = hop(L, periodic, x, mu, 1, &unused);
            long j2 = hop(L, periodic, x, mu, 2, &unused);
            cplx T[9];
            mat_mul(T, link_at(U, V, mu, i), link_at(U, V, mu, j1));
            mat_mul(N + ((long)mu * V + i) * 9, T, link_at(U, V, mu, j2));
        }
    }
}

/* ------------------------------------------------------------------ */
/* Dslash                                                               */
/* ------------------------------------------------------------------ */

/* (D psi)(x) at one site x (full-lattice index i).  psi_at(j) gives the
 * colour vector at site j. */
static void dslash_site(const int L[4], const double bc[4], double c1, double c3,
                        const cplx *U, const cplx *N, const cplx *psi, int psi_is_cb,
                        long i, cplx out[3])
{
    const long V = volume_of(L);
    int x[4];
    coords_of(L, i, x);
    out[0] = out[1] = out[2] = 0;
    for (int mu = 0; mu < 4; mu++) {
        const double eta = eta_of(x, mu);
        double b;
        long j;
        /* one-link forward:  + c1 b(x,+1) U_mu(x) psi(x+mu) */
        j = hop(L, bc, x, mu, +1, &b);
        add_mat_vec(out, eta * c1 * b, link_at(U, V, mu, i), psi + (psi_is_cb ? j / 2 : j) * 3);
        /* one-link backward: - c1 b(x,-1) U_mu(x-mu)^+ psi(x-mu) */
        j = hop(L, bc, x, mu, -1, &b);
        add_adj_mat_vec(out, -eta * c1 * b, link_at(U, V, mu, j), psi + (psi_is_cb ? j / 2 : j) * 3);
        /* three-link forward:  + c3 b(x,+3) N_mu(x) psi(x+3mu) */
        j = hop(L, bc, x, mu, +3, &b);
        add_mat_vec(out, eta * c3 * b, link_at(N, V, mu, i), psi + (psi_is_cb ? j / 2 : j) * 3);
        /* three-link backward: - c3 b(x,-3) N_mu(x-3mu)^+ psi(x-3mu) */
        j = hop(L, bc, x, mu, -3, &b);
        add_adj_mat_vec(out, -eta * c3 * b, link_at(N, V, mu, j), psi + (psi_is_cb ? j / 2 : j) * 3);
    }
}

/* D on the full lattice: out[i] = (D psi)(i) for every site i. */
void orc_dslash_full(const int L[4], const double bc[4], double c1, double c3,
                     const cplx *U, const cplx *N, const cplx *psi, cplx *out)
{
    const long V = volume_of(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++)
        dslash_site(L, bc, c1, c3, U, N, psi, 0, i, out + i * 3);
}

/* D restricted to output parity out_par (0: D_eo, 1: D_oe).  in_cb holds the
 * other parity, out_cb receives the output parity, both in checkerboard
 * order (position i/2). */
void orc_dslash_parity(const int L[4], const double bc[4], double c1, double c3,
                       const cplx *U, const cplx *N, int out_par,
                       const cplx *in_cb, cplx *out_cb)
{
    const long V = volume_of(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {
        int x[4];
        coords_of(L, i, x);
        if (parity_of(x) != out_par)
            continue;
        dslash_site(L, bc, c1, c3, U, N, in_cb, 1, i, out_cb + (i / 2) * 3);
    }
}

/* D at a list of full-lattice sites only (for sampled checks on lattices
 * too large to compare whole): out[k] = (D psi)(sites[k]), psi given on the
 * other parity in checkerboard order. */
void orc_dslash_sites(const int L[4], const double bc[4], double c1, double c3,
                      const cplx *U, const cplx *N, const cplx *in_cb,
                      const long *sites, long n, cplx *out)
{
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++)
        dslash_site(L, bc, c1, c3, U, N, in_cb, 1, sites[k], out + k * 3);
}

/* M = m^2 - D_eo D_oe on the even checkerboard (the even-odd preconditioned
 * normal operator the CG solves). */
void orc_apply_M(const int L[4], const double bc[4], double c1, double c3,
                 const cplx *U, const cplx *N, double mass,
                 const cplx *in_even, cplx *out_even)
{
    const long Vh = volume_of(L) / 2;
    cplx *t = malloc(sizeof(cplx) * 3 * Vh);
    orc_dslash_parity(L, bc, c1, c3, U, N, 1, in_even, t);
    orc_dslash_parity(L, bc, c1, c3, U, N, 0, t, out_even);
    for (long k = 0; k < 3 * Vh; k++)
        out_even[k] = mass * mass * in_even[k] - out_even[k];
    free(t);
}

/* ------------------------------------------------------------------ */
/* conjugate gradient on M                                             */
/* ------------------------------------------------------------------ */

/* <a, b> = sum conj(a) b, serial in site order */
static cplx dot(long n, const cplx *a, const cplx *b)
{
    cplx s = 0;
    for (long k = 0; k < n; k++)
        s += conj(a[k]) * b[k];
    return s;
}

static double norm2(long n, const cplx *a)
{
    double s = 0;
    for (long k = 0; k < n; k++)
        s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return s;
}

/*
 * Hestenes-Stiefel CG for M x = b on the even checkerboard, x0 = 0:
 *   alpha = |r|^2 / <p, M p>,  x += alpha p,  r -= alpha M p,
 *   beta  = |r_new|^2 / |r|^2, p = r + beta p,
 * stopping when |r| <= tol |b| or after max_iter iterations.  At exit the
 * true residual |b - M x| / |b| is recomputed.  hist (may be NULL) receives
 * alpha_k, beta_k and |r_{k+1}|^2 for every iteration k.
 *
 * Returns 0 converged, 1 not converged within max_iter, 2 breakdown
 * (<p, M p> not positive or not finite).
 */
int orc_cg(const int L[4], const double bc[4], double c1, double c3,
           const cplx *U, const cplx *N, double mass, const cplx *b, cplx *x,
           double tol, int max_iter, int *iters, double *true_rel_resid, double *hist)
{
    const long n = 3 * (volume_of(L) / 2);
    cplx *r = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n);
    cplx *Ap = malloc(sizeof(cplx) * n);
    int status = 0;
    int k = 0;

    const double bb = norm2(n, b);
    for (long q = 0; q < n; q++) {
        x[q] = 0;
        r[q] = b[q];
        p[q] = b[q];
    }
    double rr = bb;
    while (rr > tol * tol * bb && k < max_iter) {
        orc_apply_M(L, bc, c1, c3, U, N, mass, p, Ap);
        const double pAp = creal(dot(n, p, Ap));
        if (!(pAp > 0) || !isfinite(pAp)) {
            status = 2;
            break;
        }
        const double alpha = rr / pAp;
        for (long q = 0; q < n; q++) {
            x[q] += alpha * p[q];
            r[q] -= alpha * Ap[q];
        }
        const double rr_new = norm2(n, r);
        const double beta = rr_new / rr;
        for (long q = 0; q < n; q++)
            p[q] = r[q] + beta * p[q];
        if (hist) {
            hist[3 * k + 0] = alpha;
            hist[3 * k + 1] = beta;
            hist[3 * k + 2] = rr_new;
        }
        rr = rr_new;
        k++;
    }
    if (status == 0 && rr > tol * tol * bb)
        status = 1;

    /* true residual */
    orc_apply_M(L, bc, c1, c3, U, N, mass, x, Ap);
    for (long q = 0; q < n; q++)
        Ap[q] = b[q] - Ap[q];
    *true_rel_resid = bb > 0 ? sqrt(norm2(n, Ap) / bb) : 0.0;
    *iters = k;

    free(r);
    free(p);
    free(Ap);
    return status;
}

/* ------------------------------------------------------------------ */
/* gauge-covariant convolution (the learned preconditioner's layer)    */
/* ------------------------------------------------------------------ */

/*
 * One layer on the full lattice, cin input and cout output channels of
 * colour vectors, complex weights W[d][o][i] (d = 0: the site itself,
 * d = 1 + 2 mu: the neighbour x + mu transported by U_mu(x), d = 2 + 2 mu:
 * the neighbour x - mu transported by U_mu(x - mu)^+):
 *
 *   y_o(x) = sum_i [ W[0][o][i] psi_i(x)
 *                    + sum_mu ( W[1+2mu][o][i] b(x,+1) U_mu(x) psi_i(x+mu)
 *                             + W[2+2mu][o][i] b(x,-1) U_mu(x-mu)^+ psi_i(x-mu) ) ]
 *
 * with the raw links U (no phases, no coefficients) and the same boundary
 * sign b = bc_mu^w of a wrapping hop as the Dslash.  Colour-blind complex
 * weights and parallel transport make the layer gauge covariant.
 * The paper has no learned preconditioner: this layer defines the one the
 * library adds (a gauge-equivariant convolution in the sense of Lehner and
 * Wettig's gauge-equivariant preconditioners for lattice QCD).
 * psi: [cin][V][3], y: [cout][V][3].
 */
void orc_covconv(const int L[4], const double bc[4], const cplx *U, int cin, int cout,
                 const cplx *W, const cplx *psi, cplx *y)
{
    const long V = volume_of(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {
        int x[4];
        coords_of(L, i, x);
        for (int o = 0; o < cout; o++) {
            cplx acc[3] = {0, 0, 0};
            for (int c = 0; c < cin; c++) {
                const cplx *v = psi + ((long)c * V + i) * 3;
                const cplx w0 = W[(0 * cout + o) * cin + c];
                for (int a = 0; a < 3; a++)
                    acc[a] += w0 * v[a];
                for (int mu = 0; mu < 4; mu++) {
                    double b;
                    cplx t[3];
                    /* forward neighbour */
                    long j = hop(L, bc, x, mu, +1, &b);
                    t[0] = t[1] = t[2] = 0;
                    add_mat_vec(t, b, link_at(U, V, mu, i), psi + ((long)c * V + j) * 3);
                    const cplx wf = W[((1 + 2 * mu) * cout + o) * cin + c];
                    for (int a = 0; a < 3; a++)
                        acc[a] += wf * t[a];
                    /* backward neighbour */
                    j = hop(L, bc, x, mu, -1, &b);
                    t[0] = t[1] = t[2] = 0;
                    add_adj_mat_vec(t, b, link_at(U, V, mu, j), psi + ((long)c * V + j) * 3);
                    const cplx wb = W[((2 + 2 * mu) * cout + o) * cin + c];
                    for (int a = 0; a < 3; a++)
                        acc[a] += wb * t[a];
                }
            }
            for (int a = 0; a < 3; a++)
                y[((long)o * V + i) * 3 + a] = acc[a];
        }
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}
