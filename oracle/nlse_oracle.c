/*
 * nlse_oracle.c -- plain, slow, double-precision CPU reference for the
 * two-step high-order compact (2SHOC) Laplacian and the explicit RK4
 * integrator of the nonlinear Schroedinger equation (NLSE) described in
 * R. M. Caplan and R. Carretero-Gonzalez, arXiv 1109.1027.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library
 * is checked against.  Only the test suite, the smoke check and the CPU
 * baseline of the benchmark may load it.  It shares no code, header, table
 * or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is written the way the paper states it: the 2SHOC steps in the
 * paper's order (step 1 builds D, the boundary condition supplies D at the
 * boundary, step 2 re-differences D), the RK4 schedule as the paper's ten
 * numbered lines with its three work arrays, the boundary conditions of
 * Sec. 3.2 and the stability bound of Sec. 3.3.  No blocking, fusion or
 * reordering; every loop visits the grid in storage order.  Compile with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * Threads: the loops that compute one value per grid point independently of
 * the others (step 1, step 2, the boundary values, F and the RK4 axpys) carry
 * OpenMP work-sharing pragmas.  Built without -fopenmp they are ignored; with
 * it the points of such a loop are shared among threads, and since every
 * point's arithmetic is the same, the results are the same bits for any
 * thread count.  Reductions (mass, energy, the stability bound) stay serial.
 *
 * Conventions (readings of the paper where it is silent):
 *  - Grid: x_i = x_min + h*i (Sec. 2.1); n[ax] points per axis including both
 *    boundary points; one h for every axis (Secs. 2.2, 2.3).  Storage is
 *    x fastest: p = x + n0*(y + n1*z).  Complex values are interleaved
 *    (re, im) doubles.
 *  - A point is a boundary point when any active coordinate is 0 or n-1.
 *  - The standalone Laplacian returns D_b at boundary points (Sec. 3.2, the
 *    boundary value of step 1 "would also be used for the overall Laplacian
 *    boundary").
 *  - MSD "b-1" is the closest interior point: every coordinate clamped into
 *    [1, n-2] (for a face point that is its inward normal neighbour; for an
 *    edge or corner it is the diagonal inward neighbour).
 *  - Multi-storage 2SHOC needs the step-1 boundary value of each separate
 *    second derivative, which Sec. 3.2 does not give for Dirichlet.  At a
 *    point on the boundary of axis a only, D^a_b = D_b - sum of the other
 *    axes' second differences there, D_b from Eq. (dbc_lap), so that the
 *    separate derivatives add up to the boundary Laplacian.  Points on the
 *    boundary of two or more axes never enter an interior Laplacian; their
 *    separate derivatives are set to 0.
 *  - Periodic (named, not defined, in Sec. 3.2): n points per axis with
 *    spacing h and no duplicated end point (x_n = x_0); every point is
 *    interior and neighbour indices wrap.
 *  - Laplacian-zero (named in Sec. 3.2): the step-1 boundary value is
 *    D_b = 0 (Lap Psi = 0 at the boundary), and the boundary then follows the
 *    equation itself with that Laplacian, F_b = i (s|Psi_b|^2 - V_b) Psi_b.
 *  - Mass M = h^d sum_all |psi|^2; energy (the paper defines none) is the
 *    discrete Hamiltonian of Eq. (NLSE):
 *    E = h^d sum_interior [ -a Re(conj(psi) Lap psi) + V|psi|^2 - (s/2)|psi|^4 ].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Problem description.                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int dim;       /* 1, 2 or 3 */
    long n[3];     /* points per axis, boundary points included; unused axes = 1 */
    double h;      /* grid spacing */
    double a;      /* dispersion coefficient, a > 0 (Eq. NLSE) */
    double s;      /* nonlinearity coefficient (Eq. NLSE) */
    int bc;        /* 0: Dirichlet (Eqs. dbc_lap, dbc_ut); 1: MSD (Eqs. msdbc_ut, msdbc_lap);
                      2: periodic; 3: Laplacian-zero (the two further compact-friendly
                      conditions Sec. 3.2 names) */
    int lap;       /* 0: 2SHOC single storage (Sec. 2); 1: second-order central difference (CD);
                      2: 2SHOC multi storage (Eqs. 2d2shocMs1-2, 3d2shocMs1-2; in 1D the same as 0) */
} or_problem;

typedef struct { double re, im; } cplx;

static cplx c_make(double re, double im) { cplx z; z.re = re; z.im = im; return z; }
static cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static cplx c_sub(cplx a, cplx b) { return c_make(a.re - b.re, a.im - b.im); }
static cplx c_scale(double r, cplx a) { return c_make(r * a.re, r * a.im); }
static cplx c_div(cplx a, cplx b) {
    double den = b.re * b.re + b.im * b.im;
    return c_make((a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den);
}
static cplx c_times_i(cplx a) { return c_make(-a.im, a.re); }   /* i * a */
static double c_abs2(cplx a) { return a.re * a.re + a.im * a.im; }

static cplx get(const double* f, long p) { return c_make(f[2 * p], f[2 * p + 1]); }
static void put(double* f, long p, cplx z) { f[2 * p] = z.re; f[2 * p + 1] = z.im; }

static long npoints(const or_problem* P) { return P->n[0] * P->n[1] * P->n[2]; }

/* Storage index of (x, y, z); coordinates wrap on a periodic grid. */
static long idx(const or_problem* P, long x, long y, long z) {
    if (P->bc == 2) {
        x = (x % P->n[0] + P->n[0]) % P->n[0];
        y = (y % P->n[1] + P->n[1]) % P->n[1];
        z = (z % P->n[2] + P->n[2]) % P->n[2];
    }
    return x + P->n[0] * (y + P->n[1] * z);
}

static int is_boundary(const or_problem* P, long x, long y, long z) {
    if (P->bc == 2) return 0;                       /* periodic: no boundary points */
    if (x == 0 || x == P->n[0] - 1) return 1;
    if (P->dim >= 2 && (y == 0 || y == P->n[1] - 1)) return 1;
    if (P->dim >= 3 && (z == 0 || z == P->n[2] - 1)) return 1;
    return 0;
}

static long clamp_in(long v, long n) {
    if (v < 1) return 1;
    if (v > n - 2) return n - 2;
    return v;
}

/* The point "b-1" of Sec. 3.2 for boundary point (x, y, z). */
static long inward(const or_problem* P, long x, long y, long z) {
    long xi = clamp_in(x, P->n[0]);
    long yi = P->dim >= 2 ? clamp_in(y, P->n[1]) : 0;
    long zi = P->dim >= 3 ? clamp_in(z, P->n[2]) : 0;
    return idx(P, xi, yi, zi);
}

/* N = s|psi|^2 - V (Eq. nbnb1). */
static double nonlin(const or_problem* P, cplx psi, double V) {
    return P->s * c_abs2(psi) - V;
}

/* ------------------------------------------------------------------------ */
/* 2SHOC Laplacian (Sec. 2) with the step-1 boundary values of Sec. 3.2.    */
/* ------------------------------------------------------------------------ */

/* Step 1 at an interior point: the standard second-order Laplacian,
 * Eq. (2shoc1d) in 1D, Eq. (2d2shocs1) in 2D, Eq. (3d2shocs) in 3D: the sum
 * of the 2d axial neighbours minus 2d times the centre, over h^2. */
static cplx step1_interior(const or_problem* P, const double* psi, long x, long y, long z) {
    long p = idx(P, x, y, z);
    cplx sum = c_add(get(psi, idx(P, x + 1, y, z)), get(psi, idx(P, x - 1, y, z)));
    if (P->dim >= 2)
        sum = c_add(sum, c_add(get(psi, idx(P, x, y + 1, z)), get(psi, idx(P, x, y - 1, z))));
    if (P->dim >= 3)
        sum = c_add(sum, c_add(get(psi, idx(P, x, y, z + 1)), get(psi, idx(P, x, y, z - 1))));
    cplx centre = c_scale(2.0 * P->dim, get(psi, p));
    return c_scale(1.0 / (P->h * P->h), c_sub(sum, centre));
}

/* Step 2 at an interior point.
 * 1D, Eq. (2shoc1d2):  (7/6) D_i - (1/12)(D_{i+1} + D_{i-1}).
 * 2D, Eq. (2d2shocs2): -(1/12)[cross of D with centre -12]
 *                      + (1/(6h^2))[four corners of psi, centre -4].
 * 3D, Eq. (3d2shocs2): -(1/12)[six axial D, centre -10]
 *                      + (1/(6h^2))[twelve edge neighbours of psi, centre -12]. */
static cplx step2_interior(const or_problem* P, const double* psi, const double* D,
                           long x, long y, long z) {
    long p = idx(P, x, y, z);
    if (P->dim == 1) {
        cplx nb = c_add(get(D, idx(P, x + 1, y, z)), get(D, idx(P, x - 1, y, z)));
        return c_sub(c_scale(7.0 / 6.0, get(D, p)), c_scale(1.0 / 12.0, nb));
    }
    if (P->dim == 2) {
        cplx dsum = c_add(c_add(get(D, idx(P, x + 1, y, z)), get(D, idx(P, x - 1, y, z))),
                          c_add(get(D, idx(P, x, y + 1, z)), get(D, idx(P, x, y - 1, z))));
        cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(12.0, get(D, p))));
        cplx corners = c_add(c_add(get(psi, idx(P, x + 1, y + 1, z)), get(psi, idx(P, x - 1, y + 1, z))),
                             c_add(get(psi, idx(P, x + 1, y - 1, z)), get(psi, idx(P, x - 1, y - 1, z))));
        cplx ppart = c_scale(1.0 / (6.0 * P->h * P->h), c_sub(corners, c_scale(4.0, get(psi, p))));
        return c_add(dpart, ppart);
    }
    /* dim == 3 */
    cplx dsum = c_add(get(D, idx(P, x + 1, y, z)), get(D, idx(P, x - 1, y, z)));
    dsum = c_add(dsum, c_add(get(D, idx(P, x, y + 1, z)), get(D, idx(P, x, y - 1, z))));
    dsum = c_add(dsum, c_add(get(D, idx(P, x, y, z + 1)), get(D, idx(P, x, y, z - 1))));
    cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(10.0, get(D, p))));
    /* The twelve edge neighbours: both non-zero offsets in one coordinate
     * pair, the third coordinate unchanged. */
    cplx edges = c_make(0.0, 0.0);
    for (int sa = -1; sa <= 1; sa += 2)
        for (int sb = -1; sb <= 1; sb += 2) {
            edges = c_add(edges, get(psi, idx(P, x + sa, y + sb, z)));   /* x-y plane */
            edges = c_add(edges, get(psi, idx(P, x + sa, y, z + sb)));   /* x-z plane */
            edges = c_add(edges, get(psi, idx(P, x, y + sa, z + sb)));   /* y-z plane */
        }
    cplx ppart = c_scale(1.0 / (6.0 * P->h * P->h), c_sub(edges, c_scale(12.0, get(psi, p))));
    return c_add(dpart, ppart);
}

/* Step-1 boundary value D_b.
 * Dirichlet, Eq. (dbc_lap): D_b = -(s|psi_b|^2 - V_b) psi_b / a.
 * MSD, Eq. (msdbc_lap) with N from Eq. (nbnb1), and Im(i z) = Re(z):
 *   D_b = [ Re(D_{b-1} / psi_{b-1}) + (N_{b-1} - N_b)/a ] psi_b. */
static cplx boundary_D(const or_problem* P, const double* psi, const double* V, const double* D,
                       long x, long y, long z) {
    long b = idx(P, x, y, z);
    cplx pb = get(psi, b);
    double Nb = nonlin(P, pb, V[b]);
    if (P->bc == 3) return c_make(0.0, 0.0);           /* Laplacian-zero */
    if (P->bc == 0) return c_scale(-Nb / P->a, pb);
    long q = inward(P, x, y, z);
    cplx pq = get(psi, q);
    double Nq = nonlin(P, pq, V[q]);
    cplx ratio = c_div(get(D, q), pq);
    double factor = c_times_i(ratio).im + (Nq - Nb) / P->a;
    return c_scale(factor, pb);
}

/* ------------------------------------------------------------------------ */
/* Multi-storage 2SHOC (Eqs. 2d2shocMs1-2 in 2D, 3d2shocMs1-2 in 3D).        */
/* ------------------------------------------------------------------------ */

/* The second difference of psi along axis ax at (x, y, z): Eq. (2d2shocMs1),
 * Eq. (3d2shocMs1). */
static cplx delta2(const or_problem* P, const double* psi, int ax, long x, long y, long z) {
    long dx = ax == 0, dy = ax == 1, dz = ax == 2;
    cplx sum = c_add(get(psi, idx(P, x + dx, y + dy, z + dz)), get(psi, idx(P, x - dx, y - dy, z - dz)));
    return c_scale(1.0 / (P->h * P->h), c_sub(sum, c_scale(2.0, get(psi, idx(P, x, y, z)))));
}

/* Whether coordinate ax of (x, y, z) is 0 or n-1. */
static int on_axis_boundary(const or_problem* P, int ax, long x, long y, long z) {
    long c = ax == 0 ? x : (ax == 1 ? y : z);
    return c == 0 || c == P->n[ax] - 1;
}

/* Multi-storage Laplacian into lap.  Dsep: caller work space of 3 * 2N doubles
 * for D^x, D^y, D^z; Dsum (2N doubles) receives D^x + D^y (+ D^z). */
static void laplacian_ms(const or_problem* P, const double* psi, const double* V, double* Dsep,
                         double* Dsum, double* lap) {
    long N = npoints(P);
    /* Step 1 at interior points: one second difference per axis. */
    #pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < P->n[2]; ++z)
        for (long y = 0; y < P->n[1]; ++y)
            for (long x = 0; x < P->n[0]; ++x)
                if (!is_boundary(P, x, y, z))
                    for (int ax = 0; ax < P->dim; ++ax)
                        put(Dsep + 2 * N * ax, idx(P, x, y, z), delta2(P, psi, ax, x, y, z));
    /* Step-1 boundary values (Dirichlet, Eq. dbc_lap, split as stated above). */
    #pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < P->n[2]; ++z)
        for (long y = 0; y < P->n[1]; ++y)
            for (long x = 0; x < P->n[0]; ++x) {
                if (!is_boundary(P, x, y, z)) continue;
                long b = idx(P, x, y, z);
                int nb = 0, axb = -1;
                for (int ax = 0; ax < P->dim; ++ax)
                    if (on_axis_boundary(P, ax, x, y, z)) { ++nb; axb = ax; }
                for (int ax = 0; ax < P->dim; ++ax) put(Dsep + 2 * N * ax, b, c_make(0.0, 0.0));
                if (nb != 1) continue;
                cplx pb = get(psi, b);
                cplx rest = c_scale(-nonlin(P, pb, V[b]) / P->a, pb);
                for (int ax = 0; ax < P->dim; ++ax) {
                    if (ax == axb) continue;
                    cplx d = delta2(P, psi, ax, x, y, z);
                    put(Dsep + 2 * N * ax, b, d);
                    rest = c_sub(rest, d);
                }
                put(Dsep + 2 * N * axb, b, rest);
            }
    /* Step 2 at interior points, Eq. (2d2shocMs2) / Eq. (3d2shocMs2):
     * (7/6) sum_a D^a_c - (1/12) sum_a (D^a at the two neighbours along a).
     * Boundary points take D_b of Eq. (dbc_lap), as in the single-storage form. */
    #pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < P->n[2]; ++z)
        for (long y = 0; y < P->n[1]; ++y)
            for (long x = 0; x < P->n[0]; ++x) {
                long p = idx(P, x, y, z);
                cplx centre = c_make(0.0, 0.0), nbrs = c_make(0.0, 0.0);
                for (int ax = 0; ax < P->dim; ++ax) {
                    const double* Da = Dsep + 2 * N * ax;
                    long dx = ax == 0, dy = ax == 1, dz = ax == 2;
                    centre = c_add(centre, get(Da, p));
                    if (!is_boundary(P, x, y, z))
                        nbrs = c_add(nbrs, c_add(get(Da, idx(P, x + dx, y + dy, z + dz)),
                                                 get(Da, idx(P, x - dx, y - dy, z - dz))));
                }
                put(Dsum, p, centre);
                if (is_boundary(P, x, y, z)) {
                    cplx pb = get(psi, p);
                    put(lap, p, c_scale(-nonlin(P, pb, V[p]) / P->a, pb));
                } else {
                    put(lap, p, c_sub(c_scale(7.0 / 6.0, centre), c_scale(1.0 / 12.0, nbrs)));
                }
            }
}

/* Laplacian of psi into lap (2N doubles).  With P->lap == 0 this is the
 * 2SHOC scheme; with P->lap == 1 it is the second-order CD scheme (D itself);
 * with P->lap == 2 (d >= 2) the multi-storage 2SHOC scheme.  D is
 * caller-provided work space of 2N doubles (8N for the multi-storage form)
 * and holds step 1 (for the multi-storage form: the sum of the separate
 * second derivatives) on return. */
static void laplacian(const or_problem* P, const double* psi, const double* V, double* D,
                      double* lap) {
    if (P->lap == 2 && P->dim >= 2) {
        laplacian_ms(P, psi, V, D + 2 * npoints(P), D, lap);
        return;
    }
    /* Step 1, interior points first. */
    #pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < P->n[2]; ++z)
        for (long y = 0; y < P->n[1]; ++y)
            for (long x = 0; x < P->n[0]; ++x)
                if (!is_boundary(P, x, y, z))
                    put(D, idx(P, x, y, z), step1_interior(P, psi, x, y, z));
    /* Step-1 boundary condition (the MSD form needs the interior D). */
    #pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < P->n[2]; ++z)
        for (long y = 0; y < P->n[1]; ++y)
            for (long x = 0; x < P->n[0]; ++x)
                if (is_boundary(P, x, y, z))
                    put(D, idx(P, x, y, z), boundary_D(P, psi, V, D, x, y, z));
    /* Step 2 (2SHOC) or D itself (CD); the boundary keeps D_b. */
    #pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < P->n[2]; ++z)
        for (long y = 0; y < P->n[1]; ++y)
            for (long x = 0; x < P->n[0]; ++x) {
                long p = idx(P, x, y, z);
                if (is_boundary(P, x, y, z) || P->lap == 1)
                    put(lap, p, get(D, p));
                else
                    put(lap, p, step2_interior(P, psi, D, x, y, z));
            }
}

/* ------------------------------------------------------------------------ */
/* Right-hand side F(psi) (Sec. 3.1) with the boundary conditions.          */
/* ------------------------------------------------------------------------ */

/* Doubles of work space that rhs() needs for N points: the Laplacian's D
 * work space (8N, room for the multi-storage form) and Lap (2N). */
static long rhs_work_len(long N) { return 10 * N; }

/* F = i [ a Lap psi + (s|psi|^2 - V) psi ] at interior points (Sec. 3.1).
 * Boundary: Dirichlet, Eq. (dbc_ut): F_b = 0.
 *           MSD, Eq. (msdbc_ut): F_b = i Im(F_{b-1} / psi_{b-1}) psi_b.
 * work: rhs_work_len(N) doubles. */
static void rhs(const or_problem* P, const double* psi, const double* V, double* F, double* work) {
    long N = npoints(P);
    double* D = work;
    double* lap = work + 8 * N;
    laplacian(P, psi, V, D, lap);
    #pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < P->n[2]; ++z)
        for (long y = 0; y < P->n[1]; ++y)
            for (long x = 0; x < P->n[0]; ++x) {
                if (is_boundary(P, x, y, z)) continue;
                long p = idx(P, x, y, z);
                cplx ps = get(psi, p);
                cplx inner = c_add(c_scale(P->a, get(lap, p)), c_scale(nonlin(P, ps, V[p]), ps));
                put(F, p, c_times_i(inner));
            }
    #pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < P->n[2]; ++z)
        for (long y = 0; y < P->n[1]; ++y)
            for (long x = 0; x < P->n[0]; ++x) {
                if (!is_boundary(P, x, y, z)) continue;
                long b = idx(P, x, y, z);
                if (P->bc == 0) {
                    put(F, b, c_make(0.0, 0.0));
                } else if (P->bc == 3) {
                    /* Laplacian-zero: the equation with Lap_b = 0 */
                    cplx pb = get(psi, b);
                    put(F, b, c_times_i(c_scale(nonlin(P, pb, V[b]), pb)));
                } else {
                    long q = inward(P, x, y, z);
                    double w = c_div(get(F, q), get(psi, q)).im;
                    put(F, b, c_times_i(c_scale(w, get(psi, b))));
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Classic RK4 as the ten numbered lines of Eq. (RK4).                       */
/* ------------------------------------------------------------------------ */

/* Work arrays of one RK4 step: the paper's K_tot, K_tmp, psi_tmp (Sec. 3.1)
 * and the D / Lap space that rhs() needs. */
typedef struct { double *Ktot, *Ktmp, *ptmp, *work; } rk4_space;

static int rk4_alloc(rk4_space* W, long N) {
    W->Ktot = (double*)malloc(sizeof(double) * 2 * N);
    W->Ktmp = (double*)malloc(sizeof(double) * 2 * N);
    W->ptmp = (double*)malloc(sizeof(double) * 2 * N);
    W->work = (double*)malloc(sizeof(double) * rhs_work_len(N));
    return !(W->Ktot && W->Ktmp && W->ptmp && W->work);
}

static void rk4_free(rk4_space* W) {
    free(W->Ktot); free(W->Ktmp); free(W->ptmp); free(W->work);
}

/* psi <- one RK4 step of size k, the ten numbered lines of Eq. (RK4). */
static void rk4_step(const or_problem* P, double k, double* psi, const double* V, rk4_space* W) {
    long N = npoints(P);
    double *Ktot = W->Ktot, *Ktmp = W->Ktmp, *ptmp = W->ptmp, *work = W->work;
    long p;

    rhs(P, psi, V, Ktot, work);                                               /* K_tot = F(psi) */
#pragma omp parallel for schedule(static)
    for (p = 0; p < N; ++p) put(ptmp, p, c_add(get(psi, p), c_scale(k / 2.0, get(Ktot, p))));  /* psi_tmp */
    rhs(P, ptmp, V, Ktmp, work);                                              /* K_tmp = F(psi_tmp) */
#pragma omp parallel for schedule(static)
    for (p = 0; p < N; ++p) put(Ktot, p, c_add(get(Ktot, p), c_scale(2.0, get(Ktmp, p))));    /* K_tot += 2 K_tmp */
#pragma omp parallel for schedule(static)
    for (p = 0; p < N; ++p) put(ptmp, p, c_add(get(psi, p), c_scale(k / 2.0, get(Ktmp, p))));  /* psi_tmp */
    rhs(P, ptmp, V, Ktmp, work);                                              /* K_tmp = F(psi_tmp) */
#pragma omp parallel for schedule(static)
    for (p = 0; p < N; ++p) put(Ktot, p, c_add(get(Ktot, p), c_scale(2.0, get(Ktmp, p))));    /* K_tot += 2 K_tmp */
#pragma omp parallel for schedule(static)
    for (p = 0; p < N; ++p) put(ptmp, p, c_add(get(psi, p), c_scale(k, get(Ktmp, p))));        /* psi_tmp */
    rhs(P, ptmp, V, Ktmp, work);                                              /* K_tmp = F(psi_tmp) */
#pragma omp parallel for schedule(static)
    for (p = 0; p < N; ++p)                                                   /* the new state */
        put(psi, p, c_add(get(psi, p), c_scale(k / 6.0, c_add(get(Ktot, p), get(Ktmp, p)))));
}

/* ------------------------------------------------------------------------ */
/* Linearised stability bound, Eq. (kdfull) with Tables t:bc2, t:sumresults. */
/* ------------------------------------------------------------------------ */

/* The sets G of Table t:sumresults, in units of 1/12. */
static const double G1[] = {64, 63, 46, 12, -3, -4};
static const double G2[] = {128, 127, 126, 110, 109, 92, 24, 9, 8, -6, -7, -8};
static const double G3[] = {192, 191, 190, 189, 174, 173, 172, 156, 155, 138, 36, 21,
                            20, 6, 5, 4, -9, -10, -11, -12};

/* k_max = sqrt(8) h^2 / (a * max{ ||B||_inf, max_{i, g in G} |L_i - g| }),
 * L_i = (h^2/a)(s|psi_i|^2 - V_i) over every grid point, and B_b from
 * Table t:bc2: 0 for Dirichlet, (h^2/(i a)) (1/psi_{b-1}) F_{b-1} for MSD
 * (modulus taken), evaluated on the given state. */
static double stability_dt(const or_problem* P, const double* psi, const double* V) {
    const double* G; int nG;
    if (P->dim == 1) { G = G1; nG = (int)(sizeof(G1) / sizeof(G1[0])); }
    else if (P->dim == 2) { G = G2; nG = (int)(sizeof(G2) / sizeof(G2[0])); }
    else { G = G3; nG = (int)(sizeof(G3) / sizeof(G3[0])); }
    long N = npoints(P);
    double h2a = P->h * P->h / P->a;
    double worst = 0.0;
    for (long p = 0; p < N; ++p) {
        double L = h2a * nonlin(P, get(psi, p), V[p]);
        for (int g = 0; g < nG; ++g) {
            double d = fabs(L - G[g] / 12.0);
            if (d > worst) worst = d;
        }
    }
    if (P->bc == 1) {
        double* F = (double*)malloc(sizeof(double) * 2 * N);
        double* work = (double*)malloc(sizeof(double) * rhs_work_len(N));
        rhs(P, psi, V, F, work);
        for (long z = 0; z < P->n[2]; ++z)
            for (long y = 0; y < P->n[1]; ++y)
                for (long x = 0; x < P->n[0]; ++x) {
                    if (!is_boundary(P, x, y, z)) continue;
                    long q = inward(P, x, y, z);
                    /* B_b = (h^2/(i a)) F_q / psi_q ; |1/i| = 1. */
                    double B = h2a * sqrt(c_abs2(c_div(get(F, q), get(psi, q))));
                    if (B > worst) worst = B;
                }
        free(F); free(work);
    }
    return sqrt(8.0) / worst * h2a;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (called through ctypes by the test harness).       */
/* ------------------------------------------------------------------------ */

static int make_problem(or_problem* P, int dim, const long* n, double h, double a, double s,
                        int bc, int lap) {
    if (dim < 1 || dim > 3) return 1;
    P->dim = dim;
    for (int ax = 0; ax < 3; ++ax) P->n[ax] = ax < dim ? n[ax] : 1;
    for (int ax = 0; ax < dim; ++ax) if (P->n[ax] < 3) return 1;
    if (!(h > 0.0) || !(a > 0.0)) return 1;
    if (bc < 0 || bc > 3) return 1;
    if (lap != 0 && lap != 1 && lap != 2) return 1;
    if (lap == 2 && (bc == 1 || bc == 3) && dim > 1) return 1;   /* multi storage: Dirichlet or periodic */
    P->h = h; P->a = a; P->s = s; P->bc = bc; P->lap = lap;
    return 0;
}

/* Laplacian (2SHOC or CD) of psi; boundary points receive D_b.  When D_out is
 * not NULL it receives the step-1 field D. */
int oracle_laplacian(int dim, const long* n, double h, double a, double s, int bc, int lap,
                     const double* psi, const double* V, double* lap_out, double* D_out) {
    or_problem P;
    if (make_problem(&P, dim, n, h, a, s, bc, lap)) return 1;
    long N = npoints(&P);
    double* D = (double*)malloc(sizeof(double) * 8 * N);
    laplacian(&P, psi, V, D, lap_out);
    if (D_out) memcpy(D_out, D, sizeof(double) * 2 * N);
    free(D);
    return 0;
}

/* Right-hand side F(psi) including the boundary rule. */
int oracle_rhs(int dim, const long* n, double h, double a, double s, int bc, int lap,
               const double* psi, const double* V, double* F) {
    or_problem P;
    if (make_problem(&P, dim, n, h, a, s, bc, lap)) return 1;
    double* work = (double*)malloc(sizeof(double) * rhs_work_len(npoints(&P)));
    rhs(&P, psi, V, F, work);
    free(work);
    return 0;
}

/* nsteps RK4 steps of size k, in place. */
int oracle_run(int dim, const long* n, double h, double a, double s, int bc, int lap,
               double k, long nsteps, double* psi, const double* V) {
    or_problem P;
    if (make_problem(&P, dim, n, h, a, s, bc, lap)) return 1;
    rk4_space W;
    if (rk4_alloc(&W, npoints(&P))) { rk4_free(&W); return 2; }
    for (long t = 0; t < nsteps; ++t) rk4_step(&P, k, psi, V, &W);
    rk4_free(&W);
    return 0;
}

/* Mass, energy and the stability bound of the given state. */
int oracle_invariants(int dim, const long* n, double h, double a, double s, int bc, int lap,
                      const double* psi, const double* V, double* mass, double* energy,
                      double* dt_max) {
    or_problem P;
    if (make_problem(&P, dim, n, h, a, s, bc, lap)) return 1;
    long N = npoints(&P);
    double hd = pow(P.h, (double)P.dim);
    double* D = (double*)malloc(sizeof(double) * 8 * N);
    double* lap_f = (double*)malloc(sizeof(double) * 2 * N);
    laplacian(&P, psi, V, D, lap_f);
    double m = 0.0, e = 0.0;
    for (long z = 0; z < P.n[2]; ++z)
        for (long y = 0; y < P.n[1]; ++y)
            for (long x = 0; x < P.n[0]; ++x) {
                long p = idx(&P, x, y, z);
                cplx ps = get(psi, p);
                double rho = c_abs2(ps);
                m += rho;
                if (is_boundary(&P, x, y, z)) continue;
                cplx lp = get(lap_f, p);
                double re_conj_psi_lap = ps.re * lp.re + ps.im * lp.im;
                e += -P.a * re_conj_psi_lap + V[p] * rho - 0.5 * P.s * rho * rho;
            }
    *mass = hd * m;
    *energy = hd * e;
    *dt_max = stability_dt(&P, psi, V);
    free(D); free(lap_f);
    return 0;
}

/* Number of threads of the OpenMP build (the serial build ignores it and
 * reports 1).  Returns the number the loops will use. */
#ifdef _OPENMP
#include <omp.h>
int oracle_set_threads(int n) {
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}
#else
int oracle_set_threads(int n) {
    (void)n;
    return 1;
}
#endif
