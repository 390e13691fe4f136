/*
 * pe3d_oracle.c -- plain FP64 CPU oracle for the range march of the 3D
 * wide-angle parabolic equation (Xu, Wang, Chronopoulos, Yue, "Performance
 * Optimization and Parallelization of a Parabolic Equation Solver in
 * Computational Ocean Acoustics on Modern Many-core Computer", Sec. 2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may build or call it; the
 * library never links it, and it shares no code with the library.
 *
 * What it computes (paper Eq. 4 and the two-step procedure of Eq. 5-8, in the
 * order of the loop in Fig. 2):
 *
 *   [1 + (1/4 - d/4) X][1 - (d/4) Y] u^{j+1} = [1 + (1/4 + d/4) X][1 + (d/4) Y] u^j,
 *   d = i k0 dr,
 *
 * with, on the grid u[m][l] (m: azimuth, l: depth, depth z_l = (l+1) dz):
 *
 *   (X u)[m][l] = (n^2[m][l] - 1) u[m][l] + s (u[m][l+1] - 2 u[m][l] + u[m][l-1]),
 *                 s = 1 / (k0 dz)^2, ghosts u[m][-1] = u[m][Nz] = 0;
 *   (Y u)[m][l] = c (u[m+1][l] - 2 u[m][l] + u[m-1][l]),
 *                 c = 1 / (k0 r* dtheta)^2, walled ghosts u[-1] = u[Ntheta] = 0,
 *                 or m +- 1 taken modulo Ntheta for a full circle.
 *
 * Readings taken where the paper is silent or garbled:
 *   - X uses (n^2 - 1) + d^2/dz^2 / k0^2 (the printed k0^2 (n^2 - 1) term is
 *     dimensionally inconsistent with Eq. 2 divided by k0^2);
 *   - both sides of Eq. 4 use the operators at r* = r_{j+1}: Fig. 2 advances r
 *     before it updates A and B;
 *   - the medium is piecewise constant in range: slice k is active for
 *     R_k <= r* < R_{k+1} (slice 0 before R_0); or, as the range-dependent
 *     variant, n^2 is interpolated linearly in range between the slices around
 *     r* and held constant beyond the first and the last slice;
 *   - the full-circle azimuth system (cyclic) is solved with the Sherman-
 *     Morrison formula around a tridiagonal solve.
 *
 * The step, as Eq. 4 and Eq. 5/6 order it:
 *   1. w   = [1 + (d/4) Y] u^j            (rightmost factor of the RHS first)
 *   2. RHS = [1 + (1/4 + d/4) X] w
 *   3. v   : [1 + (1/4 - d/4) X] v = RHS, one tridiagonal system in l per m  (Eq. 5, 7)
 *   4. u^{j+1}: [1 - (d/4) Y] u^{j+1} = v, one system in m per l            (Eq. 6, 8)
 *
 * Systems are solved by textbook Gaussian elimination with partial pivoting on
 * the tridiagonal band (row interchanges, one fill-in superdiagonal), written
 * here rather than called from a library.
 *
 * Complex numbers: C99 double complex.  Build with -ffp-contract=off so that
 * every product and sum is rounded as written.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_SINGULAR = -3, OR_ERR_OOM = -2 };

/* ------------------------------------------------------------------------ */
/* Tridiagonal Gaussian elimination with partial pivoting.
 *
 * Row i of the system:  sub[i] x[i-1] + diag[i] x[i] + sup[i] x[i+1] = b[i]
 * (sub[0] and sup[n-1] are ignored).  b is overwritten with x.
 * Work arrays (length n each) are caller-supplied so the routine allocates
 * nothing.  Returns OR_ERR_SINGULAR on an exactly zero pivot.            */
static int tridiag_gepp(int n, const cplx *sub, const cplx *diag, const cplx *sup,
                        cplx *b, cplx *d, cplx *u1, cplx *u2)
{
    if (n <= 0) return OR_OK;
    /* d: current diagonal, u1: first superdiagonal, u2: fill-in second superdiagonal */
    for (int i = 0; i < n; ++i) {
        d[i] = diag[i];
        u1[i] = (i + 1 < n) ? sup[i] : 0.0;
        u2[i] = 0.0;
    }
    for (int i = 0; i + 1 < n; ++i) {
        cplx below = sub[i + 1];             /* entry (i+1, i) */
        if (cabs(d[i]) >= cabs(below)) {
            /* no interchange: eliminate (i+1, i) with row i */
            if (d[i] == 0.0) return OR_ERR_SINGULAR;
            cplx mult = below / d[i];
            d[i + 1] = d[i + 1] - mult * u1[i];
            /* row i has no entry in column i+2 (u2[i] is still zero) */
            b[i + 1] = b[i + 1] - mult * b[i];
        } else {
            /* interchange rows i and i+1, then eliminate */
            cplx mult = d[i] / below;
            cplx r_i1 = d[i + 1];                          /* old (i+1, i+1) */
            cplx r_i2 = (i + 2 < n) ? u1[i + 1] : 0.0;     /* old (i+1, i+2) */
            cplx o_i1 = u1[i];                             /* old (i, i+1)   */
            d[i] = below;
            u1[i] = r_i1;
            u2[i] = r_i2;
            d[i + 1] = o_i1 - mult * r_i1;
            if (i + 2 < n) u1[i + 1] = 0.0 - mult * r_i2;
            cplx bi = b[i];
            b[i] = b[i + 1];
            b[i + 1] = bi - mult * b[i];
        }
    }
    if (d[n - 1] == 0.0) return OR_ERR_SINGULAR;
    /* back substitution with the (up to) two superdiagonals */
    b[n - 1] = b[n - 1] / d[n - 1];
    if (n >= 2) b[n - 2] = (b[n - 2] - u1[n - 2] * b[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i)
        b[i] = (b[i] - u1[i] * b[i + 1] - u2[i] * b[i + 2]) / d[i];
    return OR_OK;
}

/* Exported for the tests: solve one tridiagonal system (x: rhs in, solution out). */
int oracle_tridiag_solve(int n, const cplx *sub, const cplx *diag, const cplx *sup, cplx *x)
{
    if (n < 0) return OR_ERR_ARG;
    if (n == 0) return OR_OK;
    cplx *w = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)n);
    if (!w) return OR_ERR_OOM;
    int rc = tridiag_gepp(n, sub, diag, sup, x, w, w + n, w + 2 * n);
    free(w);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Cyclic (periodic) tridiagonal system by the Sherman-Morrison formula.
 *
 * Row i:  sub[i] x[i-1 mod n] + diag[i] x[i] + sup[i] x[i+1 mod n] = b[i].
 * The periodic matrix is C = T + u v^T with
 *   gamma = -diag[0],  u = (gamma, 0, ..., 0, sup[n-1])^T,
 *   v = (1, 0, ..., 0, sub[0] / gamma)^T,
 * where T is C with its two corners removed and its first and last diagonal
 * entries replaced by diag[0] - gamma and diag[n-1] - sup[n-1] sub[0] / gamma.
 * Then x = y - (v.y / (1 + v.z)) z with T y = b and T z = u.
 * n = 1 collapses to one equation (sub + diag + sup) x = b.
 * work: 6 n complex numbers.                                             */
static int cyclic_sm(int n, const cplx *sub, const cplx *diag, const cplx *sup,
                     cplx *b, cplx *work)
{
    if (n <= 0) return OR_OK;
    if (n == 1) {
        cplx a = sub[0] + diag[0] + sup[0];
        if (a == 0.0) return OR_ERR_SINGULAR;
        b[0] = b[0] / a;
        return OR_OK;
    }
    cplx *tdiag = work, *z = work + n, *d = work + 2 * n, *u1 = work + 3 * n, *u2 = work + 4 * n;
    cplx *tsub = work + 5 * n;   /* T's sub-diagonal: C's, without the corner */
    cplx gamma = -diag[0];
    cplx corner_tr = sub[0];       /* C[0][n-1]  */
    cplx corner_bl = sup[n - 1];   /* C[n-1][0]  */
    for (int i = 0; i < n; ++i) {
        tdiag[i] = diag[i];
        tsub[i] = (i > 0) ? sub[i] : 0.0;
        z[i] = 0.0;
    }
    tdiag[0] = diag[0] - gamma;
    tdiag[n - 1] = diag[n - 1] - corner_bl * corner_tr / gamma;
    z[0] = gamma;
    z[n - 1] = corner_bl;
    int rc = tridiag_gepp(n, tsub, tdiag, sup, b, d, u1, u2);   /* b <- y */
    if (rc) return rc;
    rc = tridiag_gepp(n, tsub, tdiag, sup, z, d, u1, u2);       /* z <- T^-1 u */
    if (rc) return rc;
    cplx vy = b[0] + (corner_tr / gamma) * b[n - 1];
    cplx vz = z[0] + (corner_tr / gamma) * z[n - 1];
    cplx den = 1.0 + vz;
    if (den == 0.0) return OR_ERR_SINGULAR;
    cplx f = vy / den;
    for (int i = 0; i < n; ++i) b[i] = b[i] - f * z[i];
    return OR_OK;
}

int oracle_cyclic_solve(int n, const cplx *sub, const cplx *diag, const cplx *sup, cplx *x)
{
    if (n < 0) return OR_ERR_ARG;
    if (n == 0) return OR_OK;
    cplx *w = (cplx *)malloc(sizeof(cplx) * 6 * (size_t)n);
    if (!w) return OR_ERR_OOM;
    int rc = cyclic_sm(n, sub, diag, sup, x, w);
    free(w);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The discrete operators of Eq. 4, row by row.                            */

/* Row l of X for azimuth m: coefficients of u[m][l-1], u[m][l], u[m][l+1]. */
static void x_row(const cplx *n2_m, int Nz, double s, int l, cplx *lo, cplx *mid, cplx *hi)
{
    *lo = (l > 0) ? s : 0.0;
    *hi = (l + 1 < Nz) ? s : 0.0;
    *mid = (n2_m[l] - 1.0) - 2.0 * s;
}

/* u[m'][l] for the azimuth neighbour m' = m + dm (walled ghost: zero). */
static cplx theta_nb(const cplx *u, int Nz, int Nt, int periodic, int m, int dm, int l)
{
    int mm = m + dm;
    if (periodic) {
        mm = ((mm % Nt) + Nt) % Nt;
    } else if (mm < 0 || mm >= Nt) {
        return 0.0;
    }
    return u[(size_t)mm * Nz + l];
}

/* Row l of X^2, the square of the discrete X with its zero ghosts, as the
 * bands at columns l-2 .. l+2 (x2[0..4]): X's row l times X's columns.     */
static void x2_row(const cplx *n2_m, int Nz, double s, int l, cplx x2[5])
{
    for (int b = 0; b < 5; ++b) x2[b] = 0.0;
    cplx lo, mid, hi;
    x_row(n2_m, Nz, s, l, &lo, &mid, &hi);
    for (int k = l - 1; k <= l + 1; ++k) {
        if (k < 0 || k >= Nz) continue;
        const cplx xlk = (k == l - 1) ? lo : (k == l) ? mid : hi;    /* X[l][k] */
        cplx klo, kmid, khi;
        x_row(n2_m, Nz, s, k, &klo, &kmid, &khi);
        if (k - 1 >= 0) x2[(k - 1) - l + 2] += xlk * klo;           /* X[k][k-1] */
        x2[k - l + 2] += xlk * kmid;                                 /* X[k][k]   */
        if (k + 1 < Nz) x2[(k + 1) - l + 2] += xlk * khi;           /* X[k][k+1] */
    }
}

/* Banded Gaussian elimination with partial pivoting (row interchanges) for
 * an n x n system with kl = 2 sub- and ku = 2 superdiagonals, the textbook
 * band algorithm: ab holds column j of the matrix at ab[(KV + i - j) + j * LDAB]
 * for rows i in j-ku .. j+kl, with KV = kl + ku rows of room above for the
 * fill that interchanges cause.  On return ab holds the factors; b (length
 * n) is overwritten with x.  ipiv: n ints of work.                         */
enum { PB_KL = 2, PB_KU = 2, PB_KV = 4, PB_LDAB = 7 };
static int penta_gepp(int n, cplx *ab, cplx *b, int *ipiv)
{
#define AB(r, c) ab[(r) + (size_t)(c) * PB_LDAB]
    int ju = 0;
    for (int j = 0; j < n; ++j) {
        const int km = (PB_KL < n - 1 - j) ? PB_KL : n - 1 - j;
        int p = 0;
        double best = cabs(AB(PB_KV, j));
        for (int t = 1; t <= km; ++t)
            if (cabs(AB(PB_KV + t, j)) > best) { best = cabs(AB(PB_KV + t, j)); p = t; }
        ipiv[j] = j + p;
        if (AB(PB_KV + p, j) == 0.0) return OR_ERR_SINGULAR;
        const int jr = (j + PB_KU + p < n - 1) ? j + PB_KU + p : n - 1;
        if (jr > ju) ju = jr;
        if (p != 0)
            for (int c = j; c <= ju; ++c) {      /* swap rows j and j+p in columns j..ju */
                const cplx t = AB(PB_KV + j - c, c);
                AB(PB_KV + j - c, c) = AB(PB_KV + j + p - c, c);
                AB(PB_KV + j + p - c, c) = t;
            }
        for (int t = 1; t <= km; ++t) AB(PB_KV + t, j) = AB(PB_KV + t, j) / AB(PB_KV, j);
        for (int c = j + 1; c <= ju; ++c)        /* rows j+1..j+km of columns j+1..ju */
            for (int t = 1; t <= km; ++t)
                AB(PB_KV + j + t - c, c) = AB(PB_KV + j + t - c, c) - AB(PB_KV + t, j) * AB(PB_KV + j - c, c);
    }
    for (int j = 0; j < n; ++j) {                /* L y = P b */
        const int km = (PB_KL < n - 1 - j) ? PB_KL : n - 1 - j;
        if (ipiv[j] != j) { const cplx t = b[j]; b[j] = b[ipiv[j]]; b[ipiv[j]] = t; }
        for (int t = 1; t <= km; ++t) b[j + t] = b[j + t] - AB(PB_KV + t, j) * b[j];
    }
    for (int j = n - 1; j >= 0; --j) {           /* U x = y, U with KV superdiagonals */
        b[j] = b[j] / AB(PB_KV, j);
        const int i0 = (j - PB_KV > 0) ? j - PB_KV : 0;
        for (int i = i0; i < j; ++i) b[i] = b[i] - AB(PB_KV + i - j, j) * b[j];
    }
    return OR_OK;
#undef AB
}

/* The banded solver on its own (for its pins): row i of the system holds
 * columns i-2 .. i+2 in bands[5 i .. 5 i + 4] (entries outside the matrix
 * are ignored); b is overwritten with x.                                   */
int oracle_penta_solve(int n, const cplx *bands, cplx *b)
{
    if (n <= 0) return OR_ERR_ARG;
    cplx *ab = (cplx *)calloc((size_t)PB_LDAB * n, sizeof(cplx));
    int *ipiv = (int *)malloc(sizeof(int) * (size_t)n);
    if (!ab || !ipiv) { free(ab); free(ipiv); return OR_ERR_OOM; }
    for (int i = 0; i < n; ++i)
        for (int q = 0; q < 5; ++q) {
            const int col = i - 2 + q;
            if (col >= 0 && col < n) ab[(PB_KV + i - col) + (size_t)col * PB_LDAB] = bands[5 * (size_t)i + q];
        }
    int rc = penta_gepp(n, ab, b, ipiv);
    free(ab);
    free(ipiv);
    return rc;
}

/* One range step r_j -> r_j + dr, all operators evaluated at r* (Eq. 4-8).
 * u: [Nt][Nz] in/out.  n2: [Nt][Nz] slice active at r*.
 * With taylor, the depth factors are those of Eq. 3's Taylor form
 * sqrt(1 + x) ~ 1 + x/2 - x^2/8 under the same Crank-Nicolson split:
 * [1 - (d/2)(X/2 - X^2/8)] on the left, [1 + (d/2)(X/2 - X^2/8)] on the right,
 * pentadiagonal in depth; the azimuth factors are unchanged.              */
int oracle_step(int Nz, int Nt, double dz, double dtheta, double dr, double k0,
                double rstar, int periodic, const cplx *n2, cplx *u, int nthreads, int taylor)
{
    if (Nz <= 0 || Nt <= 0 || !(k0 > 0.0) || !(dz > 0.0) || !(dtheta > 0.0) || rstar <= 0.0)
        return OR_ERR_ARG;
    const cplx delta = I * (k0 * dr);
    const double s = 1.0 / ((k0 * dz) * (k0 * dz));
    const double c = 1.0 / ((k0 * rstar * dtheta) * (k0 * rstar * dtheta));
    const cplx alpha = 0.25 - delta / 4.0;   /* LHS factor of X: 1/4 - d/4 */
    const cplx beta = 0.25 + delta / 4.0;    /* RHS factor of X: 1/4 + d/4 */
    const cplx yfac = delta / 4.0;           /* factor of Y: d/4           */
    size_t npts = (size_t)Nz * Nt;
    cplx *w = (cplx *)malloc(sizeof(cplx) * npts);
    cplx *v = (cplx *)malloc(sizeof(cplx) * npts);
    if (!w || !v) { free(w); free(v); return OR_ERR_OOM; }
    int status = OR_OK;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#endif
    (void)nthreads;

    /* 1. w = [1 + (d/4) Y] u */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int m = 0; m < Nt; ++m)
        for (int l = 0; l < Nz; ++l) {
            cplx yu = c * (theta_nb(u, Nz, Nt, periodic, m, +1, l)
                           - 2.0 * u[(size_t)m * Nz + l]
                           + theta_nb(u, Nz, Nt, periodic, m, -1, l));
            w[(size_t)m * Nz + l] = u[(size_t)m * Nz + l] + yfac * yu;
        }

    /* 2-3 (Taylor form). per azimuth: RHS = [1 + (d/4) X - (d/16) X^2] w, then
     * solve [1 - (d/4) X + (d/16) X^2] v = RHS (pentadiagonal, banded GEPP) */
    if (taylor) {
#pragma omp parallel num_threads(nthreads)
        {
            cplx *ab = (cplx *)calloc((size_t)PB_LDAB * Nz + Nz, sizeof(cplx));
            int *ipiv = (int *)malloc(sizeof(int) * (size_t)Nz);
            if (!ab || !ipiv) {
#pragma omp atomic write
                status = OR_ERR_OOM;
            } else {
                cplx *rhs = ab + (size_t)PB_LDAB * Nz;
#pragma omp for schedule(static)
                for (int m = 0; m < Nt; ++m) {
                    const cplx *n2m = n2 + (size_t)m * Nz;
                    const cplx *wm = w + (size_t)m * Nz;
                    memset(ab, 0, sizeof(cplx) * (size_t)PB_LDAB * Nz);
                    for (int l = 0; l < Nz; ++l) {
                        cplx lo, mid, hi, x2[5];
                        x_row(n2m, Nz, s, l, &lo, &mid, &hi);
                        x2_row(n2m, Nz, s, l, x2);
                        const cplx xr[5] = {0.0, lo, mid, hi, 0.0};
                        cplx xw = 0.0, x2w = 0.0;
                        for (int b = 0; b < 5; ++b) {
                            const int col = l - 2 + b;
                            if (col < 0 || col >= Nz) continue;
                            xw = xw + xr[b] * wm[col];
                            x2w = x2w + x2[b] * wm[col];
                            const cplx a = (b == 2 ? 1.0 : 0.0) - (delta / 4.0) * xr[b] + (delta / 16.0) * x2[b];
                            ab[(PB_KV + l - col) + (size_t)col * PB_LDAB] = a;
                        }
                        rhs[l] = wm[l] + (delta / 4.0) * xw - (delta / 16.0) * x2w;
                    }
                    int rc = penta_gepp(Nz, ab, rhs, ipiv);
                    if (rc) {
#pragma omp atomic write
                        status = rc;
                    }
                    memcpy(v + (size_t)m * Nz, rhs, sizeof(cplx) * Nz);
                }
            }
            free(ab);
            free(ipiv);
        }
    } else
    /* 2-3. per azimuth: RHS = [1 + beta X] w, then solve [1 + alpha X] v = RHS */
#pragma omp parallel num_threads(nthreads)
    {
        cplx *sub = (cplx *)malloc(sizeof(cplx) * 7 * (size_t)Nz);
        if (!sub) {
#pragma omp atomic write
            status = OR_ERR_OOM;
        } else {
            cplx *dg = sub + Nz, *sp = sub + 2 * Nz, *rhs = sub + 3 * Nz;
            cplx *wd = sub + 4 * Nz, *wu1 = sub + 5 * Nz, *wu2 = sub + 6 * Nz;
#pragma omp for schedule(static)
            for (int m = 0; m < Nt; ++m) {
                const cplx *n2m = n2 + (size_t)m * Nz;
                const cplx *wm = w + (size_t)m * Nz;
                for (int l = 0; l < Nz; ++l) {
                    cplx lo, mid, hi;
                    x_row(n2m, Nz, s, l, &lo, &mid, &hi);
                    cplx xw = mid * wm[l];
                    if (l > 0) xw = xw + lo * wm[l - 1];
                    if (l + 1 < Nz) xw = xw + hi * wm[l + 1];
                    rhs[l] = wm[l] + beta * xw;
                    sub[l] = alpha * lo;
                    dg[l] = 1.0 + alpha * mid;
                    sp[l] = alpha * hi;
                }
                int rc = tridiag_gepp(Nz, sub, dg, sp, rhs, wd, wu1, wu2);
                if (rc) {
#pragma omp atomic write
                    status = rc;
                }
                memcpy(v + (size_t)m * Nz, rhs, sizeof(cplx) * Nz);
            }
            free(sub);
        }
    }

    /* 4. per depth: solve [1 - (d/4) Y] u' = v */
    if (status == OR_OK) {
#pragma omp parallel num_threads(nthreads)
        {
            cplx *sub = (cplx *)malloc(sizeof(cplx) * 10 * (size_t)Nt);
            if (!sub) {
#pragma omp atomic write
                status = OR_ERR_OOM;
            } else {
                cplx *dg = sub + Nt, *sp = sub + 2 * Nt, *x = sub + 3 * Nt, *work = sub + 4 * Nt;
                /* Y's row: c at m-1, -2c at m, c at m+1 (ghost-free in the periodic case) */
                for (int m = 0; m < Nt; ++m) {
                    cplx lo = (periodic || m > 0) ? c : 0.0;
                    cplx hi = (periodic || m + 1 < Nt) ? c : 0.0;
                    sub[m] = 0.0 - yfac * lo;
                    dg[m] = 1.0 - yfac * (-2.0 * c);
                    sp[m] = 0.0 - yfac * hi;
                }
#pragma omp for schedule(static)
                for (int l = 0; l < Nz; ++l) {
                    for (int m = 0; m < Nt; ++m) x[m] = v[(size_t)m * Nz + l];
                    int rc = periodic ? cyclic_sm(Nt, sub, dg, sp, x, work)
                                      : tridiag_gepp(Nt, sub, dg, sp, x, work, work + Nt, work + 2 * Nt);
                    if (rc) {
#pragma omp atomic write
                        status = rc;
                    }
                    for (int m = 0; m < Nt; ++m) u[(size_t)m * Nz + l] = x[m];
                }
                free(sub);
            }
        }
    }
    free(w);
    free(v);
    return status;
}

/* Index of the medium slice active at range r: the last k with R_k <= r,
 * or 0 when r precedes every slice.                                       */
static int active_slice(const double *slice_r, int K, double r)
{
    int k = 0;
    for (int i = 0; i < K; ++i)
        if (slice_r[i] <= r) k = i;
    return k;
}

/* n^2 at range r, linear in range between slices: for R_k <= r < R_{k+1},
 * (1 - t) n2_k + t n2_{k+1} with t = (r - R_k) / (R_{k+1} - R_k); slice 0 before
 * R_0 and slice K-1 from R_{K-1} on.  out: [Nt][Nz].                      */
static void interpolated_medium(const cplx *n2, const double *slice_r, int K, size_t npts, double r,
                                cplx *out)
{
    int k = active_slice(slice_r, K, r);
    if (k + 1 >= K || r < slice_r[k]) {
        memcpy(out, n2 + (size_t)k * npts, sizeof(cplx) * npts);
        return;
    }
    double t = (r - slice_r[k]) / (slice_r[k + 1] - slice_r[k]);
    const cplx *a = n2 + (size_t)k * npts, *b = n2 + (size_t)(k + 1) * npts;
    for (size_t i = 0; i < npts; ++i) out[i] = (1.0 - t) * a[i] + t * b[i];
}

/* The range loop of Fig. 2: steps j = 0 .. steps-1 advance r* = r0 + (j+1) dr;
 * after step j, when (j+1) is a multiple of `stride`, the field is stored as
 * out[(j+1)/stride - 1].  n2: [K][Nt][Nz]; u0, out snapshots: [Nt][Nz].
 * The medium slice is the one active at r*; Y is evaluated at r* too
 * (Fig. 2 advances r before updating A and B), or, with y_midpoint, at the
 * step's midpoint r0 + (j + 1/2) dr (the centred variant of the scheme).
 * With interp, the medium of step j is n^2 interpolated linearly in range at
 * r* (interpolated_medium) instead of the active slice.  With taylor, every
 * step takes the Taylor form of the depth factors (see oracle_step).      */
int oracle_march(int Nz, int Nt, double dz, double dtheta, double dr, double k0, int periodic,
                 const cplx *n2, const double *slice_r, int K, const cplx *u0, double r0,
                 int steps, int stride, cplx *out, int nthreads, int y_midpoint, int interp, int taylor)
{
    if (Nz <= 0 || Nt <= 0 || K <= 0 || steps < 0 || stride <= 0 || r0 <= 0.0) return OR_ERR_ARG;
    size_t npts = (size_t)Nz * Nt;
    cplx *u = (cplx *)malloc(sizeof(cplx) * npts);
    cplx *med = interp ? (cplx *)malloc(sizeof(cplx) * npts) : NULL;
    if (!u || (interp && !med)) {
        free(u);
        free(med);
        return OR_ERR_OOM;
    }
    memcpy(u, u0, sizeof(cplx) * npts);
    int rc = OR_OK;
    for (int j = 0; j < steps && rc == OR_OK; ++j) {
        double rstar = r0 + (double)(j + 1) * dr;
        double ry = y_midpoint ? r0 + ((double)j + 0.5) * dr : rstar;
        const cplx *n2j;
        if (interp) {
            interpolated_medium(n2, slice_r, K, npts, rstar, med);
            n2j = med;
        } else {
            n2j = n2 + (size_t)active_slice(slice_r, K, rstar) * npts;
        }
        rc = oracle_step(Nz, Nt, dz, dtheta, dr, k0, ry, periodic, n2j, u, nthreads, taylor);
        if (rc == OR_OK && (j + 1) % stride == 0)
            memcpy(out + (size_t)((j + 1) / stride - 1) * npts, u, sizeof(cplx) * npts);
    }
    free(u);
    free(med);
    return rc;
}
