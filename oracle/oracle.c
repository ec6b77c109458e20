/*
 * oracle.c -- plain FP64 CPU oracle for two-link staggered quark smearing.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU library computes.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no
 * source, header, table or helper with the CUDA library, and it never touches
 * a GPU.
 *
 * Paper: Gottlieb, Jeong, Strelchenko, "Two-link Staggered Quark Smearing in
 * QUDA", Lattice 2022 (arXiv:2301.05518), Sec. 2.
 *
 *   - two-link product V_mu(x) = U_mu(x) U_mu(x + mu)       (Sec. 2, text
 *     before Eq. tlLapl1; written W_i(x) here, i = x, y, z)
 *   - 4 Lap_two psi(x) = sum_mu [ V_mu(x) psi(x + 2mu)
 *                                 + V_mu^dag(x - 2mu) psi(x - 2mu) ] - 6 psi(x)
 *                                                      (Sec. 2, Eq. tlLapl1)
 *   - the same operator from single links applied twice  (Sec. 2, Eq. tlLapl2)
 *   - psi~ = (1 + (sigma/n) Lap_two)^n psi               (Sec. 2, Eq. tlSmear)
 *   - one-link hopping H psi(x) = sum_mu [ U_mu(x) psi(x + mu)
 *                                   + U_mu^dag(x - mu) psi(x - mu) ]  (Sec. 2, Eq. 2)
 *     and Gaussian smearing psi~ = C (1 + alpha H)^n psi with C = 1 (Sec. 2, Eq. 3)
 *   - gauge-smeared links in place of U_mu (Sec. 2, the remark after
 *     Eq. tlSmear): APE smearing with spatial staples and projection onto SU(3)
 *
 * Conventions (the paper is silent on them; these are the readings used):
 *   - "Delta" below is 4 Lap_two, so one smearing step is
 *     psi <- psi + (sigma / (4 n)) Delta psi, with no overall constant.
 *   - Every step is out of place: Delta acts on the whole previous iterate.
 *   - Spatial boundaries are periodic; t is never shifted.  A smear on one
 *     time slice leaves every other slice untouched.
 *   - Plain 4-D coordinates with a periodic wrap; no sublattice layout.
 *
 * Layouts (all double, complex = [re, im]):
 *   U    [t][z][y][x][mu][row][col][2], mu = x, y, z (, t): nd = 3 or 4
 *   W    [t][z][y][x][i][row][col][2],  i = x, y, z
 *   psi  [vec][t][z][y][x][color][2]
 * L[4] = {Lx, Ly, Lz, Lt}.
 *
 * Parity pins (tests/test_oracle_pins.py): fused = unfused (Eq. tlLapl1 vs
 * Eq. tlLapl2), free-field closed forms (Fourier multiplier and the exact
 * multinomial expansion), gauge covariance, Hermiticity, sublattice and slice
 * decoupling, SU(3) closure of W, staggered-phase invariance of W, dense
 * brute force on tiny lattices.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx;

static long site_of(const int L[4], int x, int y, int z, int t)
{
    return (((long)t * L[2] + z) * L[1] + y) * L[0] + x;
}

static int wrap(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* Site reached from (x, y, z, t) by d steps along spatial direction mu. */
static long neighbour(const int L[4], int x, int y, int z, int t, int mu, int d)
{
    int c[3] = {x, y, z};
    c[mu] = wrap(c[mu] + d, L[mu]);
    return site_of(L, c[0], c[1], c[2], t);
}

static cplx cmul(cplx a, cplx b)
{
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}

static cplx cconj(cplx a)
{
    cplx r = {a.re, -a.im};
    return r;
}

static cplx cadd(cplx a, cplx b)
{
    cplx r = {a.re + b.re, a.im + b.im};
    return r;
}

static cplx get(const double *p, long k)
{
    cplx r = {p[2 * k], p[2 * k + 1]};
    return r;
}

/* Pointer to the 3x3 link U_mu at a site. */
static const double *link_at(const double *U, int nd, long site, int mu)
{
    return U + ((site * nd + mu) * 9) * 2;
}

/* c = a b for 3x3 complex matrices. */
static void matmul(const double *a, const double *b, double *c)
{
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) {
            cplx acc = {0.0, 0.0};
            for (int k = 0; k < 3; ++k)
                acc = cadd(acc, cmul(get(a, r * 3 + k), get(b, k * 3 + s)));
            c[(r * 3 + s) * 2] = acc.re;
            c[(r * 3 + s) * 2 + 1] = acc.im;
        }
}

/* out += M v */
static void add_mat_vec(const double *M, const cplx *v, cplx *out)
{
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k)
            out[r] = cadd(out[r], cmul(get(M, r * 3 + k), v[k]));
}

/* out += M^dag v, (M^dag)[r][k] = conj(M[k][r]) */
static void add_dag_vec(const double *M, const cplx *v, cplx *out)
{
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k)
            out[r] = cadd(out[r], cmul(cconj(get(M, k * 3 + r)), v[k]));
}

static void load_vec(const double *psi, long site, cplx v[3])
{
    for (int c = 0; c < 3; ++c) v[c] = get(psi, site * 3 + c);
}

/* ------------------------------------------------------------------------ */
/* Two-link product, Sec. 2: W_i(x) = U_i(x) U_i(x + i), i = x, y, z.        */
/* ------------------------------------------------------------------------ */
void oracle_twolink(const double *U, int nd, const int L[4], double *W)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int t = 0; t < L[3]; ++t)
        for (int z = 0; z < L[2]; ++z)
            for (int y = 0; y < L[1]; ++y)
                for (int x = 0; x < L[0]; ++x) {
                    long s = site_of(L, x, y, z, t);
                    for (int i = 0; i < 3; ++i) {
                        long sp = neighbour(L, x, y, z, t, i, +1);
                        matmul(link_at(U, nd, s, i), link_at(U, nd, sp, i),
                               W + ((s * 3 + i) * 9) * 2);
                    }
                }
}

/* ------------------------------------------------------------------------ */
/* Delta psi = 4 Lap_two psi on the slices selected by t0 (Eq. tlLapl1).     */
/* t0 >= 0: slice t0 only; t0 < 0: every slice.  Sites of unselected slices  */
/* are not written.                                                          */
/* ------------------------------------------------------------------------ */
void oracle_apply_lap(const double *W, const int L[4], const double *psi,
                      double *out, int t0)
{
    int tb = t0 < 0 ? 0 : t0, te = t0 < 0 ? L[3] : t0 + 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int t = tb; t < te; ++t)
        for (int z = 0; z < L[2]; ++z)
            for (int y = 0; y < L[1]; ++y)
                for (int x = 0; x < L[0]; ++x) {
                    long s = site_of(L, x, y, z, t);
                    cplx acc[3], v[3];
                    load_vec(psi, s, v);
                    for (int c = 0; c < 3; ++c) {
                        acc[c].re = -6.0 * v[c].re;
                        acc[c].im = -6.0 * v[c].im;
                    }
                    for (int i = 0; i < 3; ++i) {
                        long fwd = neighbour(L, x, y, z, t, i, +2);
                        long bwd = neighbour(L, x, y, z, t, i, -2);
                        load_vec(psi, fwd, v);
                        add_mat_vec(W + ((s * 3 + i) * 9) * 2, v, acc);
                        load_vec(psi, bwd, v);
                        add_dag_vec(W + ((bwd * 3 + i) * 9) * 2, v, acc);
                    }
                    for (int c = 0; c < 3; ++c) {
                        out[(s * 3 + c) * 2] = acc[c].re;
                        out[(s * 3 + c) * 2 + 1] = acc[c].im;
                    }
                }
}

/* ------------------------------------------------------------------------ */
/* The same operator from single links transported twice (Eq. tlLapl2):     */
/*   U_i(x) [U_i(x+i) psi(x+2i)] + U_i^dag(x-i) [U_i^dag(x-2i) psi(x-2i)]     */
/* This is how the original CPU code applied it (Sec. 1).  It never forms W. */
/* ------------------------------------------------------------------------ */
void oracle_apply_lap_unfused(const double *U, int nd, const int L[4],
                              const double *psi, double *out, int t0)
{
    int tb = t0 < 0 ? 0 : t0, te = t0 < 0 ? L[3] : t0 + 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int t = tb; t < te; ++t)
        for (int z = 0; z < L[2]; ++z)
            for (int y = 0; y < L[1]; ++y)
                for (int x = 0; x < L[0]; ++x) {
                    long s = site_of(L, x, y, z, t);
                    cplx acc[3], v[3], tmp[3];
                    load_vec(psi, s, v);
                    for (int c = 0; c < 3; ++c) {
                        acc[c].re = -6.0 * v[c].re;
                        acc[c].im = -6.0 * v[c].im;
                    }
                    for (int i = 0; i < 3; ++i) {
                        long p1 = neighbour(L, x, y, z, t, i, +1);
                        long p2 = neighbour(L, x, y, z, t, i, +2);
                        long m1 = neighbour(L, x, y, z, t, i, -1);
                        long m2 = neighbour(L, x, y, z, t, i, -2);
                        /* forward: U_i(x) (U_i(x+i) psi(x+2i)) */
                        load_vec(psi, p2, v);
                        for (int c = 0; c < 3; ++c) tmp[c].re = tmp[c].im = 0.0;
                        add_mat_vec(link_at(U, nd, p1, i), v, tmp);
                        add_mat_vec(link_at(U, nd, s, i), tmp, acc);
                        /* backward: U_i^dag(x-i) (U_i^dag(x-2i) psi(x-2i)) */
                        load_vec(psi, m2, v);
                        for (int c = 0; c < 3; ++c) tmp[c].re = tmp[c].im = 0.0;
                        add_dag_vec(link_at(U, nd, m2, i), v, tmp);
                        add_dag_vec(link_at(U, nd, m1, i), tmp, acc);
                    }
                    for (int c = 0; c < 3; ++c) {
                        out[(s * 3 + c) * 2] = acc[c].re;
                        out[(s * 3 + c) * 2 + 1] = acc[c].im;
                    }
                }
}

/* psi <- psi + a * d on the selected slices. */
static void axpy_slices(const int L[4], int t0, double a, const double *d,
                        double *psi)
{
    long slice = (long)L[0] * L[1] * L[2] * 3 * 2;
    int tb = t0 < 0 ? 0 : t0, te = t0 < 0 ? L[3] : t0 + 1;
    for (int t = tb; t < te; ++t) {
        double *p = psi + (long)t * slice;
        const double *q = d + (long)t * slice;
#pragma omp parallel for schedule(static)
        for (long k = 0; k < slice; ++k) p[k] = p[k] + a * q[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Two-link smearing, Eq. tlSmear: psi <- (1 + (sigma/n) Lap_two)^n psi,    */
/* i.e. n steps of psi <- psi + (sigma/(4n)) Delta psi.  In place on each of */
/* the nvec vectors; only the selected slices change.  Returns 0, or -1 if   */
/* scratch cannot be allocated or the arguments are invalid.                 */
/* ------------------------------------------------------------------------ */
int oracle_smear(const double *W, const int L[4], double *psi, int nvec,
                 int n, double sigma, int t0)
{
    if (n < 0 || nvec < 0) return -1;
    if (n == 0 || nvec == 0) return 0;
    long vol = (long)L[0] * L[1] * L[2] * L[3];
    double *d = (double *)calloc((size_t)vol * 6, sizeof(double));
    if (!d) return -1;
    double a = sigma / (4.0 * n);
    for (int v = 0; v < nvec; ++v) {
        double *p = psi + (long)v * vol * 6;
        for (int it = 0; it < n; ++it) {
            oracle_apply_lap(W, L, p, d, t0);
            axpy_slices(L, t0, a, d, p);
        }
    }
    free(d);
    return 0;
}

/* Eq. tlSmear with the unfused operator of Eq. tlLapl2 (no W). */
int oracle_smear_unfused(const double *U, int nd, const int L[4], double *psi,
                         int nvec, int n, double sigma, int t0)
{
    if (n < 0 || nvec < 0) return -1;
    if (n == 0 || nvec == 0) return 0;
    long vol = (long)L[0] * L[1] * L[2] * L[3];
    double *d = (double *)calloc((size_t)vol * 6, sizeof(double));
    if (!d) return -1;
    double a = sigma / (4.0 * n);
    for (int v = 0; v < nvec; ++v) {
        double *p = psi + (long)v * vol * 6;
        for (int it = 0; it < n; ++it) {
            oracle_apply_lap_unfused(U, nd, L, p, d, t0);
            axpy_slices(L, t0, a, d, p);
        }
    }
    free(d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One-link hopping operator of Eq. 2 on the selected slices:                */
/*   H psi(x) = sum_mu [ U_mu(x) psi(x + mu) + U_mu^dag(x - mu) psi(x - mu) ] */
/* ------------------------------------------------------------------------ */
void oracle_apply_hop(const double *U, int nd, const int L[4], const double *psi, double *out, int t0)
{
    int tb = t0 < 0 ? 0 : t0, te = t0 < 0 ? L[3] : t0 + 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int t = tb; t < te; ++t)
        for (int z = 0; z < L[2]; ++z)
            for (int y = 0; y < L[1]; ++y)
                for (int x = 0; x < L[0]; ++x) {
                    long s = site_of(L, x, y, z, t);
                    cplx acc[3], v[3];
                    for (int c = 0; c < 3; ++c) acc[c].re = acc[c].im = 0.0;
                    for (int mu = 0; mu < 3; ++mu) {
                        long fwd = neighbour(L, x, y, z, t, mu, +1);
                        long bwd = neighbour(L, x, y, z, t, mu, -1);
                        load_vec(psi, fwd, v);
                        add_mat_vec(link_at(U, nd, s, mu), v, acc);
                        load_vec(psi, bwd, v);
                        add_dag_vec(link_at(U, nd, bwd, mu), v, acc);
                    }
                    for (int c = 0; c < 3; ++c) {
                        out[(s * 3 + c) * 2] = acc[c].re;
                        out[(s * 3 + c) * 2 + 1] = acc[c].im;
                    }
                }
}

/* Gaussian smearing of Eq. 3 with C = 1: n steps psi <- psi + alpha H psi,   */
/* each out of place; only the selected slices change.                        */
int oracle_smear_onelink(const double *U, int nd, const int L[4], double *psi, int nvec, int n, double alpha,
                         int t0)
{
    if (n < 0 || nvec < 0) return -1;
    if (n == 0 || nvec == 0) return 0;
    long vol = (long)L[0] * L[1] * L[2] * L[3];
    double *d = (double *)calloc((size_t)vol * 6, sizeof(double));
    if (!d) return -1;
    for (int v = 0; v < nvec; ++v) {
        double *p = psi + (long)v * vol * 6;
        for (int it = 0; it < n; ++it) {
            oracle_apply_hop(U, nd, L, p, d, t0);
            axpy_slices(L, t0, alpha, d, p);
        }
    }
    free(d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gauge-smeared links (Sec. 2: a smeared link may replace U_mu in the       */
/* smearing operator).  APE smearing on each time slice with the spatial     */
/* staples, every link updated from the previous iterate (Jacobi):           */
/*   V_mu(x) = (1 - a) U_mu(x) + (a/4) sum_{nu != mu} [                       */
/*       U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag                                    */
/*     + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]                            */
/*   U'_mu(x) = P(V_mu(x)): the unitary polar factor of V, times the cube     */
/*   root of its inverse determinant phase (principal branch), so det = 1.    */
/* ------------------------------------------------------------------------ */

static void dagger(const double *a, double *d)
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            d[(r * 3 + c) * 2] = a[(c * 3 + r) * 2];
            d[(r * 3 + c) * 2 + 1] = -a[(c * 3 + r) * 2 + 1];
        }
}

static cplx det3(const double *m)
{
    /* cofactor expansion along row 0 */
    cplx a = get(m, 0), b = get(m, 1), c = get(m, 2);
    cplx d = get(m, 3), e = get(m, 4), f = get(m, 5);
    cplx g = get(m, 6), h = get(m, 7), i = get(m, 8);
    cplx ei = cmul(e, i), fh = cmul(f, h), di = cmul(d, i), fg = cmul(f, g), dh = cmul(d, h), eg = cmul(e, g);
    cplx t0 = cmul(a, (cplx){ei.re - fh.re, ei.im - fh.im});
    cplx t1 = cmul(b, (cplx){di.re - fg.re, di.im - fg.im});
    cplx t2 = cmul(c, (cplx){dh.re - eg.re, dh.im - eg.im});
    cplx r = {t0.re - t1.re + t2.re, t0.im - t1.im + t2.im};
    return r;
}

/* inv = m^-1 by the adjugate; returns -1 if det(m) is zero. */
static int inverse3(const double *m, double *inv)
{
    cplx det = det3(m);
    double n2 = det.re * det.re + det.im * det.im;
    if (!(n2 > 0.0)) return -1;
    cplx rdet = {det.re / n2, -det.im / n2};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            /* cofactor of element (c, r): rows != c, columns != r */
            int r0 = c == 0 ? 1 : 0, r1 = c == 2 ? 1 : 2;
            int c0 = r == 0 ? 1 : 0, c1 = r == 2 ? 1 : 2;
            cplx p = cmul(get(m, r0 * 3 + c0), get(m, r1 * 3 + c1));
            cplx q = cmul(get(m, r0 * 3 + c1), get(m, r1 * 3 + c0));
            cplx cof = {p.re - q.re, p.im - q.im};
            if ((r + c) & 1) { cof.re = -cof.re; cof.im = -cof.im; }
            cplx v = cmul(cof, rdet);
            inv[(r * 3 + c) * 2] = v.re;
            inv[(r * 3 + c) * 2 + 1] = v.im;
        }
    return 0;
}

/* Projection onto SU(3) of a nonsingular 3x3 complex matrix M: Newton's
 * iteration X <- (X + X^-dag) / 2 for the unitary polar factor, stopped one
 * step after the change falls below 1e-12 (the iteration converges
 * quadratically), then X exp(-i phi/3) with phi = arg det X in (-pi, pi].
 * Returns 0, or -1 for a singular matrix or no convergence in 100 steps. */
int oracle_su3_project(const double *M, double *out)
{
    double X[18], Xi[18], Xid[18];
    memcpy(X, M, sizeof X);
    int settled = 0;
    for (int it = 0; it < 100; ++it) {
        if (inverse3(X, Xi) != 0) return -1;
        dagger(Xi, Xid);
        double d2 = 0.0;
        for (int k = 0; k < 18; ++k) {
            double nx = 0.5 * (X[k] + Xid[k]);
            d2 += (nx - X[k]) * (nx - X[k]);
            X[k] = nx;
        }
        if (settled) {
            settled = 2;
            break;
        }
        if (sqrt(d2) < 1e-12) settled = 1;
    }
    if (settled != 2) return -1;
    cplx det = det3(X);
    double phi = atan2(det.im, det.re);
    cplx ph = {cos(phi / 3.0), -sin(phi / 3.0)};
    for (int k = 0; k < 9; ++k) {
        cplx v = cmul(get(X, k), ph);
        out[2 * k] = v.re;
        out[2 * k + 1] = v.im;
    }
    return 0;
}

/* n APE steps with weight a on every spatial link; out has nd = 3 layout
 * [t][z][y][x][mu][3][3][2].  Returns 0, or -1 if a projection failed. */
int oracle_ape(const double *U, int nd, const int L[4], double a, int n, double *out)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    double *cur = (double *)malloc(sizeof(double) * V * 3 * 18);
    if (!cur) return -1;
    for (long s = 0; s < V; ++s)
        for (int mu = 0; mu < 3; ++mu) memcpy(cur + (s * 3 + mu) * 18, link_at(U, nd, s, mu), sizeof(double) * 18);
    int status = 0;
    for (int step = 0; step < n && status == 0; ++step) {
#pragma omp parallel for collapse(2) schedule(static) reduction(min : status)
        for (int t = 0; t < L[3]; ++t)
            for (int z = 0; z < L[2]; ++z)
                for (int y = 0; y < L[1]; ++y)
                    for (int x = 0; x < L[0]; ++x) {
                        const long s = site_of(L, x, y, z, t);
                        for (int mu = 0; mu < 3; ++mu) {
                            double Vm[18], st[18], tmp[18], tmp2[18], dg[18];
                            for (int k = 0; k < 18; ++k) st[k] = 0.0;
                            for (int nu = 0; nu < 3; ++nu) {
                                if (nu == mu) continue;
                                const long xp_nu = neighbour(L, x, y, z, t, nu, 1);
                                const long xp_mu = neighbour(L, x, y, z, t, mu, 1);
                                const long xm_nu = neighbour(L, x, y, z, t, nu, -1);
                                int c[3] = {x, y, z};
                                c[nu] = wrap(c[nu] - 1, L[nu]);
                                c[mu] = wrap(c[mu] + 1, L[mu]);
                                const long xm_nu_p_mu = site_of(L, c[0], c[1], c[2], t);
                                /* forward staple */
                                matmul(cur + (s * 3 + nu) * 18, cur + (xp_nu * 3 + mu) * 18, tmp);
                                dagger(cur + (xp_mu * 3 + nu) * 18, dg);
                                matmul(tmp, dg, tmp2);
                                for (int k = 0; k < 18; ++k) st[k] += tmp2[k];
                                /* backward staple */
                                dagger(cur + (xm_nu * 3 + nu) * 18, dg);
                                matmul(dg, cur + (xm_nu * 3 + mu) * 18, tmp);
                                matmul(tmp, cur + (xm_nu_p_mu * 3 + nu) * 18, tmp2);
                                for (int k = 0; k < 18; ++k) st[k] += tmp2[k];
                            }
                            const double *u = cur + (s * 3 + mu) * 18;
                            for (int k = 0; k < 18; ++k) Vm[k] = (1.0 - a) * u[k] + 0.25 * a * st[k];
                            if (oracle_su3_project(Vm, out + (s * 3 + mu) * 18) != 0) status = -1;
                        }
                    }
        memcpy(cur, out, sizeof(double) * V * 3 * 18);
    }
    if (n == 0) memcpy(out, cur, sizeof(double) * V * 3 * 18);
    free(cur);
    return status;
}

/* Number of OpenMP threads a parallel region here uses (1 without OpenMP). */
int oracle_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
