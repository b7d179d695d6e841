/*
 * Plain FP64 CPU oracle for the spherical-harmonic transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * What it computes (ESCAPE D3.3, section 4.4.1 and 4.4.2, synthesis equation):
 *
 *   f(theta, lambda) = sum_{m=-M}^{M} e^{i m lambda}
 *                        sum_{n=|m|}^{N(m)} a_n^m Pbar_n^m(cos theta)
 *
 * and the "forward" (grid -> spectral) direction, where each coefficient is
 * the inner product of the field with one basis function (section 4.4.2),
 * evaluated with Gaussian quadrature in latitude and the rectangle rule in
 * longitude.  The two-stage split (Fourier in longitude, Legendre in
 * latitude; section 4.4.1 figure) is NOT used for speed here: every step is
 * the plain definition, with no even/odd split, no FFT and no blocking.
 *
 * Readings of the paper taken here (the paper does not define them):
 *  - theta is colatitude, mu = cos(theta) = sin(latitude).
 *  - Pbar is normalised so that int_{-1}^{1} Pbar_n^m(mu)^2 dmu = 1, with no
 *    Condon-Shortley phase.
 *  - truncation is triangular, N(m) = T; a_n^{-m} = conj(a_n^m), only m >= 0
 *    is stored.
 *  - synthesis uses e^{+i m lambda}; analysis uses e^{-i m lambda} / N_j.
 *  - a grid row with N_j points keeps wavenumbers m <= M_j =
 *    min(T, floor((N_j - 1) / 2)).
 *  - Gaussian latitudes run north to south; lambda_k = 2 pi k / N_j.
 *  - octahedral row i from either pole (i = 1 .. nlat/2) has 20 + 4 i points.
 *
 * Spectral layout: per field, m-major triangular, complex interleaved;
 * coefficient (m, n) sits at complex index m (T+1) - m (m-1)/2 + (n - m).
 * Grid layout: per field, rows north to south, concatenated.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double OR_PI = 3.14159265358979323846264338327950288;

/* complex index of (m, n) in the triangular spectral array */
static long spec_index(int T, int m, int n)
{
    return (long)m * (T + 1) - (long)m * (m - 1) / 2 + (n - m);
}

long or_nspec(int T) { return (long)(T + 1) * (T + 2) / 2; }

/* Row lengths of the grid.  kind 0: every row has nlon points.  kind 1
 * (octahedral): row i counted from the nearer pole (i = 1 .. nlat/2) has
 * 20 + 4 i points. */
int or_grid_rows(int kind, int nlat, int nlon, int *rows)
{
    if (nlat < 2 || (nlat % 2) != 0) return 1;
    for (int j = 0; j < nlat; ++j) {
        if (kind == 0) {
            if (nlon < 1) return 1;
            rows[j] = nlon;
        } else {
            int i = (j < nlat / 2) ? (j + 1) : (nlat - j);
            rows[j] = 20 + 4 * i;
        }
    }
    return 0;
}

/* Legendre polynomial P_n(x) and P_{n-1}(x) by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre_pn(int n, double x, double *pn, double *pnm1)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

/* Gauss-Legendre nodes mu_j (north to south, mu descending) and weights w_j.
 * Newton iteration on P_nlat from mu0_j = cos(pi (j - 1/4) / (nlat + 1/2));
 * stop when the step is below 1e-15 and take one more step.  The weight is
 * w = 2 / ((1 - mu^2) P'_nlat(mu)^2).  Southern nodes are the mirror images
 * of the northern ones. */
int or_gauss(int nlat, double *mu, double *w)
{
    if (nlat < 1) return 1;
    int half = (nlat + 1) / 2;
    for (int j = 1; j <= half; ++j) {
        double x = cos(OR_PI * (j - 0.25) / (nlat + 0.5));
        double pn, pnm1, dp;
        int extra = 0;
        for (int it = 0; it < 100; ++it) {
            legendre_pn(nlat, x, &pn, &pnm1);
            dp = nlat * (x * pn - pnm1) / (x * x - 1.0);
            double dx = pn / dp;
            x -= dx;
            if (extra) break;
            if (fabs(dx) < 1e-15) extra = 1;
        }
        legendre_pn(nlat, x, &pn, &pnm1);
        dp = nlat * (x * pn - pnm1) / (x * x - 1.0);
        double wj = 2.0 / ((1.0 - x * x) * dp * dp);
        mu[j - 1] = x;
        w[j - 1] = wj;
        mu[nlat - j] = -x;
        w[nlat - j] = wj;
    }
    if (nlat % 2 == 1) mu[half - 1] = 0.0;
    return 0;
}

/* All normalised associated Legendre values Pbar_n^m(mu), 0 <= m <= n <= T,
 * in the triangular spectral order.  Recurrence:
 *   Pbar_0^0 = 1/sqrt(2)
 *   Pbar_m^m = sqrt((2m+1)/(2m)) sin(theta) Pbar_{m-1}^{m-1}
 *   Pbar_{m+1}^m = sqrt(2m+3) mu Pbar_m^m
 *   Pbar_n^m = sqrt((4n^2-1)/(n^2-m^2))
 *              (mu Pbar_{n-1}^m - sqrt(((n-1)^2-m^2)/(4(n-1)^2-1)) Pbar_{n-2}^m)
 * with sin(theta) = sqrt((1 - mu)(1 + mu)). */
int or_legendre(int T, double mu, double *P)
{
    if (T < 0) return 1;
    double s = sqrt((1.0 - mu) * (1.0 + mu));
    double pmm = 1.0 / sqrt(2.0);
    for (int m = 0; m <= T; ++m) {
        if (m > 0) pmm = sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm;
        long base = spec_index(T, m, m);
        P[base] = pmm;
        if (m + 1 <= T) P[base + 1] = sqrt(2.0 * m + 3.0) * mu * pmm;
        for (int n = m + 2; n <= T; ++n) {
            double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double b = sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) /
                            (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
            P[base + (n - m)] = a * (mu * P[base + (n - m) - 1] - b * P[base + (n - m) - 2]);
        }
    }
    return 0;
}

static int row_trunc(int T, int nj)
{
    int mj = (nj - 1) / 2;
    return mj < T ? mj : T;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Fourier coefficients F_m(mu_j) = sum_{n=m}^{T} a_n^m Pbar_n^m(mu_j) for
 * every row j and m <= M_j (zero for m > M_j).  Output layout
 * [field][row j][m = 0..T][re, im]. */
int or_inv_fourier(int T, int nlat, const int *rows, const double *mu,
                   const double *spec, int nf, double *four, int nthreads)
{
    long nspec = or_nspec(T);
    set_threads(nthreads);
    int err = 0;
#pragma omp parallel
    {
        double *P = (double *)malloc(sizeof(double) * nspec);
        if (!P) {
#pragma omp atomic write
            err = 2;
        }
#pragma omp for schedule(dynamic)
        for (int j = 0; j < nlat; ++j) {
            if (!P) continue;
            or_legendre(T, mu[j], P);
            int mj = row_trunc(T, rows[j]);
            for (int f = 0; f < nf; ++f) {
                const double *a = spec + (long)f * nspec * 2;
                double *F = four + ((long)f * nlat + j) * (T + 1) * 2;
                for (int m = 0; m <= T; ++m) {
                    double re = 0.0, im = 0.0;
                    if (m <= mj) {
                        for (int n = m; n <= T; ++n) {
                            long q = spec_index(T, m, n);
                            re += a[2 * q] * P[q];
                            im += a[2 * q + 1] * P[q];
                        }
                    }
                    F[2 * m] = re;
                    F[2 * m + 1] = im;
                }
            }
        }
        free(P);
    }
    return err;
}

/* Synthesis of one row from its Fourier coefficients, directly:
 *   f_k = Re F_0 + 2 sum_{m=1}^{M_j} Re(F_m e^{i m lambda_k}),
 * lambda_k = 2 pi k / N.  e^{i m lambda_k} is taken from a table of the N
 * roots of unity indexed by (m k) mod N. */
static void synth_row(int nj, int mj, const double *F, const double *cs,
                      const double *sn, double *out)
{
    for (int k = 0; k < nj; ++k) {
        double v = F[0];
        for (int m = 1; m <= mj; ++m) {
            long t = ((long)m * k) % nj;
            v += 2.0 * (F[2 * m] * cs[t] - F[2 * m + 1] * sn[t]);
        }
        out[k] = v;
    }
}

static void roots_table(int nj, double *cs, double *sn)
{
    for (int t = 0; t < nj; ++t) {
        double ang = 2.0 * OR_PI * (double)t / (double)nj;
        cs[t] = cos(ang);
        sn[t] = sin(ang);
    }
}

static long max_row(int nlat, const int *rows)
{
    long mx = 0;
    for (int j = 0; j < nlat; ++j)
        if (rows[j] > mx) mx = rows[j];
    return mx;
}

/* Grid from Fourier coefficients (the longitude stage of the synthesis). */
int or_inv_grid_from_fourier(int T, int nlat, const int *rows,
                             const double *four, int nf, double *grid, int nthreads)
{
    long npts = 0;
    long *off = (long *)malloc(sizeof(long) * nlat);
    if (!off) return 2;
    for (int j = 0; j < nlat; ++j) { off[j] = npts; npts += rows[j]; }
    long mx = max_row(nlat, rows);
    set_threads(nthreads);
    int err = 0;
#pragma omp parallel
    {
        double *cs = (double *)malloc(sizeof(double) * mx);
        double *sn = (double *)malloc(sizeof(double) * mx);
        if (!cs || !sn) {
#pragma omp atomic write
            err = 2;
        }
#pragma omp for schedule(dynamic)
        for (int j = 0; j < nlat; ++j) {
            if (!cs || !sn) continue;
            roots_table(rows[j], cs, sn);
            int mj = row_trunc(T, rows[j]);
            for (int f = 0; f < nf; ++f) {
                const double *F = four + ((long)f * nlat + j) * (T + 1) * 2;
                synth_row(rows[j], mj, F, cs, sn, grid + (long)f * npts + off[j]);
            }
        }
        free(cs);
        free(sn);
    }
    free(off);
    return err;
}

/* Inverse transform, spectral -> grid, straight from the synthesis
 * equation. */
int or_inv_trans(int T, int nlat, const int *rows, const double *mu,
                 const double *spec, int nf, double *grid, int nthreads)
{
    double *four = (double *)malloc(sizeof(double) * (size_t)nf * nlat * (T + 1) * 2);
    if (!four) return 2;
    int e = or_inv_fourier(T, nlat, rows, mu, spec, nf, four, nthreads);
    if (!e) e = or_inv_grid_from_fourier(T, nlat, rows, four, nf, grid, nthreads);
    free(four);
    return e;
}

/* Fourier analysis of every row, directly:
 *   F_m(mu_j) = (1/N_j) sum_k f_k e^{-i m lambda_k},  m <= M_j,
 * and Im F_0 := 0 (the field is real).  Output [field][row][m = 0..T][re, im],
 * zero for m > M_j. */
int or_dir_fourier(int T, int nlat, const int *rows, const double *grid,
                   int nf, double *four, int nthreads)
{
    long npts = 0;
    long *off = (long *)malloc(sizeof(long) * nlat);
    if (!off) return 2;
    for (int j = 0; j < nlat; ++j) { off[j] = npts; npts += rows[j]; }
    long mx = max_row(nlat, rows);
    set_threads(nthreads);
    int err = 0;
#pragma omp parallel
    {
        double *cs = (double *)malloc(sizeof(double) * mx);
        double *sn = (double *)malloc(sizeof(double) * mx);
        if (!cs || !sn) {
#pragma omp atomic write
            err = 2;
        }
#pragma omp for schedule(dynamic)
        for (int j = 0; j < nlat; ++j) {
            if (!cs || !sn) continue;
            int nj = rows[j];
            roots_table(nj, cs, sn);
            int mj = row_trunc(T, nj);
            for (int f = 0; f < nf; ++f) {
                const double *g = grid + (long)f * npts + off[j];
                double *F = four + ((long)f * nlat + j) * (T + 1) * 2;
                for (int m = 0; m <= T; ++m) {
                    double re = 0.0, im = 0.0;
                    if (m <= mj) {
                        for (int k = 0; k < nj; ++k) {
                            long t = ((long)m * k) % nj;
                            re += g[k] * cs[t];
                            im -= g[k] * sn[t];
                        }
                        re /= nj;
                        im /= nj;
                    }
                    if (m == 0) im = 0.0;
                    F[2 * m] = re;
                    F[2 * m + 1] = im;
                }
            }
        }
        free(cs);
        free(sn);
    }
    free(off);
    return err;
}

/* Spectral coefficients from Fourier coefficients by Gaussian quadrature:
 *   a_n^m = sum_{j=1}^{nlat} w_j F_m(mu_j) Pbar_n^m(mu_j).
 * Parallel over fields; each field walks the rows in order. */
int or_dir_spec_from_fourier(int T, int nlat, const double *mu, const double *w,
                             const double *four, int nf, double *spec, int nthreads)
{
    long nspec = or_nspec(T);
    set_threads(nthreads);
    int err = 0;
#pragma omp parallel
    {
        double *P = (double *)malloc(sizeof(double) * nspec);
        if (!P) {
#pragma omp atomic write
            err = 2;
        }
#pragma omp for schedule(dynamic)
        for (int f = 0; f < nf; ++f) {
            if (!P) continue;
            double *a = spec + (long)f * nspec * 2;
            memset(a, 0, sizeof(double) * nspec * 2);
            for (int j = 0; j < nlat; ++j) {
                or_legendre(T, mu[j], P);
                const double *F = four + ((long)f * nlat + j) * (T + 1) * 2;
                for (int m = 0; m <= T; ++m) {
                    double fr = w[j] * F[2 * m], fi = w[j] * F[2 * m + 1];
                    for (int n = m; n <= T; ++n) {
                        long q = spec_index(T, m, n);
                        a[2 * q] += fr * P[q];
                        a[2 * q + 1] += fi * P[q];
                    }
                }
            }
        }
        free(P);
    }
    return err;
}

/* Direct transform, grid -> spectral. */
int or_dir_trans(int T, int nlat, const int *rows, const double *mu, const double *w,
                 const double *grid, int nf, double *spec, int nthreads)
{
    double *four = (double *)malloc(sizeof(double) * (size_t)nf * nlat * (T + 1) * 2);
    if (!four) return 2;
    int e = or_dir_fourier(T, nlat, rows, grid, nf, four, nthreads);
    if (!e) e = or_dir_spec_from_fourier(T, nlat, mu, w, four, nf, spec, nthreads);
    free(four);
    return e;
}
