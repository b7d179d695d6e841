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

/* ------------------------------------------------------------------ derivatives
 *
 * Readings for the derivative and wind transforms of the SH dwarf's time step
 * (the paper names them, it prints no formula): the unit sphere, phi the
 * latitude (mu = sin(phi)), and
 *   H_n^m(mu) = (1 - mu^2) dPbar_n^m/dmu,
 * which stays finite at the poles.  With eps_n^m = sqrt((n^2 - m^2)/(4 n^2 - 1))
 * the normalised functions satisfy
 *   H_n^m = (n + 1) eps_n^m Pbar_{n-1}^m - n eps_{n+1}^m Pbar_{n+1}^m
 * (Pbar_{m-1}^m = 0), the textbook relation of P_n^m' to P_{n-1}^m and
 * P_{n+1}^m divided by the normalisation constants. */
static double eps_nm(int n, int m)
{
    if (n <= m) return 0.0;
    return sqrt(((double)n * n - (double)m * m) / (4.0 * n * n - 1.0));
}

/* H_n^m(mu) for all 0 <= m <= n <= T in the triangular order of T. */
int or_legendre_deriv(int T, double mu, double *H)
{
    if (T < 0) return 1;
    long n1 = or_nspec(T + 1);
    double *P = (double *)malloc(sizeof(double) * n1);
    if (!P) return 2;
    or_legendre(T + 1, mu, P);
    for (int m = 0; m <= T; ++m)
        for (int n = m; n <= T; ++n) {
            double pm1 = n - 1 >= m ? P[spec_index(T + 1, m, n - 1)] : 0.0;
            double pp1 = P[spec_index(T + 1, m, n + 1)];
            H[spec_index(T, m, n)] = (n + 1.0) * eps_nm(n, m) * pm1 - (double)n * eps_nm(n + 1, m) * pp1;
        }
    free(P);
    return 0;
}

/* Fourier coefficients of the two derivative fields of every row:
 *   dF/dlambda:            G_m = sum_n i m a_n^m Pbar_n^m(mu_j)
 *   (1 - mu^2) dF/dmu:     K_m = sum_n a_n^m H_n^m(mu_j)
 * for m <= M_j.  Layout as or_inv_fourier, twice. */
static int deriv_fourier(int T, int nlat, const int *rows, const double *mu, const double *spec, int nf,
                         double *G, double *K)
{
    long nspec = or_nspec(T);
    int err = 0;
#pragma omp parallel
    {
        double *P = (double *)malloc(sizeof(double) * nspec);
        double *H = (double *)malloc(sizeof(double) * nspec);
        if (!P || !H) {
#pragma omp atomic write
            err = 2;
        }
#pragma omp for schedule(dynamic)
        for (int j = 0; j < nlat; ++j) {
            if (!P || !H) continue;
            or_legendre(T, mu[j], P);
            or_legendre_deriv(T, mu[j], H);
            int mj = row_trunc(T, rows[j]);
            for (int f = 0; f < nf; ++f) {
                const double *a = spec + (long)f * nspec * 2;
                double *g = G + ((long)f * nlat + j) * (T + 1) * 2;
                double *k = K + ((long)f * nlat + j) * (T + 1) * 2;
                for (int m = 0; m <= T; ++m) {
                    double pr = 0.0, pi = 0.0, hr = 0.0, hi = 0.0;
                    if (m <= mj) {
                        for (int n = m; n <= T; ++n) {
                            long q = spec_index(T, m, n);
                            pr += a[2 * q] * P[q];
                            pi += a[2 * q + 1] * P[q];
                            hr += a[2 * q] * H[q];
                            hi += a[2 * q + 1] * H[q];
                        }
                    }
                    /* i m (pr + i pi) */
                    g[2 * m] = -(double)m * pi;
                    g[2 * m + 1] = (double)m * pr;
                    k[2 * m] = hr;
                    k[2 * m + 1] = hi;
                }
            }
        }
        free(P);
        free(H);
    }
    return err;
}

/* dF/dlambda and (1 - mu^2) dF/dmu (= cos(phi) dF/dphi) of each field on the
 * grid, from its spectra; out_dlam, out_dmu: [nf][npts]. */
int or_inv_trans_deriv(int T, int nlat, const int *rows, const double *mu, const double *spec, int nf,
                       double *out_dlam, double *out_dmu, int nthreads)
{
    size_t n4 = (size_t)nf * nlat * (T + 1) * 2;
    double *G = (double *)malloc(sizeof(double) * n4);
    double *K = (double *)malloc(sizeof(double) * n4);
    int e = (!G || !K) ? 2 : 0;
    set_threads(nthreads);
    if (!e) e = deriv_fourier(T, nlat, rows, mu, spec, nf, G, K);
    if (!e) e = or_inv_grid_from_fourier(T, nlat, rows, G, nf, out_dlam, nthreads);
    if (!e) e = or_inv_grid_from_fourier(T, nlat, rows, K, nf, out_dmu, nthreads);
    free(G);
    free(K);
    return e;
}

/* Wind images U = u cos(phi), V = v cos(phi) on the grid from vorticity and
 * divergence spectra (vor, div: [nf][nspec][re, im]):
 *   psi_n^m = -zeta_n^m / (n (n + 1)),  chi_n^m = -D_n^m / (n (n + 1))  (0 at n = 0)
 *   U = dchi/dlambda - (1 - mu^2) dpsi/dmu,   V = dpsi/dlambda + (1 - mu^2) dchi/dmu. */
int or_inv_trans_uv(int T, int nlat, const int *rows, const double *mu, const double *vor, const double *div,
                    int nf, double *U, double *V, int nthreads)
{
    long nspec = or_nspec(T);
    long npts = 0;
    for (int j = 0; j < nlat; ++j) npts += rows[j];
    size_t ns = (size_t)nf * nspec * 2;
    double *psi = (double *)malloc(sizeof(double) * ns);
    double *chi = (double *)malloc(sizeof(double) * ns);
    double *a = (double *)malloc(sizeof(double) * (size_t)nf * npts);
    double *b = (double *)malloc(sizeof(double) * (size_t)nf * npts);
    int e = (!psi || !chi || !a || !b) ? 2 : 0;
    if (!e) {
        for (int f = 0; f < nf; ++f)
            for (int m = 0; m <= T; ++m)
                for (int n = m; n <= T; ++n) {
                    long q = (long)f * nspec + spec_index(T, m, n);
                    double s = n == 0 ? 0.0 : -1.0 / ((double)n * (n + 1.0));
                    psi[2 * q] = s * vor[2 * q];
                    psi[2 * q + 1] = s * vor[2 * q + 1];
                    chi[2 * q] = s * div[2 * q];
                    chi[2 * q + 1] = s * div[2 * q + 1];
                }
        /* U: dchi/dlambda into U, (1 - mu^2) dpsi/dmu into b */
        e = or_inv_trans_deriv(T, nlat, rows, mu, chi, nf, U, a, nthreads);
        if (!e) e = or_inv_trans_deriv(T, nlat, rows, mu, psi, nf, V, b, nthreads);
        /* now U = dchi/dlambda, a = (1-mu^2) dchi/dmu, V = dpsi/dlambda, b = (1-mu^2) dpsi/dmu */
        if (!e)
            for (size_t i = 0; i < (size_t)nf * npts; ++i) {
                U[i] -= b[i];
                V[i] += a[i];
            }
    }
    free(psi);
    free(chi);
    free(a);
    free(b);
    return e;
}

/* Vorticity and divergence spectra from wind images U = u cos(phi),
 * V = v cos(phi) on the grid ([nf][npts]):
 *   zeta = (1 / (1 - mu^2)) (dV/dlambda - (1 - mu^2) dU/dmu),
 *   D    = (1 / (1 - mu^2)) (dU/dlambda + (1 - mu^2) dV/dmu),
 * projected on each basis function with the mu-derivative moved onto Pbar by
 * parts (U and V vanish at the poles):
 *   zeta_n^m = sum_j w_j / (1 - mu_j^2) (i m V_m Pbar_n^m + U_m H_n^m),
 *   D_n^m    = sum_j w_j / (1 - mu_j^2) (i m U_m Pbar_n^m - V_m H_n^m),
 * U_m, V_m the rows' Fourier coefficients (1/N_j sum_k e^{-i m lambda_k}). */
int or_dir_trans_vordiv(int T, int nlat, const int *rows, const double *mu, const double *w, const double *U,
                        const double *V, int nf, double *vor, double *div, int nthreads)
{
    long nspec = or_nspec(T);
    size_t n4 = (size_t)nf * nlat * (T + 1) * 2;
    double *FU = (double *)malloc(sizeof(double) * n4);
    double *FV = (double *)malloc(sizeof(double) * n4);
    int e = (!FU || !FV) ? 2 : 0;
    if (!e) e = or_dir_fourier(T, nlat, rows, U, nf, FU, nthreads);
    if (!e) e = or_dir_fourier(T, nlat, rows, V, nf, FV, nthreads);
    set_threads(nthreads);
    if (!e) {
#pragma omp parallel
        {
            double *P = (double *)malloc(sizeof(double) * nspec);
            double *H = (double *)malloc(sizeof(double) * nspec);
            if (!P || !H) {
#pragma omp atomic write
                e = 2;
            }
#pragma omp for schedule(dynamic)
            for (int f = 0; f < nf; ++f) {
                if (!P || !H) continue;
                double *z = vor + (long)f * nspec * 2;
                double *d = div + (long)f * nspec * 2;
                memset(z, 0, sizeof(double) * nspec * 2);
                memset(d, 0, sizeof(double) * nspec * 2);
                for (int j = 0; j < nlat; ++j) {
                    or_legendre(T, mu[j], P);
                    or_legendre_deriv(T, mu[j], H);
                    double c = w[j] / ((1.0 - mu[j]) * (1.0 + mu[j]));
                    const double *u = FU + ((long)f * nlat + j) * (T + 1) * 2;
                    const double *v = FV + ((long)f * nlat + j) * (T + 1) * 2;
                    for (int m = 0; m <= T; ++m) {
                        /* i m V_m and i m U_m */
                        double imvr = -(double)m * v[2 * m + 1], imvi = (double)m * v[2 * m];
                        double imur = -(double)m * u[2 * m + 1], imui = (double)m * u[2 * m];
                        for (int n = m; n <= T; ++n) {
                            long q = spec_index(T, m, n);
                            z[2 * q] += c * (imvr * P[q] + u[2 * m] * H[q]);
                            z[2 * q + 1] += c * (imvi * P[q] + u[2 * m + 1] * H[q]);
                            d[2 * q] += c * (imur * P[q] - v[2 * m] * H[q]);
                            d[2 * q + 1] += c * (imui * P[q] - v[2 * m + 1] * H[q]);
                        }
                    }
                }
                /* Im of m = 0 coefficients is zero for real fields */
                for (int n = 0; n <= T; ++n) {
                    z[2 * spec_index(T, 0, n) + 1] = 0.0;
                    d[2 * spec_index(T, 0, n) + 1] = 0.0;
                }
            }
            free(P);
            free(H);
        }
    }
    free(FU);
    free(FV);
    return e;
}
