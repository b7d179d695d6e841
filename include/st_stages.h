/*
 * st_stages.h -- the individual steps of the transform as separate entry
 * points, for parity checks of each step and for callers that fuse their own
 * work between the two stages.  Same conventions as st.h (device pointers,
 * asynchronous on `stream`, status codes).
 *
 * The "Fourier buffer" is the plan's workspace between the Legendre stage and
 * the FFT stage (the two stages of ESCAPE D3.3 section 4.4.1's figure).  For
 * the northern Gaussian row j (0 = nearest the north pole) and its mirror row
 * nlat-1-j it holds, for every kept m and field, the pair
 *   inverse: S = (F_m(mu_j) + F_m(-mu_j)) / 2,  A = (F_m(mu_j) - F_m(-mu_j)) / 2
 *   direct:  E = F_m(mu_j) + F_m(-mu_j),        O = F_m(mu_j) - F_m(-mu_j)
 * where F_m is the Fourier coefficient of the row (the even/odd split that
 * halves the Legendre work; Pbar_n^m(-mu) = (-1)^(n-m) Pbar_n^m(mu)).
 */
#ifndef ST_STAGES_H
#define ST_STAGES_H

#include "st.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Gauss-Legendre nodes (north to south) and weights by Newton iteration on
 * P_nlat, FP64 on the device; mu_dev and w_dev hold nlat doubles each.
 * ST_ERR_ARG if nlat < 2 or a pointer is NULL. */
st_status st_gauss_nodes(int nlat, double *mu_dev, double *w_dev, void *stream);

/* Normalised associated Legendre values Pbar_n^m(mu) for 0 <= m <= n <= T at
 * nmu points, FP64 three-term recurrence on the device (the Pbar of section
 * 4.4.1's synthesis equation).  out_dev[i * (T+1)(T+2)/2 + q] with q the
 * triangular index of (m, n).  ST_ERR_ARG if T < 0, nmu < 1 or a pointer is
 * NULL. */
st_status st_legendre_values(int T, const double *mu_dev, int nmu, double *out_dev, void *stream);

/* Inverse Legendre stage: spectra -> Fourier buffer (S, A). */
st_status st_inv_legendre(st_plan_t plan, const void *spec_dev, int nfields, void *stream);

/* Inverse FFT stage: Fourier buffer (S, A) -> grid. */
st_status st_inv_fft(st_plan_t plan, void *grid_dev, int nfields, void *stream);

/* Direct FFT stage: grid -> Fourier buffer (E, O), scaled by 1/N_j. */
st_status st_dir_fft(st_plan_t plan, const void *grid_dev, int nfields, void *stream);

/* Direct Legendre stage: Fourier buffer (E, O) -> spectra. */
st_status st_dir_legendre(st_plan_t plan, void *spec_dev, int nfields, void *stream);

/* Copy the Fourier buffer, as last written by the inverse (direction 0) or
 * direct (direction 1) stage for `nfields` fields, into out_dev as FP64
 * complex [2 (S,A or E,O)][T+1 (m)][nlat/2 (j)][nfields][re, im]; entries with
 * m > M_j are written as 0.  Hi/lo split storage is summed back. */
st_status st_fourier_export(st_plan_t plan, int direction, int nfields, double *out_dev,
                            void *stream);

/*
 * Failure-path test hook (not in the paper).  what = 1: the plan's next
 * tensor-core Legendre launch issues no operand copies, so the bounded wait
 * of its MMA issuer on the first stage runs out after wait_ms milliseconds;
 * the kernel then records the timeout, stops its other roles, frees its
 * tensor memory and returns, and the next st_plan_sync reports
 * ST_ERR_TIMEOUT.  Nothing faults, traps or hangs, and the plan stays usable.
 * what = 0 clears a pending injection.  ST_ERR_UNSUPPORTED for SIMT plans.
 */
st_status st_plan_inject(st_plan_t plan, int what, unsigned wait_ms);

#ifdef __cplusplus
}
#endif

#endif /* ST_STAGES_H */
