/*
 * st.h -- C ABI of the GB300 spherical-harmonic spectral transform.
 *
 * The transform is the one stated in ESCAPE D3.3 (arXiv 1908.06096),
 * section 4.4.1 (and again in 4.4.2): the synthesis
 *
 *     f(theta, lambda) = sum_{m=-T}^{T} e^{i m lambda}
 *                          sum_{n=|m|}^{T} a_n^m Pbar_n^m(cos theta)
 *
 * ("inverse", spectral -> grid) and its inverse ("direct", grid -> spectral),
 * where each coefficient is the projection of the field on one basis
 * function (section 4.4.2), evaluated with Gaussian quadrature in latitude.
 * Both run as the two stages of section 4.4.1's figure: FFTs along each
 * latitude row and a Legendre transform along latitude, which section 4.2.4
 * carries out as matrix multiplications, one per zonal wavenumber m.
 *
 * Conventions (the paper leaves these open; the readings are fixed here):
 *  - theta is colatitude; mu = cos(theta).  Gaussian latitudes run north to
 *    south.  Pbar_n^m is normalised to unit L2 norm on [-1, 1], without the
 *    Condon-Shortley phase.  Truncation is triangular at T.
 *  - Spectral array, per field: m-major triangular, complex interleaved
 *    (re, im); coefficient (m, n), 0 <= m <= n <= T, sits at complex index
 *    m (T+1) - m (m-1)/2 + (n - m).  Fields are stored one after another.
 *    Only m >= 0 is stored (a_n^{-m} = conj(a_n^m)); Im a_n^0 is ignored on
 *    input and written as 0 on output.
 *  - Grid array, per field: rows north to south, concatenated; row j holds
 *    N_j points at longitudes 2 pi k / N_j.  Fields one after another.
 *  - A row keeps wavenumbers m <= M_j = min(T, floor((N_j - 1) / 2)).
 *  - Element type: double for ST_FP64 plans, float for every other
 *    precision.  All pointers passed to the transforms are DEVICE pointers
 *    unless a name says _host.
 *
 * Ownership: the caller owns every input and output buffer.  A plan owns its
 * Gaussian nodes, Legendre tables, FFT row data and workspace; all are freed
 * by st_plan_destroy.
 *
 * Asynchrony: st_inv_trans / st_dir_trans enqueue work on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and return without waiting.
 * Argument and launch errors are returned at once.  A device-side error (a
 * bounded wait that gave up inside a kernel) is recorded in the plan and
 * returned by the next st_plan_sync.
 *
 * Concurrency: one plan runs one transform at a time (its workspace is
 * shared by both directions).  Calls on one plan must be ordered on one
 * stream; use one plan per stream for concurrent transforms.
 */
#ifndef ST_H
#define ST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct st_plan *st_plan_t;

typedef enum {
    ST_OK = 0,
    ST_ERR_ARG = 1,         /* invalid argument (null pointer, bad size, nfields > max) */
    ST_ERR_OOM = 2,         /* device allocation failed */
    ST_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    ST_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    ST_ERR_UNSUPPORTED = 5, /* valid request this build or device cannot serve */
    ST_ERR_BUSY = 6         /* resource already in use */
} st_status;

typedef enum { ST_GRID_REGULAR = 0, ST_GRID_OCTAHEDRAL = 1 } st_grid_kind;

typedef enum {
    ST_FP64 = 0,      /* FP64 everywhere (SIMT Legendre GEMM, FP64 FFT) */
    ST_FP32_TC = 1,   /* Legendre on tensor cores as 3 x TF32 (hi/lo split), FP32 accumulate */
    ST_BF16X3 = 2,    /* Legendre on tensor cores as 3 x BF16 (hi/lo split), FP32 accumulate */
    ST_FP32_SIMT = 3  /* FP32 SIMT Legendre GEMM, FP32 FFT */
} st_precision;

typedef struct {
    int kind;  /* st_grid_kind */
    int nlat;  /* number of Gaussian latitudes (even, >= 2) */
    int nlon;  /* points per row for ST_GRID_REGULAR; ignored for octahedral grids,
                  whose row i from either pole (i = 1 .. nlat/2) has 20 + 4 i points */
} st_grid_desc;

typedef struct {
    int T, nlat, kind, precision, max_fields;
    int max_m;                /* largest m kept by any row (min(T, max_j M_j)) */
    size_t spec_elems;        /* complex coefficients per field: (T+1)(T+2)/2 */
    size_t grid_points;       /* grid points per field: sum_j N_j */
    size_t element_bytes;     /* 8 for ST_FP64, else 4 */
    size_t device_bytes;      /* device memory held by the plan */
    size_t table_bytes;       /* of which Legendre tables */
    size_t workspace_bytes;   /* of which workspace */
    int launch_shape[6];      /* inverse FFT variant, its smem budget (KB), direct FFT variant, its
                                 budget (KB), inverse Legendre column-tile width (0: automatic), the
                                 same for the upper half of the wavenumbers (0: as the former) */
} st_plan_info;

/*
 * Create a plan for truncation T on `grid` (section 4.4.1 statement of the
 * transform; grid geometry per st_grid_desc).  Builds, on the device and in
 * FP64, the Gaussian nodes and weights (Newton iteration on P_nlat) and the
 * normalised associated Legendre tables (three-term recurrence), then
 * converts them to the layout and precision `prec` needs.  Allocates the
 * workspace for up to `max_fields` fields per call.  Work runs on `stream`;
 * the call returns once the plan is ready (it synchronises the stream).
 * Errors: ST_ERR_ARG for T < 1, odd or too small nlat, nlon < 1 on a regular
 * grid, unknown kind or precision, max_fields < 1; ST_ERR_OOM; ST_ERR_CUDA;
 * ST_ERR_UNSUPPORTED if the device is not sm_103 for a tensor-core precision.
 * On error *out is set to NULL.
 */
st_status st_plan_create(st_plan_t *out, int T, const st_grid_desc *grid, int prec,
                         int max_fields, void *stream);

/*
 * A second plan with the same transform as `base` that shares base's
 * read-only device data (Gaussian nodes, Legendre tables, FFT row data) and
 * owns only a new workspace for up to max_fields fields.  Plans sharing data
 * can run concurrently on different streams (each has its own workspace);
 * the shared data is freed with the last plan that holds it, in any order.
 * Not in the paper: it lets a server keep one set of tables per truncation
 * resident while several requests of that truncation are in flight.
 */
st_status st_plan_create_shared(st_plan_t *out, st_plan_t base, int max_fields, void *stream);

/*
 * Autotuner (not in the paper).  Times, on this plan and for `nfields`
 * fields, candidate FFT launch shapes (fields per CTA, through the per-CTA
 * shared-memory budget) for each direction and, on tensor-core plans,
 * candidate column-tile widths of the inverse per-m Legendre GEMMs (re-laying
 * out the tables), first for all m, then for the upper half of the
 * wavenumbers on its own, and keeps the fastest.  Synchronous; allocates a temporary grid buffer.  If cache_path is
 * not NULL the choice is appended to that text file; st_plan_create applies a
 * matching entry (same T, grid, precision, field-count bucket and SM count)
 * from the file named by the ST_TUNE_CACHE environment variable.
 * ST_ERR_BUSY if the plan shares its tables with another plan.
 */
st_status st_plan_autotune(st_plan_t plan, int nfields, const char *cache_path, void *stream);

/* Release everything the plan holds.  NULL is accepted.  The caller must make
 * sure no work on the plan is still in flight. */
st_status st_plan_destroy(st_plan_t plan);

/* Plan facts (sizes, precision, memory). */
st_status st_plan_query(st_plan_t plan, st_plan_info *info);

/* Copy the row lengths N_j (nlat ints, north to south) to host memory. */
st_status st_plan_row_lengths(st_plan_t plan, int *rows_host);

/* Copy the device-computed Gaussian nodes mu_j and weights w_j (FP64,
 * north to south, nlat each) to host memory (synchronous). */
st_status st_plan_nodes(st_plan_t plan, double *mu_host, double *w_host);

/*
 * Inverse transform, spectral -> grid (the synthesis equation of section
 * 4.4.1): spec_dev holds nfields spectral arrays, grid_dev receives nfields
 * grid arrays (layouts above).  1 <= nfields <= max_fields, else ST_ERR_ARG.
 * Stages: per-m Legendre GEMMs (section 4.2.4) producing the symmetric and
 * antisymmetric Fourier coefficients, then per-row inverse real FFTs
 * (section 4.2.5).  Asynchronous on `stream`.
 */
st_status st_inv_trans(st_plan_t plan, const void *spec_dev, void *grid_dev, int nfields,
                       void *stream);

/*
 * Direct transform, grid -> spectral (each coefficient the quadrature of the
 * field against one basis function, section 4.4.2): per-row real FFTs scaled
 * by 1/N_j, then per-m Legendre GEMMs against w_j Pbar_n^m(mu_j).
 * Asynchronous on `stream`.  Same argument rules as st_inv_trans.
 */
st_status st_dir_trans(st_plan_t plan, const void *grid_dev, void *spec_dev, int nfields,
                       void *stream);

/*
 * Inverse transform exactly like st_inv_trans, but its scratch (the packed
 * spectral operand and the Fourier buffer) lives in one fixed array compiled
 * into the library (st_static_scratch_bytes() bytes, 32 MiB) instead of the
 * plan's workspace.  The paper has no counterpart: it is for callers that
 * cannot allocate device memory where they run the transform -- real-time
 * loops where an allocation may stall, frameworks that own all device memory
 * through their own allocator -- and it calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *  - Returns ST_ERR_ARG (message in st_last_error) when the plan and
 *    `nfields` need more scratch than the array holds; nfields may exceed the
 *    plan's max_fields as long as the scratch suffices.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    life of the process; make that first call before any stream capture,
 *    and do not call the entry point on a device after cudaDeviceReset.
 *  - Every call on a device shares the one array and it keeps the last
 *    call's contents; the call clears what must start at zero itself.  Calls
 *    that can overlap on the GPU (other streams, or the same array used from
 *    several host threads without ordering) race on it and give wrong results.
 *  - Every GPU that loads the library holds the array until the process exits.
 *  - Its launches are counted and timed with the plan's (st_plan_timings).
 */
st_status st_inv_trans_static(st_plan_t plan, const void *spec_dev, void *grid_dev, int nfields,
                              void *stream);

/*
 * Derivative and wind transforms, the other transforms of the SH dwarf's time
 * step (ESCAPE D3.3 sections 4.2.2-4.2.3 name them; the formulas are the
 * standard ones, stated here).  Unit sphere, phi the latitude, mu = sin(phi),
 * H_n^m = (1 - mu^2) dPbar_n^m/dmu; wind images U = u cos(phi), V = v cos(phi);
 * stream function psi = -zeta / (n (n+1)) and velocity potential
 * chi = -D / (n (n+1)) from vorticity zeta and divergence D (0 for n = 0).
 *
 * st_plan_enable_derivatives builds, once per plan and in FP64 on the device,
 * three more Legendre table sets in the plan's precision (H for synthesis,
 * w_j Pbar / (1 - mu_j^2) and w_j H / (1 - mu_j^2) for analysis) and a second
 * Fourier buffer and spectral output.  Synchronous; ST_ERR_OOM if they do not
 * fit.  The calls below need it, and need 2 nfields <= max_fields (they run
 * the FFT and Legendre stages on 2 nfields column pairs); ST_ERR_ARG otherwise.
 * Same layouts, element type and asynchrony as st_inv_trans / st_dir_trans.
 */
st_status st_plan_enable_derivatives(st_plan_t plan, void *stream);

/* out_dev [2 nfields][grid]: fields 0 .. nfields-1 are dF/dlambda, fields
 * nfields .. 2 nfields-1 are (1 - mu^2) dF/dmu = cos(phi) dF/dphi of the
 * nfields spectra in spec_dev. */
st_status st_inv_trans_deriv(st_plan_t plan, const void *spec_dev, void *out_dev, int nfields, void *stream);

/* vordiv_dev [2 nfields][spectra]: vorticity fields, then divergence fields;
 * uv_dev [2 nfields][grid] receives U fields, then V fields:
 *   U = dchi/dlambda - (1 - mu^2) dpsi/dmu,  V = dpsi/dlambda + (1 - mu^2) dchi/dmu. */
st_status st_inv_trans_uv(st_plan_t plan, const void *vordiv_dev, void *uv_dev, int nfields, void *stream);

/* The reverse: uv_dev [2 nfields][grid] (U fields, then V fields) ->
 * vordiv_dev [2 nfields][spectra] (vorticity, then divergence), by Gaussian
 * quadrature with the mu-derivative moved onto Pbar by parts:
 *   zeta_n^m = sum_j w_j / (1 - mu_j^2) (i m V_m Pbar_n^m + U_m H_n^m),
 *   D_n^m    = sum_j w_j / (1 - mu_j^2) (i m U_m Pbar_n^m - V_m H_n^m),
 * U_m, V_m the rows' Fourier coefficients (1/N_j sum_k e^{-i m lambda_k}). */
st_status st_dir_trans_vordiv(st_plan_t plan, const void *uv_dev, void *vordiv_dev, int nfields, void *stream);

/*
 * On-disk table cache (not in the paper; the restart analogue of the SH
 * dwarf's once-per-run set-up).  st_plan_save_tables writes the plan's
 * Gaussian nodes and weights and both Legendre table sets, exactly as they
 * sit on the device, to `path`, with a header naming the truncation, grid,
 * precision and table layout and a checksum of the contents.
 * st_plan_load_tables reads such a file into a plan created with the same
 * truncation, grid, precision and layout: ST_ERR_ARG (message in
 * st_last_error) if the header does not match or the checksum fails -- the
 * plan's tables are then untouched -- and ST_ERR_BUSY if the plan shares its
 * tables with another plan.  Both are synchronous.  When the environment
 * variable ST_TABLE_CACHE names a directory, st_plan_create loads a plan's
 * tables from a matching file there instead of building them, and writes
 * one after building them.
 */
st_status st_plan_save_tables(st_plan_t plan, const char *path);
st_status st_plan_load_tables(st_plan_t plan, const char *path);

/* Size in bytes of the array st_inv_trans_static uses. */
size_t st_static_scratch_bytes(void);

/* Wait for the plan's work on `stream` and report any device-side error
 * recorded since the last call (then clear it). */
st_status st_plan_sync(st_plan_t plan, void *stream);

/*
 * Batched transforms of many plans at once (ESCAPE D3.3 sections 4.2.3-4.2.5:
 * fewer, larger kernels instead of many small library calls; here across
 * requests of different truncations and grids as well as across m and rows).
 * A batch is built once from a list of items; st_batch_run then issues one
 * launch per stage for all items (spectral pack, Legendre, FFT, and the same
 * for the direct direction), optionally recorded once into a CUDA graph and
 * replayed on later runs.
 *  direction 0: inverse, spec_in -> grid
 *  direction 1: direct, grid -> spec_out
 *  direction 2: round trip, spec_in -> grid -> spec_out
 * Every pointer is a device pointer the caller owns and keeps alive while
 * the batch exists.  A plan may appear in at most one item of a batch
 * (ST_ERR_BUSY otherwise); nfields must lie in [1, the plan's max_fields].
 * Items are grouped by precision; at most 64 items of one precision run in
 * one launch (larger groups take several).
 */
typedef struct st_batch *st_batch_t;

typedef struct {
    st_plan_t plan;
    int direction;
    const void *spec_in;
    void *grid;
    void *spec_out;
    int nfields;
} st_batch_item;

st_status st_batch_create(st_batch_t *out, const st_batch_item *items, int n);
/* use_graph 0: one launch per stage.  1: the first run records those
 * launches into a CUDA graph on `stream` and every run replays it (the
 * stream must not be capturing).  2: the whole batch as one persistent
 * cooperative launch, one CTA per SM looping over every request's work of
 * each stage in turn, with bounded grid-wide barriers between the stages (a
 * barrier that gives up sets bit 16 in the error word of the first item's
 * plan, reported by st_plan_sync as ST_ERR_TIMEOUT).  Mode 2 takes BF16x3
 * batches of at most 64 items a direction whose rows all have compile-time
 * FFT plans of length up to 4096 (truncations up to T639 on octahedral
 * grids); any other batch returns
 * ST_ERR_UNSUPPORTED with the reason in st_last_error.  Modes 0 and 1 give
 * the same results bit for bit; mode 2 agrees with them to within the last
 * bits (its row-FFT bodies are separately compiled instances of the same
 * code). */
st_status st_batch_run(st_batch_t batch, void *stream, int use_graph);
st_status st_batch_destroy(st_batch_t batch);

/*
 * Per-kernel timing (not in the paper; a measurement aid).  While enabled,
 * every kernel the plan launches is bracketed by two CUDA events recorded on
 * its launch stream; st_plan_timings waits for them and reports, per kernel,
 * the number of kernel launches and the summed event time since the last reset.
 * Do not enable timing while capturing the plan's calls into a CUDA graph.
 * Launch counts are kept whether or not timing is enabled.
 */
typedef struct {
    const char *name;   /* kernel name (static storage) */
    long long launches; /* launches since the last reset */
    double total_ms;    /* summed event time of the timed launches */
    long long timed;    /* launches that were timed */
} st_kernel_time;

st_status st_plan_set_timing(st_plan_t plan, int enable);
/* Fill up to `max` entries (one per kernel kind); *n receives the count.
 * Synchronises on the recorded events. */
st_status st_plan_timings(st_plan_t plan, st_kernel_time *out, int max, int *n);
st_status st_plan_reset_timings(st_plan_t plan);

/*
 * Deployment check (not in the paper): the compute capability of the current
 * device and the architecture the library's kernels were compiled for, as
 * the CUDA runtime reports it for a kernel of this library
 * (cudaFuncAttributes::binaryVersion: 103 for sm_103a code).  Any pointer
 * may be NULL.  ST_ERR_CUDA when there is no usable device or the kernels
 * cannot run on it.
 */
st_status st_build_info(int *cc_major, int *cc_minor, int *binary_version);

/* Text for a status code (static storage). */
const char *st_status_string(st_status s);

/* Last CUDA error text seen by the library on this thread ("" if none). */
const char *st_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ST_H */
