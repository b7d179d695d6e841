// Internal declarations shared by the CUDA translation units of the
// spherical-harmonic transform library.  Nothing here is part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "st.h"
#include "st_stages.h"

namespace st {

enum Prec { P_FP64 = 0, P_TF32X3 = 1, P_BF16X3 = 2, P_FP32 = 3 };

// Storage modes of a data operand written for the Legendre stage.
enum Store { S_F64 = 0, S_F32 = 1, S_TF32_SPLIT = 2, S_BF16_SPLIT = 3 };

inline int store_of(int prec)
{
    switch (prec) {
    case P_FP64: return S_F64;
    case P_TF32X3: return S_TF32_SPLIT;
    case P_BF16X3: return S_BF16_SPLIT;
    default: return S_F32;
    }
}
inline int store_bytes(int s) { return s == S_F64 ? 8 : (s == S_BF16_SPLIT ? 2 : 4); }
inline int store_planes(int s) { return (s == S_TF32_SPLIT || s == S_BF16_SPLIT) ? 2 : 1; }
inline bool prec_is_tc(int prec) { return prec == P_TF32X3 || prec == P_BF16X3; }

// Element (row r, column c) of plane 0 of a GEMM data operand stored in mode S.
// Split-TF32 operands are stored column-major (reduction index contiguous):
// the tensor cores read TF32 only from K-major shared-memory tiles.  All
// other modes are row-major with the data columns contiguous.
__host__ __device__ inline long long op_index(int S, long long r, int c, int Cp, long long Rp)
{
    return S == S_TF32_SPLIT ? (long long)c * Rp + r : r * (long long)Cp + c;
}
// Row counts are padded to a multiple of 4 so that a TF32 row coordinate of a
// tensor copy is always 16-byte aligned.
__host__ __device__ inline long long rows_padded(long long rows) { return (rows + 3) / 4 * 4; }

constexpr int MAX_RADICES = 24;

// One northern Gaussian row j (0 = nearest the pole) and its mirror row
// nlat-1-j; both have N points.
//  mode 0: the N-point DFT runs as Stockham passes over the radices of N.
//  mode 1: Bluestein: the N-point DFT is a chirp-weighted circular
//          convolution of length fftlen = L >= N + 2M (L 5-smooth), done with
//          two L-point Stockham FFTs and a precomputed kernel spectrum.
struct RowPair {
    int N;                    // points per row
    int M;                    // wavenumbers kept: 0..M
    int mode;                 // 0 direct mixed radix, 1 Bluestein
    int fftlen;               // length of the FFTs run: N (mode 0) or L (mode 1)
    int nrad;                 // number of radix stages of length fftlen
    int rad[MAX_RADICES];     // radix of each stage (decimation-in-frequency order)
    int swz;                  // shared-memory address map (see fft_swz)
    long long tw_off;         // first of the row's fftlen roots of unity e^{-2 pi i t / fftlen}
    long long chirp_off;      // mode 1: N chirp values w_k = e^{-i pi k^2 / N}
    long long kern_off;       // mode 1: L values FFT_L(b) / L, b the conjugate chirp over the row's
                              // offsets wrapped circularly (direct; the inverse's mirror image
                              // follows all rows' direct spectra)
    long long off_n;          // offset of the northern row inside one field's grid
    long long off_s;          // offset of the southern row
    int j;                    // row pair index (0 = nearest the north pole)
    int fast;                 // compile-time FP32 plan of length fftlen (ST_FF_PLANS id), -1: generic kernel
};

// FP32 FFT plans with compile-time radices (fft_fast.cuh): id, translation-
// unit group, radices R1 .. R4 (1 = unused), L = R1 R2 R3 R4.  Later radices
// are 16 wherever the length allows, which keeps every pass free of shared-
// memory bank conflicts under the pad-16 layout.
#define ST_FF_PLANS(X)                                                                                 \
    X(0, 0, 4, 4, 1, 1) X(1, 0, 5, 4, 1, 1) X(2, 0, 6, 4, 1, 1) X(3, 0, 2, 16, 1, 1)                      \
    X(4, 0, 10, 4, 1, 1) X(5, 0, 3, 16, 1, 1) X(6, 0, 4, 16, 1, 1) X(7, 0, 5, 16, 1, 1)                   \
    X(8, 0, 6, 16, 1, 1) X(9, 0, 8, 16, 1, 1) X(10, 0, 10, 16, 1, 1) X(11, 0, 12, 16, 1, 1)               \
    X(12, 0, 16, 16, 1, 1) X(13, 1, 2, 10, 16, 1) X(14, 1, 3, 8, 16, 1) X(15, 1, 2, 16, 16, 1)            \
    X(16, 1, 4, 10, 16, 1) X(17, 1, 3, 16, 16, 1) X(18, 1, 4, 16, 16, 1) X(19, 1, 5, 16, 16, 1)           \
    X(20, 1, 6, 16, 16, 1) X(21, 1, 8, 16, 16, 1) X(22, 1, 10, 16, 16, 1) X(23, 1, 12, 16, 16, 1)         \
    X(24, 1, 16, 16, 16, 1) X(25, 2, 2, 10, 16, 16) X(26, 2, 2, 12, 16, 16) X(27, 2, 2, 16, 16, 16)
constexpr int FF_NPLANS = 28;
constexpr int FF_NGROUPS = 3;
// shared-memory slot of one field for a plan of length L (pad-16 layout)
__host__ __device__ inline int ff_slot(int L) { return L + (L >> 4) + 1; }
// host lookups into ST_FF_PLANS
inline int ff_group(int id)
{
    switch (id) {
#define X(i, g, a, b, c, d) \
    case i: return g;
        ST_FF_PLANS(X)
#undef X
    }
    return -1;
}
inline int ff_radices(int id, int *rad)
{
    switch (id) {
#define X(i, g, a, b, c, d)                                                  \
    case i: {                                                                \
        const int r_[4] = {a, b, c, d};                                      \
        int n_ = 0;                                                          \
        for (int k_ = 0; k_ < 4; ++k_)                                       \
            if (r_[k_] > 1) rad[n_++] = r_[k_];                              \
        return n_;                                                           \
    }
        ST_FF_PLANS(X)
#undef X
    }
    return 0;
}
inline int ff_length(int id)
{
    int rad[4], L = 1;
    const int n = ff_radices(id, rad);
    for (int k = 0; k < n; ++k) L *= rad[k];
    return n ? L : 0;
}
// Shared memory of a fast-kernel CTA beyond its field slots (FP32 complex
// elements): the L / R1 base roots when there are at most 512 of them.
inline int ff_table_elems(int id)
{
    int rad[4];
    ff_radices(id, rad);
    const int twn = ff_length(id) / rad[0];
    return twn <= 512 ? twn : 0;
}

// One Legendre GEMM: zonal wavenumber m, parity p (n - m even: 0, odd: 1),
// in one direction.  out[col][c] = sum_r tab[col][r] * data[r][c].
//   inverse: col = northern row j (ncol = J), r = k with n = m + p + 2k
//   direct:  col = k (ncol = K_m^p), r = northern row j (K = J)
// Place of frequency m after in-place decimation-in-frequency passes over
// the radices rad[0..nrad) of L: m = d1 + R1 (d2 + R2 (...)), place =
// sum_s d_s L / (R1 ... Rs) (the mixed-radix digit reversal).
__host__ __device__ inline int dif_pos(int m, const RowPair &rp)
{
    int pos = 0, stride = rp.fftlen;
    for (int q = 0; q < rp.nrad; ++q) {
        const int R = rp.rad[q];
        const int d = m % R;
        m /= R;
        stride /= R;
        pos += d * stride;
    }
    return pos;
}

// Shared-memory address of FFT element i for a row's address map: 0 plain,
// 1 one pad slot per 16, 2 one pad slot per 32, 3 XOR of bits 4-7 into bits
// 0-3.  The plan picks, per row, the map with the fewest bank conflicts over
// that row's passes.
__host__ __device__ inline int fft_swz(int i, int mode)
{
    switch (mode) {
    case 1: return i + (i >> 4);
    case 2: return i + (i >> 5);
    case 3: return i ^ ((i >> 4) & 15);
    default: return i;
    }
}
__host__ __device__ inline int fft_swz_size(int L, int mode)
{
    // mode 3 permutes within aligned blocks of 16, so a partial last block
    // reaches up to the next multiple of 16
    if (mode == 3) return (L + 15) & ~15;
    return mode == 1 ? L + (L >> 4) + 1 : (mode == 2 ? L + (L >> 5) + 1 : L);
}

// Legendre table sets.  H_n^m = (1 - mu^2) dPbar_n^m/dmu has the opposite
// parity in mu to Pbar_n^m, so the H sets exchange the Fourier-buffer halves:
// synthesis group (m, p) writes the half 1 - p, analysis group (m, p) reads it.
enum TableSet {
    SET_SYN = 0,      // Pbar_n^m(mu_j)                        synthesis
    SET_ANA = 1,      // w_j Pbar_n^m(mu_j)                    analysis
    SET_SYN_H = 2,    // H_n^m(mu_j)                           synthesis, halves exchanged
    SET_ANA_P1 = 3,   // w_j / (1 - mu_j^2) Pbar_n^m(mu_j)     analysis
    SET_ANA_H1 = 4,   // w_j / (1 - mu_j^2) H_n^m(mu_j)        analysis, halves exchanged
    NSETS = 5
};
inline int set_dir(int set) { return (set == SET_SYN || set == SET_SYN_H) ? 0 : 1; }

struct LegGroup {
    int m, p;
    int ncol;                 // valid columns of the table
    int K;                    // valid reduction length
    int r0;                   // first reduction index worth visiting (row trimming)
    int nt;                   // column-tile width (tensor-core layout)
    int nct;                  // number of column tiles
    int nkc;                  // number of reduction chunks in the stored table
    long long data_row0;      // data-operand row holding reduction index 0
    long long out_row0;       // output row holding column 0
    long long tab_off;        // table offset: elements (SIMT) or bytes (tensor-core images)
};

struct LegTile {
    int g;                    // group index (2 m + p)
    int ct;                   // column tile
};

// ---- batched launches: every kernel takes up to MAX_JOBS per-request jobs in
// its launch parameters; a CTA (or a persistent tile) finds its job by binary
// search over the jobs' prefix sums.  A single-plan call is a batch of one.
constexpr int MAX_JOBS = 64;

template <int MAXJ>
__device__ inline int find_job(const long long *prefix, int njobs, long long b)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One FFT stage of one request over a run of rows that share a launch shape.
struct FftJob {
    const RowPair *rps;
    const void *tw, *chirp, *kern;
    const void *src;          // direct: grid; inverse: Fourier buffer (S, A)
    void *dst;                // direct: Fourier-buffer operand (E, O); inverse: grid
    long long npts, Rp, ps;
    int nfields, G, Sslot, Cp, T, Jp, nfg;
    int r0, J;                // entries r0 .. r0 + J - 1 of the plan's row-pair array
    int kind;                 // -1: generic kernel; else the fast kernel group of `plan`
    int plan;                 // fast plan id (ST_FF_PLANS)
    int smode;                // storage mode of the direct output (fast kernels)
    int smem;                 // dynamic shared memory one CTA of this job needs (bytes)
    int a_top;                // inverse: the odd half at m = T holds data (derivative syntheses);
                              // otherwise no GEMM writes it (no n = T + 1) and it reads as zero
    int *err;                 // the plan's device error word (bounded waits set bit 8 on expiry)
};
template <int MAXJ>
struct FftBatch {
    int njobs;
    long long prefix[MAXJ + 1];  // CTAs of job q: [prefix[q], prefix[q+1])
    FftJob job[MAXJ];
};

// Spectral pack (inverse) or unpack (direct) of one request.
struct PackJob {
    const void *src;
    void *dst;
    const long long *srow;
    long long nspec, Rp, ps;
    int T, max_m, nfields, Cp, nft, nm;  // nft field tiles of 32, nm wavenumbers launched
    int scale;                           // pack: 1 multiplies a_n^m by -1 / (n (n+1)) (0 at n = 0)
};
template <int MAXJ>
struct PackBatch {
    int njobs;
    long long prefix[MAXJ + 1];
    PackJob job[MAXJ];
};

// SIMT Legendre stage of one request.
struct SimtJob {
    const LegGroup *groups;
    const LegTile *tiles;
    const void *tab, *data;
    void *out;
    int ncm, C, Cp;
};
template <int MAXJ>
struct SimtBatch {
    int njobs;
    long long prefix[MAXJ + 1];
    SimtJob job[MAXJ];
};

}  // namespace st

// The plan object behind st_plan_t.
struct st_plan {
    int T = 0, nlat = 0, J = 0, Jp = 0, kind = 0, nlon = 0, prec = 0, max_fields = 0;
    int max_m = 0;
    int device = 0, sm_count = 0;
    std::vector<int> rows;     // nlat row lengths
    std::vector<int> Mrow;     // J kept wavenumbers of each northern row
    std::vector<int> j0;       // T+1: first northern row with M_j >= m (J if none)
    long long npts = 0;        // grid points per field
    long long nspec = 0;       // complex coefficients per field
    // first row of each (m, parity) group in the packed spectral operand
    // (index 2 m + p); 4-aligned for split TF32, compact otherwise
    std::vector<long long> srow_h;
    long long *srow = nullptr;
    long long srow_total = 0;  // rows of the packed spectral operand (padded to 4)

    double *mu = nullptr, *w = nullptr;  // device FP64 nodes and weights (nlat)

    // FFT data
    st::RowPair *rowpairs = nullptr;     // device, J entries
    std::vector<st::RowPair> rowpairs_h;  // by row index j
    std::vector<int> row_order;           // device array entry r holds row row_order[r]
                                          // (longest padded FFT first)
    void *tw = nullptr;                  // device roots of unity (double2 or float2)
    long long ntw = 0;
    void *chirp = nullptr;               // Bluestein chirps (double2 or float2)
    void *kern = nullptr;                // Bluestein kernel spectra (double2 or float2)
    long long nchirp = 0, nkern = 0;
    int max_row = 0;                     // largest N
    int max_fft = 0;                     // largest fftlen
    int max_fft_smem = 0;                // largest shared-memory slot (fftlen after padding)
    int max_chirp = 0;                   // largest N among Bluestein rows
    int nfast = 0;                       // rows on the fast kernels: entries 0 .. nfast-1 of rowpairs

    // Legendre table sets (see st::TableSet): [0] Pbar synthesis, [1] w Pbar
    // analysis, and, once derivatives are enabled, [2] H synthesis, [3] and
    // [4] the analysis sets of the wind transforms.  Work lists exist per
    // direction ([0] synthesis, [1] analysis): a set has its direction's tiles.
    void *tab[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t tab_bytes[5] = {0, 0, 0, 0, 0};
    st::LegGroup *groups[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<st::LegGroup> groups_h[5];
    st::LegTile *tiles[2] = {nullptr, nullptr};
    int ntiles[2] = {0, 0};
    // derivative support (st_plan_enable_derivatives): sets 2-4 and a second
    // Fourier buffer and spectral output, owned by this plan
    bool deriv = false;
    void *fb2 = nullptr, *sout2 = nullptr;

    // workspace.  GEMM data operands live in buffers of their own that only
    // ever hold zeros (from creation) or finite values written in their own
    // storage mode: a tile may read rows beyond its group, which meet zero
    // table entries, and those rows must never decode as Inf or NaN.
    void *fb = nullptr;       // inverse Legendre output: 2 (T+1) Jp rows x Cp columns, FP32/FP64
    void *fbop = nullptr;     // direct Legendre operand: same rows, in the precision's storage mode
    size_t fb_bytes = 0, fbop_bytes = 0;
    void *sop = nullptr;      // inverse Legendre operand (packed spectra): srow_total rows x Cp, storage mode
    void *sout = nullptr;     // direct Legendre output: srow_total rows x Cp, FP32/FP64
    size_t sop_bytes = 0, sout_bytes = 0;
    int *err = nullptr;       // device error word (bit flags set by bounded waits)

    size_t device_bytes = 0, table_bytes = 0, workspace_bytes = 0;

    // Read-only device data (nodes, FFT rows, tables, groups, tiles, row
    // bases) may be shared by several plans (st_plan_create_shared); it is
    // freed when the last plan holding it is destroyed.
    std::shared_ptr<void> core;

    // launch shapes (autotuned; see st_plan_autotune), per direction [0] inverse [1] direct
    int fft_var[2] = {0, 0};       // FFT launch variant (threads per CTA, CTAs per SM)
    int fft_kb[2] = {100, 100};    // FFT shared-memory budget per CTA (KB): fields per CTA
    int nt_inv = 0;                // inverse Legendre column-tile width (0: automatic)
    int nt_inv_hi = 0;             // the same for m >= (max_m + 1) / 2 (0: as nt_inv)

    // fault injection (tests): the next tensor-core Legendre launch withholds
    // its operand copies and bounds its waits by inject_wait_ns
    int inject_withhold = 0;
    unsigned long long inject_wait_ns = 0;

    // launch accounting and optional event timing, per kernel kind
    bool timing = false;
    long long launches[16] = {0};
    long long timed[16] = {0};
    double total_ms[16] = {0};
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
};

namespace st {

// ---- error plumbing (host) ----
void set_last_error(const std::string &s);
st_status cuda_fail(cudaError_t e, const char *what);
#define ST_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return st::cuda_fail(e_, #call);    \
    } while (0)

// Fourier buffer rows: (p, m, j) -> (p (T+1) + m) Jp + j, Jp = J rounded up to 4
inline long long fb_rows(const st_plan *p) { return 2LL * (p->T + 1) * p->Jp; }
inline long long fb_row(const st_plan *p, int par, int m, int j) { return ((long long)par * (p->T + 1) + m) * p->Jp + j; }
// Row pitch (columns) of the packed operands and the Fourier buffer for
// 2 nfields data columns: a multiple of 8 (16-byte rows in the bf16 planes),
// and from 256 columns on a multiple of 64, so that every row of every plane
// starts on a 128-byte line.  Rows that start inside a 32-byte sector leave
// partly written sectors behind the GEMM epilogue and the pack stores: at
// T639 O640, 548 fields (1096 columns) ran the Legendre kernels 7-9 % slower
// than 544 fields (1088 = 17 x 64).  No kernel reads or writes the padding
// columns; the pitch grows with nfields, so a workspace sized for max_fields
// holds every smaller call.
inline int cols_padded(int nfields)
{
    const int C = 2 * nfields;
    return C < 256 ? ((C + 7) / 8) * 8 : ((C + 63) / 64) * 64;
}

// Tensor-core Legendre kernel geometry: 128 data columns per tile; a reduction
// chunk is 128 bytes of the K-major table row (64 bf16 or 32 tf32 values).
constexpr int TC_M = 128;
inline int tc_kc(int prec) { return prec == P_BF16X3 ? 64 : 32; }
constexpr int SIMT_TILE = 64;

// Kernel kinds for launch accounting.
enum KernelKind {
    K_PACK = 0, K_LEG_INV, K_FFT_INV, K_FFT_DIR, K_LEG_DIR, K_UNPACK, K_EXPORT, K_TABLES, K_COMBINE, K_NKINDS
};
const char *kernel_name(const st_plan *p, int kind);

// ---- job builders and batched launchers ----
st_status fft_jobs(st_plan *p, int dir, int nfields, const void *src, void *dst, std::vector<FftJob> &jobs,
                   size_t *smem, int kb = 0);
st_status fft_dir_jobs(st_plan *p, int nfields, const void *grid, std::vector<FftJob> &jobs, size_t *smem,
                       int kb = 0);
st_status launch_fb_tf32split(st_plan *p, int nfields, cudaStream_t s);
st_status launch_fft_jobs(int dir, int prec, const FftJob *jobs, int n, size_t smem, cudaStream_t s,
                          int variant = 0);
// fast-kernel launch of n jobs of one group (all jobs' kind == group), one direction
st_status launch_fftf(int dir, int group, const FftJob *jobs, int n, cudaStream_t s, int variant = 0);
st_status launch_fftf_dirw_g0(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_dirw_g1(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_dirw_g2(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_invw_g0(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_invw_g1(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_invw_g2(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_dir_g0(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_dir_g1(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_dir_g2(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_inv_g0(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_inv_g1(const FftJob *jobs, int n, cudaStream_t s);
st_status launch_fftf_inv_g2(const FftJob *jobs, int n, cudaStream_t s);
// scale: 0 none, 1 the inverse Laplacian -1 / (n (n+1)) (0 at n = 0);
// cp: column stride of the operand (0: the one of nfields)
st_status pack_job(st_plan *p, int dir, int nfields, const void *src, void *dst, PackJob *job, int scale = 0,
                   int cp = 0);
st_status launch_pack_jobs(int dir, int prec, const PackJob *jobs, int n, cudaStream_t s);
st_status simt_job(st_plan *p, int set, int nfields, const void *data, void *out, SimtJob *job, long long *blocks,
                   int cp = 0);
st_status launch_simt_jobs(int prec, const SimtJob *jobs, const long long *blocks, int n, cudaStream_t s);
// Tensor-core Legendre stage of one request (the data operand's tensor map
// travels with it).
struct TcJob {
    CUtensorMap map;
    const LegGroup *groups;
    const LegTile *tiles;
    const char *tab;
    float *out;
    int *err;
    long long ntiles;         // tiles[] entries x data tiles
    int ncm, C, Cp, max_nt;
};
st_status tc_job(st_plan *p, int set, int nfields, void *data, void *out, TcJob *job, int cp = 0);
st_status launch_tc_jobs(int prec, const TcJob *jobs, int n, int sm_count, cudaStream_t s, int withhold = 0,
                         unsigned long long wait_ns = 2000000000ull);

// ---- persistent batch kernel (batch_persistent.cu) ----
// Shared memory of each half of its CTA in the row-FFT stages.
constexpr int FF_HALF_BYTES = 110 * 1024;
// The stage jobs of one precision group of a batch; fft jobs built within
// FF_HALF_BYTES of shared memory a CTA.
struct PersInput {
    int prec = 0;
    int sm_count = 0;
    int *err = nullptr;  // error word the grid barriers report into
    std::vector<PackJob> pack, unpack;
    std::vector<TcJob> tc_inv, tc_dir;
    std::vector<FftJob> fft_inv, fft_dir;
};
struct PersState;
st_status pers_prepare(const PersInput &in, PersState **out);
st_status pers_launch(PersState *ps, cudaStream_t s);
void pers_free(PersState *ps);
size_t tc_smem_bytes(int prec, int max_nt, int *stages_out, size_t cap = 0);

// ---- kernel launch count of the calling thread (api.cu): every launcher of
// a transform kernel adds its launches, so that a plan's per-kind counters
// report kernels, not calls.
int &kernel_launches();

// ---- plan helpers (api.cu) ----
st_status count_launch(st_plan *p, int kind, cudaStream_t s, const std::function<st_status()> &f);
st_status plan_alloc(st_plan *p, void **ptr, size_t bytes);
void build_groups_deriv(st_plan *p, int set);

// ---- on-disk table cache (cache.cu) ----
std::string table_cache_path(const st_plan *p, const char *dir);
st_status save_tables(st_plan *p, const char *path);
st_status load_tables(st_plan *p, const char *path);

// ---- autotuner support (api.cu) ----
st_status rebuild_legendre(st_plan *p, cudaStream_t s);
std::string tune_key(const st_plan *p, int nfields);

// ---- launchers implemented in the .cu files ----
st_status launch_tables(st_plan *p, cudaStream_t s);
st_status launch_twiddles(st_plan *p, cudaStream_t s);
st_status launch_bluestein_setup(st_plan *p, cudaStream_t s);
st_status launch_fft_dir(st_plan *p, const void *grid, int nfields, cudaStream_t s);
// The optional buffer arguments below replace the plan's own workspace
// buffers for one call (nullptr: use the plan's).
st_status launch_fft_inv(st_plan *p, void *grid, int nfields, cudaStream_t s, const void *fb = nullptr,
                         int a_top = 0);
st_status launch_pack(st_plan *p, const void *spec, int nfields, cudaStream_t s, void *sop = nullptr);
st_status launch_unpack(st_plan *p, void *spec, int nfields, cudaStream_t s);
st_status launch_leg_simt(st_plan *p, int dir, int nfields, cudaStream_t s, void *data = nullptr,
                          void *out = nullptr);
st_status launch_leg_tc(st_plan *p, int dir, int nfields, cudaStream_t s, void *data = nullptr, void *out = nullptr);
// Legendre stage of table set `set` (SIMT or tensor cores by precision), data
// and out explicit; cp as for the job builders
st_status launch_leg_set(st_plan *p, int set, int nfields, cudaStream_t s, void *data, void *out, int cp = 0);
st_status launch_tables_deriv(st_plan *p, cudaStream_t s);
// Fourier-space combination of the P and H syntheses (mode 0: winds from psi,
// chi; mode 1: d/dlambda and (1 - mu^2) d/dmu of a scalar), in place in fb
st_status launch_deriv_combine(st_plan *p, int mode, int nfields, void *fb, const void *fb2, cudaStream_t s);
// spectral combination of the P and H analyses into vorticity and divergence,
// in place in sout
st_status launch_vordiv_combine(st_plan *p, int nfields, void *sout, const void *sout2, cudaStream_t s);
st_status launch_fourier_export(st_plan *p, int dir, int nfields, double *out, cudaStream_t s);
st_status launch_gauss(int nlat, double *mu, double *w, cudaStream_t s);
st_status launch_legendre_values(int T, const double *mu, int nmu, double *out, cudaStream_t s);

}  // namespace st
