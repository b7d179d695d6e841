// Legendre stage on the 5th-generation tensor cores (tcgen05, accumulators in
// tensor memory), split precision.
//
// ESCAPE D3.3 section 4.2.4 runs the Legendre transform as one matrix product
// per zonal wavenumber m and pads them to one size for a uniform batched
// call.  Here every (m, parity) product of a direction is a group of one
// persistent grouped GEMM with no padding beyond the 16-column granularity of
// the instruction:
//
//     D[c][col] = sum_r data[r][c] * tab[col][r]
//
// with A = data (M = 128 data columns c = 2 field + re/im, MN-major, loaded by
// TMA tensor copies with 128-byte swizzle) and B = Legendre table (N = the
// group's column tile, up to 256; K-major; stored at plan time as ready-made
// swizzled shared-memory images and fetched with one bulk copy per stage).
// The transposes of section 4.2.6.3 vanish into this orientation: D^T is
// written straight out, one TMEM lane per data column, so each warp store is
// 128 contiguous bytes.
//
// Split precision: x = hi + lo (BF16 + BF16, or TF32 + TF32); the three
// products hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor memory.
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = TMEM allocator +
// single-thread MMA issuer, warps 2-5 = epilogue (TMEM -> registers -> HBM).
// Every wait is bounded in time; on expiry the kernel records an error bit,
// drains its own copies and MMAs (again bounded), frees TMEM and returns.
#include "legendre_tc_dev.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

namespace st {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    return fn;
}

// 3-D view of a split operand, 128-byte swizzle, zero fill outside the
// tensor.  BF16: [plane][row][column], box = 64 columns x 64 rows x 1 plane.
// TF32 (stored transposed): [plane][column][row], box = 32 rows x 128
// columns x 1 plane.  `rows` is the padded row count (a multiple of 4).
static st_status make_operand_map(CUtensorMap *map, void *base, bool bf16, int C, long long rows, int Cp)
{
    auto enc = encode_fn();
    if (!enc) {
        set_last_error("cuTensorMapEncodeTiled entry point not available");
        return ST_ERR_UNSUPPORTED;
    }
    const int es = bf16 ? 2 : 4;
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3];
    if (bf16) {
        dims[0] = (cuuint64_t)C; dims[1] = (cuuint64_t)rows; dims[2] = 2;
        strides[0] = (cuuint64_t)Cp * es;
        box[0] = 64; box[1] = 64; box[2] = 1;
    } else {
        dims[0] = (cuuint64_t)rows; dims[1] = (cuuint64_t)C; dims[2] = 2;
        strides[0] = (cuuint64_t)rows * es;
        box[0] = 32; box[1] = TC_M; box[2] = 1;
    }
    strides[1] = (cuuint64_t)rows * Cp * es;
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_last_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
        return ST_ERR_CUDA;
    }
    return ST_OK;
}

static int tc_max_nt(const st_plan *p, int set)
{
    int mx = 16;
    for (const auto &g : p->groups_h[set])
        if (g.nt > mx) mx = g.nt;
    return mx;
}

size_t tc_smem_bytes(int prec, int max_nt, int *stages_out, size_t cap)
{
    const size_t a = 2 * (size_t)TC_M * 128;  // two planes of 128 columns x 128 bytes
    const size_t stage = a + 2 * (size_t)max_nt * 128;
    const size_t ctrl = 256;
    const size_t limit = (cap ? cap : 227 * 1024) - 1024 - ctrl;
    int S = (int)(limit / stage);
    if (S > tc::MAX_STAGES) S = tc::MAX_STAGES;
    if (stages_out) *stages_out = S;
    (void)prec;
    return 1024 + (size_t)S * stage + ctrl;
}

st_status tc_job(st_plan *p, int set, int nfields, void *data, void *out, TcJob *job, int cp)
{
    TcJob &J = *job;
    const int dir = set_dir(set);
    const int C = 2 * nfields, Cp = cp ? cp : cols_padded(nfields);
    const bool bf16 = p->prec == P_BF16X3;
    const long long rows = dir == 0 ? p->srow_total : fb_rows(p);
    st_status r = make_operand_map(&J.map, data, bf16, C, rows, Cp);
    if (r != ST_OK) return r;
    J.groups = p->groups[set];
    J.tiles = p->tiles[dir];
    J.tab = (const char *)p->tab[set];
    J.out = (float *)out;
    J.err = p->err;
    J.C = C;
    J.Cp = Cp;
    J.ncm = (C + TC_M - 1) / TC_M;
    J.ntiles = (long long)p->ntiles[dir] * J.ncm;
    J.max_nt = tc_max_nt(p, set);
    return ST_OK;
}

template <int MAXJ>
static st_status run_tc_batch(int prec, const TcJob *jobs, int n, int sm_count, cudaStream_t s, int withhold,
                              unsigned long long wait_ns)
{
    tc::TcBatch<MAXJ> B;  // copied into the kernel's parameters at launch
    B.njobs = n;
    B.withhold_loads = withhold;
    B.wait_ns = wait_ns;
    long long tot = 0;
    int max_nt = 16;
    for (int q = 0; q < n; ++q) {
        B.prefix[q] = tot;
        B.job[q] = jobs[q];
        tot += jobs[q].ntiles;
        max_nt = std::max(max_nt, jobs[q].max_nt);
    }
    B.prefix[n] = tot;
    if (tot == 0) return ST_OK;
    B.max_nt = max_nt;
    int S = 0;
    const size_t smem = tc_smem_bytes(prec, max_nt, &S);
    if (S < 2) return ST_ERR_UNSUPPORTED;
    B.stages = S;
    const int grid = (int)(tot < sm_count ? tot : sm_count);
    if (prec == P_BF16X3) {
        auto k = tc::k_leg_tc<0, MAXJ>;
        ST_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, tc::THREADS, smem, s>>>(B);
        ++kernel_launches();
    } else {
        auto k = tc::k_leg_tc<1, MAXJ>;
        ST_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, tc::THREADS, smem, s>>>(B);
        ++kernel_launches();
    }
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

st_status launch_tc_jobs(int prec, const TcJob *jobs, int n, int sm_count, cudaStream_t s, int withhold,
                         unsigned long long wait_ns)
{
    if (n <= 0) return ST_OK;
    if (n > MAX_JOBS) return ST_ERR_ARG;
    if (n == 1) return run_tc_batch<1>(prec, jobs, n, sm_count, s, withhold, wait_ns);
    return run_tc_batch<MAX_JOBS>(prec, jobs, n, sm_count, s, withhold, wait_ns);
}

st_status launch_leg_tc(st_plan *p, int dir, int nfields, cudaStream_t s, void *data_in, void *out_in)
{
    void *data = data_in ? data_in : (dir == 0 ? p->sop : p->fbop);
    void *out = out_in ? out_in : (dir == 0 ? p->fb : p->sout);
    TcJob J;
    st_status r = tc_job(p, dir, nfields, data, out, &J);
    if (r) return r;
    const int withhold = p->inject_withhold;
    const unsigned long long wait_ns = withhold ? p->inject_wait_ns : tc::WAIT_NS;
    p->inject_withhold = 0;  // one launch only
    return launch_tc_jobs(p->prec, &J, 1, p->sm_count, s, withhold, wait_ns);
}

}  // namespace st
