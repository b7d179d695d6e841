// Persistent batch kernel: a whole batch of round trips (include/st.h,
// st_batch_run with use_graph = 2) in one cooperative launch.
//
// ESCAPE D3.3 sections 4.2.3-4.2.4 argue for fewer, larger kernels.  Here
// every stage of every request of a batch runs in one kernel of one CTA per
// SM (512 threads): the spectral pack, the tcgen05 Legendre GEMMs of the
// inverse, the inverse row FFTs, the direct row FFTs, the direct GEMMs and
// the unpack, each stage a loop of the CTAs over that stage's work items of
// all requests, separated by grid-wide barriers.  The stage bodies are the
// per-stage kernels' own (pack_dev.cuh, legendre_tc_dev.cuh, and the row-FFT
// bodies compiled at this CTA width in fft_wide_*.cu).  Every barrier wait is
// bounded: past two seconds the CTA records bit 16 in the error word of the
// batch's first plan and every CTA leaves at its next barrier.
//
// Scope: one precision of the tensor-core forms (BF16x3 or 3xTF32), at most
// 64 items a direction, every row on a compile-time FFT plan of groups 0 and
// 1 (lengths up to 4096, truncations up to T639 on octahedral grids).  Other
// batches are refused with ST_ERR_UNSUPPORTED and run per stage.
#include "legendre_tc_dev.cuh"
#include "pack_dev.cuh"

#include <algorithm>
#include <cstring>

namespace st {

namespace ffw {
__device__ void wide_dir_g0(const FftJob &J, const RowPair &rp, int f0);
__device__ void wide_dir_g1(const FftJob &J, const RowPair &rp, int f0);
__device__ void wide_inv_g0(const FftJob &J, const RowPair &rp, int f0);
__device__ void wide_inv_g1(const FftJob &J, const RowPair &rp, int f0);
}  // namespace ffw

namespace pers {

constexpr int THREADS = 512;
constexpr int ERR_GRID = 16;
constexpr unsigned long long WAIT_NS = 2000000000ull;

struct Args {
    const void *tc_inv, *tc_dir;  // tc::TcBatch<MAX_JOBS> in global memory
    const PackJob *pack, *unpack;
    const long long *pack_pre, *unpack_pre;
    const FftJob *fi, *fd;
    const long long *fi_pre, *fd_pre;
    int npack, nunpack, nfi, nfd;
    long long ntc_inv, ntc_dir;   // GEMM tiles of each direction
    unsigned long long *count;    // grid-barrier arrivals (zeroed before each launch)
    int *err;
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// All CTAs: make this stage's writes visible (also to the tensor-copy
// engine, which reads the operands of the next GEMM stage), then wait,
// bounded, until every CTA has arrived `target` arrivals in all.  false:
// the batch is being abandoned.
__device__ bool grid_sync(const Args &A, unsigned long long target, volatile int *abort_s)
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(A.count, 1ull);
        const unsigned long long t0 = tc::gtimer();
        int ab = 0;
        while (ld_acquire(A.count) < target) {
            if (*(volatile int *)A.err & ERR_GRID) { ab = 1; break; }
            if (tc::gtimer() - t0 > WAIT_NS) {
                atomicOr(A.err, ERR_GRID);
                ab = 1;
                break;
            }
        }
        *abort_s = ab;
    }
    __syncthreads();
    __threadfence();
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return *abort_s == 0;
}

__device__ __forceinline__ void half_sync(int h) { asm volatile("bar.sync %0, 256;" ::"r"(2 + h) : "memory"); }

// One stage of pack (UNPACK false) or unpack blocks: each CTA runs two
// 256-thread blocks at a time, one per half, each with its own tile and
// barrier.
template <bool UNPACK, int S>
__device__ void pack_stage(const PackJob *jobs, const long long *pre, int n, unsigned char *smem)
{
    if (n <= 0) return;
    const int h = threadIdx.x >> 8, w = (threadIdx.x >> 5) & 7, lane = threadIdx.x & 31;
    float(*tile)[65] = (float(*)[65])(smem + h * (32 * 65 * sizeof(float)));
    const long long tot = pre[n];
    for (long long u = 2LL * blockIdx.x + h; u < tot; u += 2LL * gridDim.x) {
        const int q = find_job<1>(pre, n, u);
        const int b = (int)(u - pre[q]);
        if (UNPACK) unpack_block<float>(jobs[q], b, tile, w, lane, [h] { half_sync(h); });
        else pack_block<float, S>(jobs[q], b, tile, w, lane, [h] { half_sync(h); });
    }
}

// One stage of row FFTs: the CTAs take the stage's (row pair, field group)
// items in turn.
// A row whose bounded wait gave up (error bit 8 of its plan) ends the
// stage for this CTA and marks the batch abandoned.
template <int DIR>
__device__ void fft_stage(const Args &A, const FftJob *jobs, const long long *pre, int n, RowPair *rp,
                          volatile int *stop)
{
    if (n <= 0) return;
    const long long tot = pre[n];
    for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
        const int q = find_job<1>(pre, n, u);
        const FftJob &J = jobs[q];
        const int b = (int)(u - pre[q]);
        const int rr = b / J.nfg;
        const int f0 = (b - rr * J.nfg) * J.G;
        const int nw = (int)(sizeof(RowPair) / sizeof(int));
        const int *src = (const int *)(J.rps + J.r0 + rr);
        for (int i = threadIdx.x; i < nw; i += THREADS) ((int *)rp)[i] = src[i];
        __syncthreads();
        if (J.kind == 0) {
            if (DIR) ffw::wide_dir_g0(J, *rp, f0);
            else ffw::wide_inv_g0(J, *rp, f0);
        } else {
            if (DIR) ffw::wide_dir_g1(J, *rp, f0);
            else ffw::wide_inv_g1(J, *rp, f0);
        }
        if (threadIdx.x == 0) {
            *stop = (*(volatile int *)J.err & 8) != 0;
            if (*stop) atomicOr(A.err, ERR_GRID);
        }
        __syncthreads();
        if (*stop) return;
    }
}

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1) k_batch_persistent(const __grid_constant__ Args A)
{
    extern __shared__ __align__(1024) unsigned char pers_smem[];
    __shared__ RowPair rp;
    __shared__ int abort_s;
    constexpr int S = KIND == 0 ? S_BF16_SPLIT : S_TF32_SPLIT;
    const unsigned long long g = gridDim.x;

    pack_stage<false, S>(A.pack, A.pack_pre, A.npack, pers_smem);
    if (!grid_sync(A, 1 * g, &abort_s)) return;
    if (A.ntc_inv > 0 && threadIdx.x < tc::THREADS)
        tc::leg_tc_body<KIND>(*(const tc::TcBatch<MAX_JOBS> *)A.tc_inv, pers_smem, blockIdx.x, gridDim.x, false);
    if (!grid_sync(A, 2 * g, &abort_s)) return;
    fft_stage<0>(A, A.fi, A.fi_pre, A.nfi, &rp, &abort_s);
    if (!grid_sync(A, 3 * g, &abort_s)) return;
    fft_stage<1>(A, A.fd, A.fd_pre, A.nfd, &rp, &abort_s);
    if (!grid_sync(A, 4 * g, &abort_s)) return;
    if (A.ntc_dir > 0 && threadIdx.x < tc::THREADS)
        tc::leg_tc_body<KIND>(*(const tc::TcBatch<MAX_JOBS> *)A.tc_dir, pers_smem, blockIdx.x, gridDim.x, false);
    if (!grid_sync(A, 5 * g, &abort_s)) return;
    pack_stage<true, S>(A.unpack, A.unpack_pre, A.nunpack, pers_smem);
}

}  // namespace pers

// ---------------------------------------------------------------- host

struct PersState {
    int prec = 0;
    int grid = 0;
    size_t smem = 0;
    void *dev = nullptr;  // job tables, tile batches and the barrier counter
    pers::Args args;
};

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class J>
long long prefix_of(const std::vector<J> &jobs, std::vector<long long> &pre, long long (*units)(const J &))
{
    pre.assign(jobs.size() + 1, 0);
    for (size_t q = 0; q < jobs.size(); ++q) pre[q + 1] = pre[q] + units(jobs[q]);
    return pre.back();
}

long long pack_units(const PackJob &J) { return (long long)J.nm * J.nft; }
long long fft_units(const FftJob &J) { return (long long)J.J * J.nfg; }

st_status tc_batch(int prec, const std::vector<TcJob> &jobs, tc::TcBatch<MAX_JOBS> *B, size_t *smem, long long *tiles)
{
    memset((void *)B, 0, sizeof(*B));
    B->njobs = (int)jobs.size();
    B->withhold_loads = 0;
    B->wait_ns = tc::WAIT_NS;
    long long tot = 0;
    int max_nt = 16;
    for (size_t q = 0; q < jobs.size(); ++q) {
        B->prefix[q] = tot;
        B->job[q] = jobs[q];
        tot += jobs[q].ntiles;
        max_nt = std::max(max_nt, jobs[q].max_nt);
    }
    B->prefix[jobs.size()] = tot;
    B->max_nt = max_nt;
    int S = 0;
    *smem = tc_smem_bytes(prec, max_nt, &S);
    if (S < 2) return ST_ERR_UNSUPPORTED;
    B->stages = S;
    *tiles = tot;
    return ST_OK;
}

}  // namespace

st_status pers_prepare(const PersInput &in, PersState **out)
{
    *out = nullptr;
    if (in.prec != P_BF16X3 && in.prec != P_TF32X3) {
        set_last_error("the persistent batch kernel runs BF16x3 and 3xTF32 batches only");
        return ST_ERR_UNSUPPORTED;
    }
    if (in.tc_inv.size() > (size_t)MAX_JOBS || in.tc_dir.size() > (size_t)MAX_JOBS) {
        set_last_error("the persistent batch kernel takes at most 64 items a direction");
        return ST_ERR_UNSUPPORTED;
    }
    size_t fft_smem = 0;
    for (const auto *v : {&in.fft_inv, &in.fft_dir})
        for (const FftJob &J : *v) {
            if (J.kind != 0 && J.kind != 1) {
                set_last_error("a row of this batch has no compile-time FFT plan of lengths up to 4096");
                return ST_ERR_UNSUPPORTED;
            }
            fft_smem = std::max(fft_smem, (size_t)J.smem);
        }
    auto *B0 = new tc::TcBatch<MAX_JOBS>;
    auto *B1 = new tc::TcBatch<MAX_JOBS>;
    size_t sm0 = 0, sm1 = 0;
    long long t0 = 0, t1 = 0;
    st_status r = tc_batch(in.prec, in.tc_inv, B0, &sm0, &t0);
    if (r == ST_OK) r = tc_batch(in.prec, in.tc_dir, B1, &sm1, &t1);
    if (r != ST_OK) {
        delete B0;
        delete B1;
        set_last_error("no GEMM pipeline fits the persistent batch kernel's shared memory");
        return r;
    }
    std::vector<long long> pp, up, fip, fdp;
    prefix_of<PackJob>(in.pack, pp, pack_units);
    prefix_of<PackJob>(in.unpack, up, pack_units);
    prefix_of<FftJob>(in.fft_inv, fip, fft_units);
    prefix_of<FftJob>(in.fft_dir, fdp, fft_units);

    // one CTA per SM: ask for more shared memory than two CTAs could share
    size_t smem = std::max({sm0, sm1, fft_smem, (size_t)2 * 32 * 65 * sizeof(float), (size_t)120 * 1024});
    if (smem > 227 * 1024) {
        delete B0;
        delete B1;
        set_last_error("the persistent batch kernel needs more shared memory than a CTA has");
        return ST_ERR_UNSUPPORTED;
    }

    // device tables, one allocation
    size_t off = 0;
    const size_t o_tc0 = off; off = up256(off + sizeof(*B0));
    const size_t o_tc1 = off; off = up256(off + sizeof(*B1));
    const size_t o_pk = off; off = up256(off + sizeof(PackJob) * in.pack.size());
    const size_t o_pkp = off; off = up256(off + sizeof(long long) * pp.size());
    const size_t o_up = off; off = up256(off + sizeof(PackJob) * in.unpack.size());
    const size_t o_upp = off; off = up256(off + sizeof(long long) * up.size());
    const size_t o_fi = off; off = up256(off + sizeof(FftJob) * in.fft_inv.size());
    const size_t o_fip = off; off = up256(off + sizeof(long long) * fip.size());
    const size_t o_fd = off; off = up256(off + sizeof(FftJob) * in.fft_dir.size());
    const size_t o_fdp = off; off = up256(off + sizeof(long long) * fdp.size());
    const size_t o_cnt = off; off = up256(off + sizeof(unsigned long long));
    std::vector<unsigned char> host(off, 0);
    memcpy(host.data() + o_tc0, (const void *)B0, sizeof(*B0));
    memcpy(host.data() + o_tc1, (const void *)B1, sizeof(*B1));
    delete B0;
    delete B1;
    if (!in.pack.empty()) memcpy(host.data() + o_pk, in.pack.data(), sizeof(PackJob) * in.pack.size());
    memcpy(host.data() + o_pkp, pp.data(), sizeof(long long) * pp.size());
    if (!in.unpack.empty()) memcpy(host.data() + o_up, in.unpack.data(), sizeof(PackJob) * in.unpack.size());
    memcpy(host.data() + o_upp, up.data(), sizeof(long long) * up.size());
    if (!in.fft_inv.empty()) memcpy(host.data() + o_fi, in.fft_inv.data(), sizeof(FftJob) * in.fft_inv.size());
    memcpy(host.data() + o_fip, fip.data(), sizeof(long long) * fip.size());
    if (!in.fft_dir.empty()) memcpy(host.data() + o_fd, in.fft_dir.data(), sizeof(FftJob) * in.fft_dir.size());
    memcpy(host.data() + o_fdp, fdp.data(), sizeof(long long) * fdp.size());

    auto *ps = new PersState;
    ps->prec = in.prec;
    cudaError_t e = cudaMalloc(&ps->dev, off);
    if (e != cudaSuccess) {
        delete ps;
        return cuda_fail(e, "cudaMalloc (persistent batch tables)");
    }
    e = cudaMemcpy(ps->dev, host.data(), off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pers_free(ps);
        return cuda_fail(e, "cudaMemcpy (persistent batch tables)");
    }
    unsigned char *d = (unsigned char *)ps->dev;
    pers::Args &A = ps->args;
    A.tc_inv = d + o_tc0;
    A.tc_dir = d + o_tc1;
    A.pack = (const PackJob *)(d + o_pk);
    A.pack_pre = (const long long *)(d + o_pkp);
    A.unpack = (const PackJob *)(d + o_up);
    A.unpack_pre = (const long long *)(d + o_upp);
    A.fi = (const FftJob *)(d + o_fi);
    A.fi_pre = (const long long *)(d + o_fip);
    A.fd = (const FftJob *)(d + o_fd);
    A.fd_pre = (const long long *)(d + o_fdp);
    A.npack = (int)in.pack.size();
    A.nunpack = (int)in.unpack.size();
    A.nfi = (int)in.fft_inv.size();
    A.nfd = (int)in.fft_dir.size();
    A.ntc_inv = t0;
    A.ntc_dir = t1;
    A.count = (unsigned long long *)(d + o_cnt);
    A.err = in.err;

    const void *k = in.prec == P_BF16X3 ? (const void *)pers::k_batch_persistent<0> : (const void *)pers::k_batch_persistent<1>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, pers::THREADS, smem);
    if (e != cudaSuccess) {
        pers_free(ps);
        return cuda_fail(e, "persistent batch kernel set-up");
    }
    if (per_sm < 1) {
        pers_free(ps);
        set_last_error("the persistent batch kernel does not fit an SM");
        return ST_ERR_UNSUPPORTED;
    }
    ps->grid = in.sm_count;
    ps->smem = smem;
    *out = ps;
    return ST_OK;
}

st_status pers_launch(PersState *ps, cudaStream_t s)
{
    if (!ps) return ST_ERR_ARG;
    ST_CUDA(cudaMemsetAsync(ps->args.count, 0, sizeof(unsigned long long), s));
    const void *k =
        ps->prec == P_BF16X3 ? (const void *)pers::k_batch_persistent<0> : (const void *)pers::k_batch_persistent<1>;
    void *params[] = {(void *)&ps->args};
    ST_CUDA(cudaLaunchCooperativeKernel(k, dim3(ps->grid), dim3(pers::THREADS), params, ps->smem, s));
    return ST_OK;
}

void pers_free(PersState *ps)
{
    if (!ps) return;
    if (ps->dev) cudaFree(ps->dev);
    delete ps;
}

}  // namespace st
