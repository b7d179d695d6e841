// Persistent batch kernel: a whole batch of round trips (include/st.h,
// st_batch_run with use_graph = 2) in one cooperative launch.
//
// ESCAPE D3.3 sections 4.2.3-4.2.4 argue for fewer, larger kernels.  Here
// every stage of every request of a batch runs in one kernel of one CTA per
// SM (512 threads): the spectral pack, the tcgen05 Legendre GEMMs of the
// inverse, the inverse row FFTs, the direct row FFTs, the direct GEMMs and
// the unpack, separated by grid-wide barriers.  In the pack, FFT and unpack
// stages each half of a CTA works as one 256-thread CTA of the per-stage
// kernels would, claiming the stage's work items of all requests one at a
// time (the row FFTs longest first); the GEMM stages run the persistent
// tcgen05 body on six warps.  The stage bodies are the per-stage kernels'
// own (pack_dev.cuh, legendre_tc_dev.cuh, and the row-FFT bodies compiled
// for half CTAs in fft_half_*.cu).  Every barrier wait is
// bounded: past two seconds the CTA records bit 16 in the error word of the
// batch's first plan and every CTA leaves at its next barrier.
//
// Scope: BF16x3 batches (the 3xTF32 direct operand needs a transpose after
// the row FFTs, which this kernel does not run), at most 64 items a
// direction, every row on a compile-time FFT plan of groups 0 and 1
// (lengths up to 4096, truncations up to T639 on octahedral grids).  Other
// batches are refused with ST_ERR_UNSUPPORTED and run per stage.
#include "legendre_tc_dev.cuh"
#include "pack_dev.cuh"

#include <algorithm>
#include <cstring>

namespace st {

namespace ffh {
__device__ void half_dir_g0(const FftJob &J, const RowPair &rp, int f0);
__device__ void half_dir_g1(const FftJob &J, const RowPair &rp, int f0);
__device__ void half_inv_g0(const FftJob &J, const RowPair &rp, int f0);
__device__ void half_inv_g1(const FftJob &J, const RowPair &rp, int f0);
}  // namespace ffh

namespace pers {

constexpr int THREADS = 512;
constexpr int ERR_GRID = 16;
constexpr unsigned long long WAIT_NS = 2000000000ull;

// Work-item counters of the stages whose items are claimed one at a time.
enum { C_PACK = 0, C_FFT_INV = 1, C_FFT_DIR = 2, C_UNPACK = 3, NCLAIM = 4 };

// Units a half claims at once in the pack and FFT stages.
constexpr int PACK_CHUNK = 4, FFT_CHUNK = 8;

// A GEMM batch as the tcgen05 body reads it: tile prefix and launch facts in
// kernel parameters, the jobs themselves in global memory.
struct TcView {
    const tc::TcLite *job;  // set in the kernel: the CTA's copy in shared memory
    long long prefix[MAX_JOBS + 1];
    int njobs, max_nt, stages, withhold_loads;
    unsigned long long wait_ns;
};

struct Args {
    CUtensorMap maps_inv[MAX_JOBS], maps_dir[MAX_JOBS];  // the GEMM jobs' operand maps (kernel parameters)
    TcView tc_inv, tc_dir;
    const tc::TcLite *tcj_inv, *tcj_dir;  // the GEMM jobs in global memory
    const PackJob *pack, *unpack;
    const long long *pack_pre, *unpack_pre;
    const FftJob *fi, *fd;
    const long long *fi_pre, *fd_pre;
    int npack, nunpack, nfi, nfd;
    long long ntc_inv, ntc_dir;   // GEMM tiles of each direction
    unsigned long long *count;    // grid-barrier arrivals, then NCLAIM claim counters (zeroed before each launch)
    int *err;
};
static_assert(sizeof(Args) <= 32000, "kernel parameters");

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

// The next work item of a stage for this half (thread 0 of the half claims
// it, the half reads it after its barrier).
__device__ __forceinline__ long long claim(unsigned long long *ctr, long long *slot, int h, int chunk)
{
    if ((threadIdx.x & 255) == 0) *slot = (long long)atomicAdd(ctr, (unsigned long long)chunk);
    half_sync(h);
    const long long u = *(volatile long long *)slot;
    half_sync(h);
    return u;
}

// One stage of pack (UNPACK false) or unpack blocks: the CTA runs eight
// 64-thread blocks at a time, each with its own tile and barrier, claiming
// PACK_CHUNK blocks at once; the stage's job table is first copied to shared
// memory.
template <bool UNPACK, int S>
__device__ void pack_stage(const Args &A, const PackJob *jobs_g, const long long *pre_g, int n,
                           unsigned char *smem, long long *slots)
{
    if (n <= 0) return;
    constexpr int NB = 8, NWB = THREADS / 32 / NB;  // blocks per CTA, warps per block
    constexpr size_t TILE = 32 * 65 * sizeof(float);
    PackJob *jobs = (PackJob *)(smem + NB * TILE);
    long long *pre = (long long *)(jobs + MAX_JOBS);
    for (int i = threadIdx.x; i < n * (int)(sizeof(PackJob) / 8); i += THREADS)
        ((long long *)jobs)[i] = ((const long long *)jobs_g)[i];
    for (int i = threadIdx.x; i <= n; i += THREADS) pre[i] = pre_g[i];
    __syncthreads();
    const int blk = threadIdx.x / (32 * NWB), w = (threadIdx.x >> 5) % NWB, lane = threadIdx.x & 31;
    float(*tile)[65] = (float(*)[65])(smem + blk * TILE);
    auto bsync = [blk] { asm volatile("bar.sync %0, %1;" ::"r"(2 + blk), "n"(32 * NWB) : "memory"); };
    const long long tot = pre[n];
    unsigned long long *ctr = A.count + 1 + (UNPACK ? C_UNPACK : C_PACK);
    for (;;) {
        if ((threadIdx.x & (32 * NWB - 1)) == 0) slots[blk] = (long long)atomicAdd(ctr, (unsigned long long)PACK_CHUNK);
        bsync();
        const long long u0 = *(volatile long long *)&slots[blk];
        bsync();
        if (u0 >= tot) break;
        for (long long u = u0; u < u0 + PACK_CHUNK && u < tot; ++u) {
            const int q = find_job<1>(pre, n, u);
            const int b = (int)(u - pre[q]);
            if (UNPACK) unpack_block<float, 1, NWB>(jobs[q], b, tile, w, lane, bsync);
            else pack_block<float, S, 1, NWB>(jobs[q], b, tile, w, lane, bsync);
        }
    }
}

// One stage of row FFTs: each half takes (row pair, field group) items in
// turn, FFT_CHUNK a claim, the stage's jobs sorted longest rows first; the
// next item's row description is fetched asynchronously while the current
// item runs.  A row whose bounded wait gave up (error bit 8 of its plan)
// ends the stage for this half and marks the batch abandoned.
template <int DIR>
__device__ void fft_stage(const Args &A, const FftJob *jobs, const long long *pre, int n, RowPair (*rps)[2],
                          long long *slots)
{
    if (n <= 0) return;
    const int h = threadIdx.x >> 8, t = threadIdx.x & 255;
    constexpr int NW = (int)(sizeof(RowPair) / sizeof(int));
    const long long tot = pre[n];
    unsigned long long *ctr = A.count + 1 + (DIR ? C_FFT_DIR : C_FFT_INV);
    // item u of job q: its row-pair entry
    auto fetch = [&](int q, long long u, RowPair *dst) {
        const FftJob &J = jobs[q];
        const int rr = (int)(u - pre[q]) / J.nfg;
        const int *src = (const int *)(J.rps + J.r0 + rr);
        if (t < NW)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared((int *)dst + t)),
                         "l"(src + t)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int *errp = jobs[0].err;
    for (;;) {
        // claim the next FFT_CHUNK items, or stop (the claimed batch is done,
        // or the last item's plan recorded a bounded wait that gave up)
        if (t == 0) {
            const bool failed = (*(volatile const int *)errp & 8) != 0;
            if (failed) atomicOr(A.err, ERR_GRID);
            slots[h] = failed ? tot : (long long)atomicAdd(ctr, (unsigned long long)FFT_CHUNK);
        }
        half_sync(h);
        const long long u0 = *(volatile long long *)&slots[h];
        half_sync(h);
        if (u0 >= tot) break;
        const long long u1 = u0 + FFT_CHUNK < tot ? u0 + FFT_CHUNK : tot;
        int q = find_job<1>(pre, n, u0);
        fetch(q, u0, &rps[h][0]);
        int qn = q;
        for (long long u = u0; u < u1; ++u) {
            const int buf = (int)((u - u0) & 1);
            asm volatile("cp.async.wait_all;" ::: "memory");
            half_sync(h);
            if (u + 1 < u1) {
                while (pre[qn + 1] <= u + 1) ++qn;
                fetch(qn, u + 1, &rps[h][buf ^ 1]);
            }
            const FftJob &J = jobs[q];
            const int b = (int)(u - pre[q]);
            const int f0 = (b - (b / J.nfg) * J.nfg) * J.G;
            if (J.kind == 0) {
                if (DIR) ffh::half_dir_g0(J, rps[h][buf], f0);
                else ffh::half_inv_g0(J, rps[h][buf], f0);
            } else {
                if (DIR) ffh::half_dir_g1(J, rps[h][buf], f0);
                else ffh::half_inv_g1(J, rps[h][buf], f0);
            }
            q = qn;
            half_sync(h);
        }
        errp = jobs[q].err;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// One GEMM stage: the jobs are copied to shared memory (their per-tile
// lookups then cost no global round trips), then six warps run the tcgen05
// body over the stage's tiles.
template <int KIND>
__device__ void gemm_stage(const TcView &V, const tc::TcLite *jobs_g, const CUtensorMap *maps, long long tiles,
                           tc::TcLite *jobs_s, unsigned char *smem)
{
    if (tiles <= 0) return;
    for (int i = threadIdx.x; i < V.njobs * (int)(sizeof(tc::TcLite) / 8); i += THREADS)
        ((long long *)jobs_s)[i] = ((const long long *)jobs_g)[i];
    __syncthreads();
    if (threadIdx.x < tc::THREADS) {
        TcView v = V;
        v.job = jobs_s;
        tc::leg_tc_body<KIND>(v, smem, blockIdx.x, gridDim.x, false, maps);
    }
}

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1) k_batch_persistent(const __grid_constant__ Args A)
{
    extern __shared__ __align__(1024) unsigned char pers_smem[];
    __shared__ RowPair rps[2][2];
    __shared__ long long slots[8];
    __shared__ int abort_s;
    __shared__ __align__(16) tc::TcLite tcj[MAX_JOBS];
    constexpr int S = KIND == 0 ? S_BF16_SPLIT : S_TF32_SPLIT;
    const unsigned long long g = gridDim.x;

    pack_stage<false, S>(A, A.pack, A.pack_pre, A.npack, pers_smem, slots);
    if (!grid_sync(A, 1 * g, &abort_s)) return;
    gemm_stage<KIND>(A.tc_inv, A.tcj_inv, A.maps_inv, A.ntc_inv, tcj, pers_smem);
    if (!grid_sync(A, 2 * g, &abort_s)) return;
    fft_stage<0>(A, A.fi, A.fi_pre, A.nfi, rps, slots);
    if (!grid_sync(A, 3 * g, &abort_s)) return;
    fft_stage<1>(A, A.fd, A.fd_pre, A.nfd, rps, slots);
    if (!grid_sync(A, 4 * g, &abort_s)) return;
    gemm_stage<KIND>(A.tc_dir, A.tcj_dir, A.maps_dir, A.ntc_dir, tcj, pers_smem);
    if (!grid_sync(A, 5 * g, &abort_s)) return;
    pack_stage<true, S>(A, A.unpack, A.unpack_pre, A.nunpack, pers_smem, slots);
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

st_status tc_view(int prec, const std::vector<TcJob> &jobs, pers::TcView *B, size_t *smem, long long *tiles)
{
    memset((void *)B, 0, sizeof(*B));
    B->njobs = (int)jobs.size();
    B->withhold_loads = 0;
    B->wait_ns = tc::WAIT_NS;
    long long tot = 0;
    int max_nt = 16;
    for (size_t q = 0; q < jobs.size(); ++q) {
        B->prefix[q] = tot;
        tot += jobs[q].ntiles;
        max_nt = std::max(max_nt, jobs[q].max_nt);
    }
    B->prefix[jobs.size()] = tot;
    B->max_nt = max_nt;
    int S = 0;
    *smem = tc_smem_bytes(prec, max_nt, &S, 2 * (size_t)FF_HALF_BYTES);
    if (S < 2) return ST_ERR_UNSUPPORTED;
    B->stages = S;
    *tiles = tot;
    return ST_OK;
}

}  // namespace

st_status pers_prepare(const PersInput &in, PersState **out)
{
    *out = nullptr;
    if (in.prec != P_BF16X3) {
        set_last_error("the persistent batch kernel runs BF16x3 batches only");
        return ST_ERR_UNSUPPORTED;
    }
    if (in.tc_inv.size() > (size_t)MAX_JOBS || in.tc_dir.size() > (size_t)MAX_JOBS) {
        set_last_error("the persistent batch kernel takes at most 64 items a direction");
        return ST_ERR_UNSUPPORTED;
    }
    for (const auto *v : {&in.fft_inv, &in.fft_dir})
        for (const FftJob &J : *v) {
            if (J.kind != 0 && J.kind != 1) {
                set_last_error("a row of this batch has no compile-time FFT plan of lengths up to 4096");
                return ST_ERR_UNSUPPORTED;
            }
            if (J.smem > FF_HALF_BYTES) {
                set_last_error("a row job of this batch needs more shared memory than half a CTA holds");
                return ST_ERR_UNSUPPORTED;
            }
        }
    // row-FFT jobs longest rows first, so that the items claimed last are short
    auto by_size = [](const FftJob &a, const FftJob &b) {
        return (long long)a.G * a.Sslot > (long long)b.G * b.Sslot;
    };
    std::vector<FftJob> fi = in.fft_inv, fd = in.fft_dir;
    std::stable_sort(fi.begin(), fi.end(), by_size);
    std::stable_sort(fd.begin(), fd.end(), by_size);
    auto *ps = new PersState;
    ps->prec = in.prec;
    pers::Args &A = ps->args;
    size_t sm0 = 0, sm1 = 0;
    long long t0 = 0, t1 = 0;
    st_status r = tc_view(in.prec, in.tc_inv, &A.tc_inv, &sm0, &t0);
    if (r == ST_OK) r = tc_view(in.prec, in.tc_dir, &A.tc_dir, &sm1, &t1);
    if (r != ST_OK) {
        delete ps;
        set_last_error("no GEMM pipeline fits the persistent batch kernel's shared memory");
        return r;
    }
    std::vector<long long> pp, up, fip, fdp;
    prefix_of<PackJob>(in.pack, pp, pack_units);
    prefix_of<PackJob>(in.unpack, up, pack_units);
    prefix_of<FftJob>(fi, fip, fft_units);
    prefix_of<FftJob>(fd, fdp, fft_units);

    // one CTA per SM: ask for more shared memory than two CTAs could share
    size_t smem = std::max({sm0, sm1, (size_t)2 * FF_HALF_BYTES, (size_t)8 * 32 * 65 * sizeof(float) + 8192});
    if (smem > 227 * 1024) {
        delete ps;
        set_last_error("the persistent batch kernel needs more shared memory than a CTA has");
        return ST_ERR_UNSUPPORTED;
    }

    // device tables, one allocation
    size_t off = 0;
    const size_t o_ti = off; off = up256(off + sizeof(tc::TcLite) * in.tc_inv.size());
    const size_t o_td = off; off = up256(off + sizeof(tc::TcLite) * in.tc_dir.size());
    const size_t o_pk = off; off = up256(off + sizeof(PackJob) * in.pack.size());
    const size_t o_pkp = off; off = up256(off + sizeof(long long) * pp.size());
    const size_t o_up = off; off = up256(off + sizeof(PackJob) * in.unpack.size());
    const size_t o_upp = off; off = up256(off + sizeof(long long) * up.size());
    const size_t o_fi = off; off = up256(off + sizeof(FftJob) * fi.size());
    const size_t o_fip = off; off = up256(off + sizeof(long long) * fip.size());
    const size_t o_fd = off; off = up256(off + sizeof(FftJob) * fd.size());
    const size_t o_fdp = off; off = up256(off + sizeof(long long) * fdp.size());
    const size_t o_cnt = off; off = up256(off + sizeof(unsigned long long) * (1 + pers::NCLAIM));
    std::vector<unsigned char> host(off, 0);
    for (int dir = 0; dir < 2; ++dir) {
        const std::vector<TcJob> &v = dir ? in.tc_dir : in.tc_inv;
        tc::TcLite *t = (tc::TcLite *)(host.data() + (dir ? o_td : o_ti));
        for (size_t q = 0; q < v.size(); ++q)
            t[q] = tc::TcLite{v[q].groups, v[q].tiles, v[q].tab, v[q].out, v[q].err, v[q].ntiles,
                          v[q].ncm, v[q].C, v[q].Cp, v[q].max_nt};
    }
    if (!in.pack.empty()) memcpy(host.data() + o_pk, in.pack.data(), sizeof(PackJob) * in.pack.size());
    memcpy(host.data() + o_pkp, pp.data(), sizeof(long long) * pp.size());
    if (!in.unpack.empty()) memcpy(host.data() + o_up, in.unpack.data(), sizeof(PackJob) * in.unpack.size());
    memcpy(host.data() + o_upp, up.data(), sizeof(long long) * up.size());
    if (!fi.empty()) memcpy(host.data() + o_fi, fi.data(), sizeof(FftJob) * fi.size());
    memcpy(host.data() + o_fip, fip.data(), sizeof(long long) * fip.size());
    if (!fd.empty()) memcpy(host.data() + o_fd, fd.data(), sizeof(FftJob) * fd.size());
    memcpy(host.data() + o_fdp, fdp.data(), sizeof(long long) * fdp.size());

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
    A.tcj_inv = (const tc::TcLite *)(d + o_ti);
    A.tcj_dir = (const tc::TcLite *)(d + o_td);
    for (size_t q = 0; q < in.tc_inv.size(); ++q) A.maps_inv[q] = in.tc_inv[q].map;
    for (size_t q = 0; q < in.tc_dir.size(); ++q) A.maps_dir[q] = in.tc_dir[q].map;
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
    A.nfi = (int)fi.size();
    A.nfd = (int)fd.size();
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
    ST_CUDA(cudaMemsetAsync(ps->args.count, 0, sizeof(unsigned long long) * (1 + pers::NCLAIM), s));
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
