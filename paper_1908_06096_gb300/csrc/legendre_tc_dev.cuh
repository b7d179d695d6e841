// Device side of the tcgen05 Legendre GEMM (legendre_tc.cu): PTX helpers,
// the batch layout and the body of one persistent CTA, shared by the
// per-stage kernel and the persistent batch kernel (batch_persistent.cu).
#pragma once

#include "st_internal.cuh"

#include <cuda.h>

namespace st {

namespace tc {

constexpr int THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s: no legitimate wait comes close
constexpr int MAX_STAGES = 6;

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ inline void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ inline void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ inline bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` to complete.  Returns false
// if the CTA is aborting or the wait ran past WAIT_NS (then it starts the
// abort and records `code` in the error word).
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err, int code,
                                 uint64_t wait_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > wait_ns) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}

// Drain wait (used after an abort): bounded, records nothing.
__device__ inline void mbar_drain(uint32_t bar, uint32_t parity, uint64_t wait_ns)
{
    uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > wait_ns) return;
    }
}

__device__ inline void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ inline void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ inline void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ inline void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ inline void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// KIND 0: kind::f16 with BF16 inputs; KIND 1: kind::tf32.
template <int KIND>
__device__ inline void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    if (KIND == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
}

__device__ inline void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ inline void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ inline void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: start, leading and stride byte offsets (in
// 16-byte units), descriptor version 1, 128-byte swizzle.
__device__ inline uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of the kind's 16/19-bit
// type, A MN-major (BF16) or K-major (TF32), B K-major, M = 128, N = n.
template <int KIND>
__device__ inline uint32_t idesc(int n)
{
    const uint32_t fmt = KIND == 0 ? 1u : 2u;  // BF16 : TF32
    const uint32_t a_mn = KIND == 0 ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (a_mn << 15) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(TC_M >> 4) << 24);
}

template <int MAXJ>
struct TcBatch {
    TcJob job[MAXJ];
    long long prefix[MAXJ + 1];  // tiles of job q: [prefix[q], prefix[q+1])
    int njobs;
    int max_nt;
    int stages;
    int withhold_loads;          // fault injection (tests): the producer issues no copies
    unsigned long long wait_ns;  // bound of every wait in this launch
};

// BF16 (KIND 0): the data operand A is MN-major (data columns contiguous in
// global memory and shared memory): per plane, TC_M / 64 TMA boxes of 64
// columns x 64 reduction rows, 128-byte swizzle; atoms of 8 reduction rows
// are 1024 bytes apart (SBO), 64-column blocks one box apart (LBO); an MMA K
// step of 16 spans two atoms.
// TF32 (KIND 1): the tensor cores take TF32 only K-major, so the data operand
// is stored transposed (reduction index contiguous) and A is K-major: one TMA
// box of 32 reduction values x 128 columns per plane; rows of 128 bytes in
// 1024-byte atoms of 8 (SBO); an MMA K step of 8 is 32 bytes along the row.
template <int KIND>
struct Geo {
    static constexpr int ES = KIND == 0 ? 2 : 4;        // bytes per element
    static constexpr int KC = 128 / ES;                 // reduction chunk (elements) = one 128-byte row
    static constexpr int UK = 32 / ES;                  // K of one MMA instruction
    static constexpr int A_PLANE = TC_M * KC * ES;      // 16 KB
    static constexpr bool A_MN = KIND == 0;
    static constexpr int BOX_C = A_MN ? 128 / ES : TC_M;  // data columns per TMA box
    static constexpr int NBOX = TC_M / BOX_C;           // boxes per plane per stage
    static constexpr int BOX_BYTES = BOX_C * KC * ES;
    static constexpr int A_LBO = A_MN ? BOX_BYTES : 16; // MN-direction atom stride (unused K-major)
    static constexpr int A_STEP = A_MN ? UK / 8 * 1024 : 32;  // bytes per MMA K step in A
};

// A GEMM job without its tensor map, as the persistent batch kernel keeps it
// in shared memory (its maps stay in kernel parameters).
struct TcLite {
    const LegGroup *groups;
    const LegTile *tiles;
    const char *tab;
    float *out;
    int *err;
    long long ntiles;
    int ncm, C, Cp, max_nt;
};
__device__ __forceinline__ const CUtensorMap *job_map(const TcJob &J, const CUtensorMap *maps, int q)
{
    return maps ? &maps[q] : &J.map;
}
__device__ __forceinline__ const CUtensorMap *job_map(const TcLite &, const CUtensorMap *maps, int q)
{
    return &maps[q];
}

// Named barrier of the kernel's THREADS threads (warps 0 .. 5): a launch of
// more warps (the persistent batch kernel) runs the body in its first six.
__device__ __forceinline__ void tc_sync() { asm volatile("bar.sync 1, %0;" ::"n"(THREADS) : "memory"); }

// The body of one CTA over tiles cta, cta + ncta, ... of batch B (B in
// kernel parameters or global memory); smem_raw: the dynamic shared memory.
// relinquish: give up the CTA's right to allocate tensor memory once its
// columns are held (a CTA that runs the body again must keep it).
// maps: the jobs' operand tensor maps when B lives in global memory (kernel
// parameters keep descriptor fetches cheap); null: each job's own.
template <int KIND, class BATCH>
__device__ __forceinline__ void leg_tc_body(const BATCH &B, unsigned char *smem_raw, long long cta, long long ncta,
                                            bool relinquish = true, const CUtensorMap *maps = nullptr)
{
    typedef Geo<KIND> G;
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = B.stages;
    const uint32_t b_bytes = 2u * (uint32_t)B.max_nt * 128u;
    const long long total = B.prefix[B.njobs];
    const uint64_t wait_ns = B.wait_ns;
    const uint32_t stage_bytes = 2u * G::A_PLANE + b_bytes;
    unsigned char *ctrl = smem + (size_t)S * stage_bytes;
    uint64_t *full = (uint64_t *)ctrl;
    uint64_t *empty = full + MAX_STAGES;
    uint64_t *tfull = empty + MAX_STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t smem_base = smem_u32(smem);

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&tfull[a]), 1);
            mbar_init(smem_u32(&tempty[a]), 128);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), 512);
        if (relinquish) tmem_relinquish();
    }
    fence_before();
    tc_sync();
    fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer
            int stage = 0;
            uint32_t ph = 0;
            int issued_mask = 0;
            uint32_t last_par[MAX_STAGES];
            for (int s = 0; s < MAX_STAGES; ++s) last_par[s] = 0;
            bool ok = true;
            for (long long t = cta; ok && t < total; t += ncta) {
                const int q = find_job<1>(B.prefix, B.njobs, t);
                const auto &J = B.job[q];
                const CUtensorMap *mp = job_map(J, maps, q);
                const long long lt_i = t - B.prefix[q];
                const LegTile lt = J.tiles[lt_i / J.ncm];
                const int cm = (int)(lt_i % J.ncm);
                const LegGroup g = J.groups[lt.g];
                const int kc_end = (g.K + G::KC - 1) / G::KC;
                const uint32_t bimg = 2u * (uint32_t)g.nt * 128u;
                for (int kc = g.r0 / G::KC; kc < kc_end; ++kc) {
                    if (!mbar_wait(smem_u32(&empty[stage]), ph ^ 1, abort_flag, J.err, 1, wait_ns)) { ok = false; break; }
                    const uint32_t fb = smem_u32(&full[stage]);
                    if (B.withhold_loads) {
                        // injected fault: nothing arms this stage, so the MMA issuer's
                        // bounded wait on it runs out
                        if (++stage == S) { stage = 0; ph ^= 1; }
                        continue;
                    }
                    mbar_expect_tx(fb, 2u * G::A_PLANE + bimg);
                    const uint32_t sa = smem_base + (uint32_t)stage * stage_bytes;
                    const int row = (int)(g.data_row0 + (long long)kc * G::KC);
#pragma unroll
                    for (int pl = 0; pl < 2; ++pl) {
                        if (G::A_MN) {
#pragma unroll
                            for (int bx = 0; bx < G::NBOX; ++bx)
                                tma_load_3d(sa + pl * G::A_PLANE + bx * G::BOX_BYTES, mp, cm * TC_M + bx * G::BOX_C,
                                            row, pl, fb);
                        } else {
                            tma_load_3d(sa + pl * G::A_PLANE, mp, row, cm * TC_M, pl, fb);
                        }
                    }
                    const char *src = J.tab + g.tab_off + (size_t)(lt.ct * g.nkc + kc) * bimg;
                    bulk_load(sa + 2 * G::A_PLANE, src, bimg, fb);
                    issued_mask |= 1 << stage;
                    last_par[stage] = ph;
                    if (++stage == S) { stage = 0; ph ^= 1; }
                }
            }
            // make sure no copy into this CTA's shared memory is still in flight
            for (int s = 0; s < S; ++s)
                if (issued_mask & (1 << s)) mbar_drain(smem_u32(&full[s]), last_par[s], wait_ns);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int stage = 0;
            uint32_t ph = 0;
            int local = 0;
            bool ok = true;
            bool any = false;
            for (long long t = cta; ok && t < total; t += ncta, ++local) {
                const int q = find_job<1>(B.prefix, B.njobs, t);
                const auto &J = B.job[q];
                const LegTile lt = J.tiles[(t - B.prefix[q]) / J.ncm];
                const LegGroup g = J.groups[lt.g];
                const int kc_end = (g.K + G::KC - 1) / G::KC;
                const int acc = local & 1;
                const uint32_t acc_ph = (local >> 1) & 1;
                if (!mbar_wait(smem_u32(&tempty[acc]), acc_ph ^ 1, abort_flag, J.err, 2, wait_ns)) { ok = false; break; }
                fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * 256);
                const uint32_t id = idesc<KIND>(g.nt);
                uint32_t accum = 0;
                for (int kc = g.r0 / G::KC; kc < kc_end; ++kc) {
                    if (!mbar_wait(smem_u32(&full[stage]), ph, abort_flag, J.err, 2, wait_ns)) { ok = false; break; }
                    fence_after();
                    const uint32_t sa = smem_base + (uint32_t)stage * stage_bytes;
                    const uint32_t sb = sa + 2 * G::A_PLANE;
                    const int kval = min(G::KC, g.K - kc * G::KC);
                    const int nks = (kval + G::UK - 1) / G::UK;
                    for (int ks = 0; ks < nks; ++ks) {
                        const uint64_t a_hi = sdesc(sa + ks * G::A_STEP, G::A_LBO, 1024);
                        const uint64_t a_lo = sdesc(sa + G::A_PLANE + ks * G::A_STEP, G::A_LBO, 1024);
                        const uint64_t b_hi = sdesc(sb + ks * 32, 16, 1024);
                        const uint64_t b_lo = sdesc(sb + (uint32_t)g.nt * 128u + ks * 32, 16, 1024);
                        mma<KIND>(d, a_hi, b_hi, id, accum);
                        mma<KIND>(d, a_hi, b_lo, id, 1);
                        mma<KIND>(d, a_lo, b_hi, id, 1);
                        accum = 1;
                    }
                    mma_commit(smem_u32(&empty[stage]));
                    any = true;
                    if (++stage == S) { stage = 0; ph ^= 1; }
                }
                if (!ok) break;
                mma_commit(smem_u32(&tfull[acc]));
            }
            if (!ok && any) {
                // wait (bounded) for every MMA issued so far before TMEM is released
                mma_commit(smem_u32(drain));
                mbar_drain(smem_u32(drain), 0, wait_ns);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lanes 32*(warp%4) ..
        const int q = warp & 3;
        const int i = q * 32 + lane;
        int local = 0;
        for (long long t = cta; t < total; t += ncta, ++local) {
            const int q = find_job<1>(B.prefix, B.njobs, t);
            const auto &J = B.job[q];
            const long long lt_i = t - B.prefix[q];
            const LegTile lt = J.tiles[lt_i / J.ncm];
            const int cm = (int)(lt_i % J.ncm);
            const LegGroup g = J.groups[lt.g];
            const int acc = local & 1;
            const uint32_t acc_ph = (local >> 1) & 1;
            // every lane observes the barrier; the decision to stop is warp-uniform so
            // that the .sync.aligned TMEM loads below never run in a partial warp
            const bool ok = mbar_wait(smem_u32(&tfull[acc]), acc_ph, abort_flag, J.err, 4, wait_ns);
            if (!__all_sync(0xffffffffu, ok)) break;
            fence_after();
            const int c = cm * TC_M + i;
            const int col0 = lt.ct * g.nt;
            const uint32_t taddr = tmem_base + (uint32_t)(acc * 256) + ((uint32_t)(q * 32) << 16);
            float *o = J.out + g.out_row0 * (long long)J.Cp + c;
            // the tile's columns that hold data (a group's last tile may be
            // partial), 32 a round: two loads from tensor memory in flight
            // before the wait
            const int jend = min(g.nt, (g.ncol - col0 + 15) & ~15);
            int j0 = 0;
            for (; j0 + 32 <= jend; j0 += 32) {
                uint32_t ra[16], rb[16];
                tmem_ld16(taddr + (uint32_t)j0, ra);
                tmem_ld16(taddr + (uint32_t)(j0 + 16), rb);
                tmem_ld_wait();
                if (c < J.C) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int col = col0 + j0 + u;
                        if (col < g.ncol) o[(long long)col * J.Cp] = __uint_as_float(ra[u]);
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int col = col0 + j0 + 16 + u;
                        if (col < g.ncol) o[(long long)col * J.Cp] = __uint_as_float(rb[u]);
                    }
                }
            }
            if (j0 < jend) {
                uint32_t r[16];
                tmem_ld16(taddr + (uint32_t)j0, r);
                tmem_ld_wait();
                if (c < J.C) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int col = col0 + j0 + u;
                        if (col < g.ncol) o[(long long)col * J.Cp] = __uint_as_float(r[u]);
                    }
                }
            }
            fence_before();
            mbar_arrive(smem_u32(&tempty[acc]));
        }
    }

    fence_before();
    tc_sync();
    fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, 512);
    // retire the barriers: a persistent CTA that runs the body again sets
    // them up afresh, possibly at other addresses of its shared memory
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_inval(smem_u32(&full[s]));
            mbar_inval(smem_u32(&empty[s]));
        }
        for (int a = 0; a < 2; ++a) {
            mbar_inval(smem_u32(&tfull[a]));
            mbar_inval(smem_u32(&tempty[a]));
        }
        mbar_inval(smem_u32(drain));
    }
}


template <int KIND, int MAXJ>
__global__ void __launch_bounds__(THREADS, 1) k_leg_tc(const __grid_constant__ TcBatch<MAXJ> B)
{
    extern __shared__ unsigned char smem_raw[];
    leg_tc_body<KIND>(B, smem_raw, blockIdx.x, gridDim.x);
}

}  // namespace tc
}  // namespace st
