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
#include "st_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

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

template <int KIND, int MAXJ>
__global__ void __launch_bounds__(THREADS, 1) k_leg_tc(const __grid_constant__ TcBatch<MAXJ> B)
{
    typedef Geo<KIND> G;
    extern __shared__ unsigned char smem_raw[];
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
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
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
            for (long long t = blockIdx.x; ok && t < total; t += gridDim.x) {
                const int q = find_job<MAXJ>(B.prefix, B.njobs, t);
                const TcJob &J = B.job[q];
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
                                tma_load_3d(sa + pl * G::A_PLANE + bx * G::BOX_BYTES, &J.map, cm * TC_M + bx * G::BOX_C,
                                            row, pl, fb);
                        } else {
                            tma_load_3d(sa + pl * G::A_PLANE, &J.map, row, cm * TC_M, pl, fb);
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
            for (long long t = blockIdx.x; ok && t < total; t += gridDim.x, ++local) {
                const int q = find_job<MAXJ>(B.prefix, B.njobs, t);
                const TcJob &J = B.job[q];
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
        for (long long t = blockIdx.x; t < total; t += gridDim.x, ++local) {
            const int q = find_job<MAXJ>(B.prefix, B.njobs, t);
            const TcJob &J = B.job[q];
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
            for (int j0 = 0; j0 < g.nt; j0 += 16) {
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
    __syncthreads();
    fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, 512);
}

}  // namespace tc

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

size_t tc_smem_bytes(int prec, int max_nt, int *stages_out)
{
    const size_t a = 2 * (size_t)TC_M * 128;  // two planes of 128 columns x 128 bytes
    const size_t stage = a + 2 * (size_t)max_nt * 128;
    const size_t ctrl = 256;
    const size_t limit = 227 * 1024 - 1024 - ctrl;
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
    } else {
        auto k = tc::k_leg_tc<1, MAXJ>;
        ST_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, tc::THREADS, smem, s>>>(B);
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
