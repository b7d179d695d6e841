// Spectral pack / unpack bodies (legendre_simt.cu): one 256-thread block's
// work, shared by the per-stage kernels and the persistent batch kernel.
#pragma once

#include "st_internal.cuh"

#include <cuda_bf16.h>

#include <type_traits>

namespace st {

__device__ inline float round_tf32_p(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int S, typename Rr>
__device__ inline void put_op(void *base, long long idx, long long ps, Rr v)
{
    if (S == S_F64) {
        ((double *)base)[idx] = (double)v;
    } else if (S == S_F32) {
        ((float *)base)[idx] = (float)v;
    } else if (S == S_TF32_SPLIT) {
        float f = (float)v, hi = round_tf32_p(f), lo = round_tf32_p(f - hi);
        ((float *)base)[idx] = hi;
        ((float *)base)[idx + ps] = lo;
    } else {
        float f = (float)v;
        __nv_bfloat16 hi = __float2bfloat16_rn(f);
        __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
        ((__nv_bfloat16 *)base)[idx] = hi;
        ((__nv_bfloat16 *)base)[idx + ps] = lo;
    }
}

// Spectra [field][(m,n)][re,im] -> operand rows: (m, n) with n - m = 2k + p
// goes to row srow[2m + p] + k (the even half, then the odd half of each m);
// column 2 f + (re, im).  One CTA per (m, 32-field tile); smem transpose.
// One 256-thread block b of job J: warp, lane of the block's own threads,
// tile 32 x 65 values of shared memory, sync() a barrier of the block.
// CH: chunks of 32 degrees moved per round (tile CH x 32 rows), so that a
// block with few neighbours on its SM keeps more loads in flight.
// NW: warps of the block (8: 256 threads; fewer for blocks that share a CTA).
template <typename Rr, int S, int CH = 1, int NW = 8, class SYNC>
__device__ __forceinline__ void pack_block(const PackJob &J, int b, Rr (*tile)[65], int warp, int lane, SYNC sync)
{
    const int m = b / J.nft;
    const int f0 = (b - m * J.nft) * 32;
    const int T = J.T, nfields = J.nfields, Cp = J.Cp;
    const long long nspec = J.nspec, Rp = J.Rp, ps = J.ps;
    const Rr *spec = (const Rr *)J.src;
    void *out = J.dst;
    const long long q0 = (long long)m * (T + 1) - (long long)m * (m - 1) / 2;
    const int len = T - m + 1;
    const long long rowE = J.srow[2 * m], rowO = J.srow[2 * m + 1];
    // one vector load per complex value where the caller's spectra allow it
    // (every value then starts at a multiple of its own size)
    using V2 = std::conditional_t<std::is_same<Rr, double>::value, double2, float2>;
    const bool vec = (reinterpret_cast<uintptr_t>(spec) & (sizeof(V2) - 1)) == 0;
    for (int d0 = 0; d0 < len; d0 += 32 * CH) {
        // load: warp w reads fields w, w + NW, ... of each chunk (all loads
        // in flight before the first store); lane = d
        constexpr int FK = 32 / NW;
        Rr re[CH][FK], im[CH][FK];
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < FK; ++k) {
                const int fld = f0 + warp + NW * k, d = d0 + 32 * c + lane;
                re[c][k] = im[c][k] = 0;
                if (fld < nfields && d < len) {
                    const Rr *a = spec + ((long long)fld * nspec + q0 + d) * 2;
                    if (vec) {
                        const V2 z = *reinterpret_cast<const V2 *>(a);
                        re[c][k] = z.x;
                        im[c][k] = z.y;
                    } else {
                        re[c][k] = a[0];
                        im[c][k] = a[1];
                    }
                    if (m == 0) im[c][k] = 0;
                    if (J.scale) {
                        // inverse Laplacian on the unit sphere: -1 / (n (n+1)), 0 at n = 0
                        const int n = m + d;
                        const Rr f = n == 0 ? (Rr)0 : (Rr)(-1.0 / ((double)n * (n + 1.0)));
                        re[c][k] *= f;
                        im[c][k] *= f;
                    }
                }
            }
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < FK; ++k) {
                tile[32 * c + lane][2 * (warp + NW * k)] = re[c][k];
                tile[32 * c + lane][2 * (warp + NW * k) + 1] = im[c][k];
            }
        sync();
        if constexpr (S == S_TF32_SPLIT) {
            // column-major operand (rows contiguous per column): warp w
            // writes columns w, w + NW, ...; lanes cover the rows
            for (int cc = warp; cc < 64; cc += NW) {
                const int c = 2 * f0 + cc;
                if (c >= 2 * nfields) continue;
                for (int dd = lane; dd < 32 * CH; dd += 32) {
                    const int d = d0 + dd;
                    if (d >= len) continue;
                    const long long row = ((d & 1) ? rowO : rowE) + (d >> 1);
                    put_op<S, Rr>(out, op_index(S, row, c, Cp, Rp), ps, tile[dd][cc]);
                }
            }
        } else {
            // store: warp w writes rows d = w, w + NW, ...; lanes cover 64 columns
            for (int dd = warp; dd < 32 * CH; dd += NW) {
                int d = d0 + dd;
                if (d >= len) continue;
                long long row = ((d & 1) ? rowO : rowE) + (d >> 1);
                for (int cc = lane; cc < 64; cc += 32) {
                    int c = 2 * f0 + cc;
                    if (c < 2 * nfields) put_op<S, Rr>(out, op_index(S, row, c, Cp, Rp), ps, tile[dd][cc]);
                }
            }
        }
        sync();
    }
}

// Operand rows (direct GEMM output, FP32/FP64) -> spectra.  Wavenumbers kept
// by no row (m > max_m) are written as zero; Im a_n^0 is written as zero.
template <typename Rr, int CH = 1, int NW = 8, class SYNC>
__device__ __forceinline__ void unpack_block(const PackJob &J, int b, Rr (*tile)[65], int warp, int lane, SYNC sync)
{
    const int m = b / J.nft;
    const int f0 = (b - m * J.nft) * 32;
    const int T = J.T, nfields = J.nfields, Cp = J.Cp;
    const long long nspec = J.nspec;
    const Rr *in = (const Rr *)J.src;
    Rr *spec = (Rr *)J.dst;
    const long long q0 = (long long)m * (T + 1) - (long long)m * (m - 1) / 2;
    const int len = T - m + 1;
    const long long rowE = J.srow[2 * m], rowO = J.srow[2 * m + 1];
    const bool zero = m > J.max_m;
    // one vector store per complex value where the caller's spectra allow it
    using V2 = std::conditional_t<std::is_same<Rr, double>::value, double2, float2>;
    const bool vec = (reinterpret_cast<uintptr_t>(spec) & (sizeof(V2) - 1)) == 0;
    for (int d0 = 0; d0 < len; d0 += 32 * CH) {
        // rows d = w, w+8, ... of each chunk; all loads in flight first
        constexpr int DK = 32 / NW;
        Rr v[CH][DK][2];
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < DK; ++k) {
                const int d = d0 + 32 * c + warp + NW * k;
                const long long row = ((d & 1) ? rowO : rowE) + (d >> 1);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int col = 2 * f0 + lane + 32 * h;
                    v[c][k][h] = 0;
                    if (!zero && d < len && col < 2 * nfields) v[c][k][h] = in[row * Cp + col];
                }
            }
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < DK; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) tile[32 * c + warp + NW * k][lane + 32 * h] = v[c][k][h];
        sync();
        for (int ff = warp; ff < 32; ff += NW) {
            const int fld = f0 + ff;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int d = d0 + 32 * c + lane;
                if (fld < nfields && d < len) {
                    Rr *a = spec + ((long long)fld * nspec + q0 + d) * 2;
                    const Rr re = tile[32 * c + lane][2 * ff];
                    const Rr im = m == 0 ? (Rr)0 : tile[32 * c + lane][2 * ff + 1];
                    if (vec) {
                        V2 z;
                        z.x = re;
                        z.y = im;
                        *reinterpret_cast<V2 *>(a) = z;
                    } else {
                        a[0] = re;
                        a[1] = im;
                    }
                }
            }
        }
        sync();
    }
}


}  // namespace st
