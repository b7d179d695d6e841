// Spectral pack / unpack bodies (legendre_simt.cu): one 256-thread block's
// work, shared by the per-stage kernels and the persistent batch kernel.
#pragma once

#include "st_internal.cuh"

#include <cuda_bf16.h>

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
template <typename Rr, int S, class SYNC>
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
    for (int d0 = 0; d0 < len; d0 += 32) {
        // load: warp w reads fields w, w+8, ...; lane = d
        for (int ff = warp; ff < 32; ff += 8) {
            int fld = f0 + ff, d = d0 + lane;
            Rr re = 0, im = 0;
            if (fld < nfields && d < len) {
                const Rr *a = spec + ((long long)fld * nspec + q0 + d) * 2;
                re = a[0];
                im = m == 0 ? (Rr)0 : a[1];
                if (J.scale) {
                    // inverse Laplacian on the unit sphere: -1 / (n (n+1)), 0 at n = 0
                    const int n = m + d;
                    const Rr f = n == 0 ? (Rr)0 : (Rr)(-1.0 / ((double)n * (n + 1.0)));
                    re *= f;
                    im *= f;
                }
            }
            tile[lane][2 * ff] = re;
            tile[lane][2 * ff + 1] = im;
        }
        sync();
        // store: warp w writes rows d = w, w+8, ...; lanes cover 64 columns
        for (int dd = warp; dd < 32; dd += 8) {
            int d = d0 + dd;
            if (d >= len) continue;
            long long row = ((d & 1) ? rowO : rowE) + (d >> 1);
            for (int cc = lane; cc < 64; cc += 32) {
                int c = 2 * f0 + cc;
                if (c < 2 * nfields) put_op<S, Rr>(out, op_index(S, row, c, Cp, Rp), ps, tile[dd][cc]);
            }
        }
        sync();
    }
}

// Operand rows (direct GEMM output, FP32/FP64) -> spectra.  Wavenumbers kept
// by no row (m > max_m) are written as zero; Im a_n^0 is written as zero.
template <typename Rr, class SYNC>
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
    for (int d0 = 0; d0 < len; d0 += 32) {
        for (int dd = warp; dd < 32; dd += 8) {
            int d = d0 + dd;
            long long row = ((d & 1) ? rowO : rowE) + (d >> 1);
            for (int cc = lane; cc < 64; cc += 32) {
                int c = 2 * f0 + cc;
                Rr v = 0;
                if (!zero && d < len && c < 2 * nfields) v = in[row * Cp + c];
                tile[dd][cc] = v;
            }
        }
        sync();
        for (int ff = warp; ff < 32; ff += 8) {
            int fld = f0 + ff, d = d0 + lane;
            if (fld < nfields && d < len) {
                Rr *a = spec + ((long long)fld * nspec + q0 + d) * 2;
                a[0] = tile[lane][2 * ff];
                a[1] = m == 0 ? (Rr)0 : tile[lane][2 * ff + 1];
            }
        }
        sync();
    }
}


}  // namespace st
