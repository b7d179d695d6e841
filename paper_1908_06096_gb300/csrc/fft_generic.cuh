// Generic ragged real FFTs along the latitude rows (device code; the
// instances live in fft_gen_*.cu, the job builder in fft.cu) (the Fourier stage of ESCAPE D3.3
// section 4.4.1; section 4.2.5 notes that batched library FFTs cannot mix row
// lengths and that a custom variable-size batched FFT would lift that limit:
// this is that FFT).
//
// One CTA takes one northern row j and its mirror row (same length N) for a
// group of G fields.  The two real rows of a field are packed as one complex
// sequence z = north + i south, so a single complex FFT of length N serves
// both.  Every transform runs in place in shared memory (one buffer per
// field) as mixed-radix passes over radices 2, 3, 4, 5; each pass fuses two
// radix stages in registers (a 16-point pass for 4 x 4), so a 3888-point FFT
// takes 4 trips through shared memory.  Roots of unity come from a two-level
// table in shared memory; chirps and kernel spectra are read through the
// read-only cache.  The plan stores the rows longest first and gives each
// run of rows its own number of fields per CTA (G).
//
//  mode 0 (N 5-smooth): decimation-in-frequency passes; the output sits in
//          digit-reversed order and is read through the index map pos(m).
//  mode 1 (Bluestein): the N-point DFT as a chirp-weighted circular
//          convolution of length L >= N + 2M (2M + 1 wavenumbers on one
//          side, N points on the other):
//              Z_m = w_m sum_k (z_k w_k) conj(w_{m-k}),  w_k = e^{-i pi k^2 / N}
//          done as DIF (natural -> digit-reversed), a pointwise product with
//          the kernel spectrum stored in that same digit-reversed order, and
//          DIT (digit-reversed -> natural), with IFFT(v) = conj(FFT(conj v))/L
//          (the 1/L is folded into the stored kernel).
//
// Direct stage: grid rows -> E = F(north) + F(south), O = F(north) - F(south)
// for m <= M_j, scaled by 1/N, written in the storage the direct Legendre
// GEMM reads.  Inverse stage: S, A -> F(north) = S + A, F(south) = S - A ->
// Hermitian spectra -> one complex inverse FFT -> both rows.
#pragma once

#include "st_internal.cuh"

#include <algorithm>

namespace st {

template <typename R> struct CT;
template <> struct CT<double> { typedef double2 T; };
template <> struct CT<float> { typedef float2 T; };

template <typename C> __device__ inline C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ inline C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ inline C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ inline C cconj(C a) { a.y = -a.y; return a; }
// multiply by -i
template <typename C> __device__ inline C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

// ------------------------------------------------------------------ R-point DFTs, W = e^{-2 pi i / R}

template <typename C> __device__ inline void dft2(C *v)
{
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <typename C> __device__ inline void dft4(C *v)
{
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
}

// W = c + i s, c = -1/2, s = -sqrt(3)/2
template <typename C> __device__ inline void dft3(C *v)
{
    typedef decltype(v[0].x) Rr;
    const Rr c = (Rr)-0.5, s = (Rr)-0.86602540378443864676;
    C t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    C a;
    a.x = v[0].x + c * t1.x;
    a.y = v[0].y + c * t1.y;
    C b;  // i s t2
    b.x = -s * t2.y;
    b.y = s * t2.x;
    v[0] = cadd(v[0], t1);
    v[1] = cadd(a, b);
    v[2] = csub(a, b);
}

// W^k = c_k + i s_k, c1 = cos(2pi/5), s1 = -sin(2pi/5), c2 = cos(4pi/5), s2 = -sin(4pi/5)
template <typename C> __device__ inline void dft5(C *v)
{
    typedef decltype(v[0].x) Rr;
    const Rr c1 = (Rr)0.30901699437494742410, s1 = (Rr)-0.95105651629515357212;
    const Rr c2 = (Rr)-0.80901699437494742410, s2 = (Rr)-0.58778525229247312917;
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    C v0 = v[0];
    C a1, a2, b1, b2;
    a1.x = v0.x + c1 * t1.x + c2 * t2.x;
    a1.y = v0.y + c1 * t1.y + c2 * t2.y;
    a2.x = v0.x + c2 * t1.x + c1 * t2.x;
    a2.y = v0.y + c2 * t1.y + c1 * t2.y;
    // b1 = i (s1 d1 + s2 d2), b2 = i (s2 d1 - s1 d2)
    Rr u1x = s1 * d1.x + s2 * d2.x, u1y = s1 * d1.y + s2 * d2.y;
    Rr u2x = s2 * d1.x - s1 * d2.x, u2y = s2 * d1.y - s1 * d2.y;
    b1.x = -u1y;
    b1.y = u1x;
    b2.x = -u2y;
    b2.y = u2x;
    v[0] = cadd(v0, cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <int R, typename C> __device__ inline void dftR(C *v)
{
    if (R == 2) dft2(v);
    if (R == 3) dft3(v);
    if (R == 4) dft4(v);
    if (R == 5) dft5(v);
}

// ------------------------------------------------------------------ in-place passes
//
// DIF stage of radix R on blocks of size Ns: for each block and n1 < Ns/R,
// the R elements n1 + r Ns/R go through an R-point DFT, output q is then
// multiplied by W_Ns^{n1 q}, and written back to the same R places.  The DIT
// stage is its transpose (twiddle first, then the DFT) and runs the stages in
// the opposite order.  A pass fuses two consecutive stages (Ra on blocks of
// Ns, then Rb on the sub-blocks of Ns/Ra) in registers.  tw holds
// e^{-2 pi i t / L}; W_Ns^t = tw[t L / Ns].  Each stage loads one base root
// and forms its powers by multiplication.  Element i of a field lives at
// shared-memory slot Swz(i).

template <int MODE>
struct Swz {
    __device__ int operator()(int i) const
    {
        if (MODE == 1) return i + (i >> 4);
        if (MODE == 2) return i + (i >> 5);
        if (MODE == 3) return i ^ ((i >> 4) & 15);
        return i;
    }
};

// n / d for 0 <= n < 2^22 without an integer divide: float reciprocal, then
// one correction step.
struct FastDiv {
    int d;
    float inv;
    __device__ explicit FastDiv(int d_) : d(d_), inv(1.0f / (float)d_) {}
    __device__ int operator()(int n) const
    {
        int q = __float2int_rz((float)n * inv);
        const int r = n - q * d;
        if (r >= d) ++q;
        else if (r < 0) --q;
        return q;
    }
};

// Roots of unity W_L^n of one row for the passes.  With a shared-memory
// table, W^n = T1[n / 128] T2[n % 128] (T1[a] = W^(128 a), T2[b] = W^b, both
// copied from the row's global table at CTA start; one extra rounding); rows
// longer than TW_SPLIT^2 read the global table.
constexpr int TW_SPLIT = 128;
template <typename C> struct Tw {
    const C *g;  // W_L^n, n < L (global)
    const C *s;  // T1 at s[0, 128), T2 at s[128, 256) (shared), or null
    __device__ inline C operator()(int n) const
    {
        if (s) return cmul(s[n >> 7], s[TW_SPLIT + (n & (TW_SPLIT - 1))]);
        return __ldg(&g[n]);
    }
};

template <typename C>
__device__ inline Tw<C> make_tw(const C *g, int L, C *sbuf)
{
    Tw<C> t;
    t.g = g;
    t.s = nullptr;
    if (L <= TW_SPLIT * TW_SPLIT) {
        for (int i = threadIdx.x; i < 2 * TW_SPLIT; i += blockDim.x) {
            const int n = i < TW_SPLIT ? i * TW_SPLIT : i - TW_SPLIT;
            if (n < L) sbuf[i] = __ldg(&g[n]);
        }
        t.s = sbuf;
    }
    return t;
}

// v[q] *= w^q, q = 1 .. R-1
template <int R, typename C> __device__ inline void twiddle_powers(C *v, C w)
{
    C p = w;
#pragma unroll
    for (int q = 1; q < R; ++q) {
        v[q] = cmul(v[q], p);
        if (q + 1 < R) p = cmul(p, w);
    }
}

template <int Ra, int Rb, bool DIT, typename C, class SW>
__device__ inline void pass2(C *x, const Tw<C> tw, int L, int S, int Ns, int G, SW sw,
                             const C *__restrict__ kern)
{
    const int ma = Ns / Ra, mb = ma / Rb;
    const int per = L / (Ra * Rb);
    const int sa = L / Ns, sb = L / ma;
    const C c = tw(mb * sa);  // e^{-2 pi i / (Ra Rb)}
    const FastDiv dper(per), dmb(mb);
    for (int idx = threadIdx.x; idx < G * per; idx += blockDim.x) {
        const int f = dper(idx), t = idx - f * per;
        const int b = dmb(t), n1 = t - b * mb;
        C *xf = x + (size_t)f * S;
        const int i0 = b * Ns + n1;
        C v[Ra][Rb];
#pragma unroll
        for (int ra = 0; ra < Ra; ++ra)
#pragma unroll
            for (int rb = 0; rb < Rb; ++rb) v[ra][rb] = xf[sw(i0 + ra * ma + rb * mb)];
        const C wa0 = tw(n1 * sa);
        const C wb = tw(n1 * sb);
        if (!DIT) {
            C wa = wa0;
#pragma unroll
            for (int rb = 0; rb < Rb; ++rb) {
                C u[Ra];
#pragma unroll
                for (int ra = 0; ra < Ra; ++ra) u[ra] = v[ra][rb];
                dftR<Ra>(u);
                twiddle_powers<Ra>(u, wa);
#pragma unroll
                for (int q = 0; q < Ra; ++q) v[q][rb] = u[q];
                if (rb + 1 < Rb) wa = cmul(wa, c);
            }
#pragma unroll
            for (int ra = 0; ra < Ra; ++ra) {
                dftR<Rb>(v[ra]);
                twiddle_powers<Rb>(v[ra], wb);
            }
        } else {
#pragma unroll
            for (int ra = 0; ra < Ra; ++ra) {
                twiddle_powers<Rb>(v[ra], wb);
                dftR<Rb>(v[ra]);
            }
            C wa = wa0;
#pragma unroll
            for (int rb = 0; rb < Rb; ++rb) {
                C u[Ra];
#pragma unroll
                for (int r = 0; r < Ra; ++r) u[r] = v[r][rb];
                twiddle_powers<Ra>(u, wa);
                dftR<Ra>(u);
#pragma unroll
                for (int q = 0; q < Ra; ++q) v[q][rb] = u[q];
                if (rb + 1 < Rb) wa = cmul(wa, c);
            }
        }
        if (kern) {
            // last DIF pass of a Bluestein row: times the kernel spectrum (kept in
            // this digit-reversed order), then conjugated for the second FFT
#pragma unroll
            for (int ra = 0; ra < Ra; ++ra)
#pragma unroll
                for (int rb = 0; rb < Rb; ++rb)
                    v[ra][rb] = cconj(cmul(v[ra][rb], __ldg(&kern[i0 + ra * ma + rb * mb])));
        }
#pragma unroll
        for (int ra = 0; ra < Ra; ++ra)
#pragma unroll
            for (int rb = 0; rb < Rb; ++rb) xf[sw(i0 + ra * ma + rb * mb)] = v[ra][rb];
    }
}

template <int R, bool DIT, typename C, class SW>
__device__ inline void pass1(C *x, const Tw<C> tw, int L, int S, int Ns, int G, SW sw,
                             const C *__restrict__ kern)
{
    const int m = Ns / R;
    const int per = L / R;
    const int sa = L / Ns;
    const FastDiv dper(per), dm(m);
    for (int idx = threadIdx.x; idx < G * per; idx += blockDim.x) {
        const int f = dper(idx), t = idx - f * per;
        const int b = dm(t), n1 = t - b * m;
        C *xf = x + (size_t)f * S;
        const int i0 = b * Ns + n1;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = xf[sw(i0 + r * m)];
        const C w = tw(n1 * sa);
        if (!DIT) {
            dftR<R>(v);
            twiddle_powers<R>(v, w);
        } else {
            twiddle_powers<R>(v, w);
            dftR<R>(v);
        }
        if (kern) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = cconj(cmul(v[r], __ldg(&kern[i0 + r * m])));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) xf[sw(i0 + r * m)] = v[r];
    }
}

template <bool DIT, typename C, class SW>
__device__ inline void run_pass2(int Ra, int Rb, C *x, const Tw<C> tw, int L, int S, int Ns, int G, SW sw,
                                 const C *kern)
{
#define ST_P2(A, B) \
    if (Ra == A && Rb == B) { pass2<A, B, DIT, C, SW>(x, tw, L, S, Ns, G, sw, kern); return; }
    ST_P2(4, 4) ST_P2(4, 3) ST_P2(3, 4) ST_P2(3, 3) ST_P2(4, 2) ST_P2(2, 4) ST_P2(3, 5) ST_P2(5, 3)
    ST_P2(2, 5) ST_P2(5, 2) ST_P2(2, 3) ST_P2(3, 2) ST_P2(2, 2)
#undef ST_P2
}

template <bool DIT, typename C, class SW>
__device__ inline void run_pass1(int R, C *x, const Tw<C> tw, int L, int S, int Ns, int G, SW sw, const C *kern)
{
    if (R == 2) pass1<2, DIT, C, SW>(x, tw, L, S, Ns, G, sw, kern);
    else if (R == 3) pass1<3, DIT, C, SW>(x, tw, L, S, Ns, G, sw, kern);
    else if (R == 4) pass1<4, DIT, C, SW>(x, tw, L, S, Ns, G, sw, kern);
    else pass1<5, DIT, C, SW>(x, tw, L, S, Ns, G, sw, kern);
}

// Stages are fused in pairs when the pair holds at most 16 points (the
// register budget); fusing or not does not change the result.
constexpr int MAX_FUSED = 16;
// Items per thread per round in the load and store loops (independent global
// loads in flight before the first use).
constexpr int FFT_U = 4;

// All DIF stages over rp.rad (natural -> digit-reversed).  With `kern`, the
// last pass also multiplies by the kernel spectrum and conjugates.
template <typename C, class SW>
__device__ void fft_dif(C *x, const Tw<C> tw, const RowPair &rp, int G, int S, const C *kern)
{
    const int L = rp.fftlen;
    const SW sw;
    int Ns = L;
    for (int q = 0; q < rp.nrad;) {
        if (q + 1 < rp.nrad && rp.rad[q] * rp.rad[q + 1] <= MAX_FUSED) {
            const bool last = q + 2 >= rp.nrad;
            run_pass2<false, C, SW>(rp.rad[q], rp.rad[q + 1], x, tw, L, S, Ns, G, sw, last ? kern : nullptr);
            Ns /= rp.rad[q] * rp.rad[q + 1];
            q += 2;
        } else {
            const bool last = q + 1 >= rp.nrad;
            run_pass1<false, C, SW>(rp.rad[q], x, tw, L, S, Ns, G, sw, last ? kern : nullptr);
            Ns /= rp.rad[q];
            q += 1;
        }
        __syncthreads();
    }
}

// All DIT stages (digit-reversed -> natural): the stages in reverse order.
template <typename C, class SW>
__device__ void fft_dit(C *x, const Tw<C> tw, const RowPair &rp, int G, int S)
{
    const int L = rp.fftlen;
    const SW sw;
    int Ns = 1;
    for (int q = rp.nrad - 1; q >= 0;) {
        if (q >= 1 && rp.rad[q - 1] * rp.rad[q] <= MAX_FUSED) {
            Ns *= rp.rad[q - 1] * rp.rad[q];
            run_pass2<true, C, SW>(rp.rad[q - 1], rp.rad[q], x, tw, L, S, Ns, G, sw, (const C *)nullptr);
            q -= 2;
        } else {
            Ns *= rp.rad[q];
            run_pass1<true, C, SW>(rp.rad[q], x, tw, L, S, Ns, G, sw, (const C *)nullptr);
            q -= 1;
        }
        __syncthreads();
    }
}

// Forward N-point DFT of each field's sequence, already in x (mode 0: natural
// order; mode 1: premultiplied by the chirp and zero up to L).  Afterwards
// fft_value(m) gives Z_m.
template <typename C, class SW>
__device__ inline void fft_forward(C *x, const Tw<C> tw, const C *__restrict__ kern, const RowPair &rp, int G, int S)
{
    fft_dif<C, SW>(x, tw, rp, G, S, rp.mode == 1 ? kern : nullptr);
    if (rp.mode == 1) fft_dit<C, SW>(x, tw, rp, G, S);
}

template <typename C, class SW>
__device__ inline C fft_value(const C *xf, const C *__restrict__ chirp, const RowPair &rp, int m)
{
    const SW sw;
    if (rp.mode == 0) return xf[sw(dif_pos(m, rp))];
    return cmul(__ldg(&chirp[m]), cconj(xf[sw(m)]));
}

// Z_{-m} (= Z_{N-m}), 1 <= m <= M.  Bluestein rows hold offset -m at L - m,
// and w_{-m} = w_m.
template <typename C, class SW>
__device__ inline C fft_value_neg(const C *xf, const C *__restrict__ chirp, const RowPair &rp, int m)
{
    const SW sw;
    if (rp.mode == 0) return xf[sw(dif_pos(rp.N - m, rp))];
    return cmul(__ldg(&chirp[m]), cconj(xf[sw(rp.fftlen - m)]));
}

__device__ inline float round_tf32_f(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Store one real value of the Fourier buffer in storage mode S.
template <int S, typename Rr>
__device__ inline void store_val(void *base, long long idx, long long plane_stride, Rr v)
{
    if (S == S_F64) {
        ((double *)base)[idx] = (double)v;
    } else if (S == S_F32) {
        ((float *)base)[idx] = (float)v;
    } else if (S == S_TF32_SPLIT) {
        float f = (float)v;
        float hi = round_tf32_f(f);
        float lo = round_tf32_f(f - hi);
        ((float *)base)[idx] = hi;
        ((float *)base)[idx + plane_stride] = lo;
    } else {
        float f = (float)v;
        __nv_bfloat16 hi = __float2bfloat16_rn(f);
        __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
        ((__nv_bfloat16 *)base)[idx] = hi;
        ((__nv_bfloat16 *)base)[idx + plane_stride] = lo;
    }
}

// Store the (re, im) pair of columns (c, c + 1) of row r; c is even, so
// row-major storage takes one 8-, 16- or (per plane) 4-byte store.
template <int S, typename Rr>
__device__ inline void store_pair(void *base, long long r, int c, int Cp, long long Rp, long long ps, Rr re, Rr im)
{
    const long long idx = op_index(S, r, c, Cp, Rp);
    if (S == S_F64) {
        *(double2 *)((double *)base + idx) = make_double2((double)re, (double)im);
    } else if (S == S_F32) {
        *(float2 *)((float *)base + idx) = make_float2((float)re, (float)im);
    } else if (S == S_BF16_SPLIT) {
        const float fr = (float)re, fi = (float)im;
        const __nv_bfloat162 hi = __floats2bfloat162_rn(fr, fi);
        const __nv_bfloat162 lo = __floats2bfloat162_rn(fr - __low2float(hi), fi - __high2float(hi));
        *(__nv_bfloat162 *)((__nv_bfloat16 *)base + idx) = hi;
        *(__nv_bfloat162 *)((__nv_bfloat16 *)base + idx + ps) = lo;
    } else {
        store_val<S, Rr>(base, idx, ps, re);
        store_val<S, Rr>(base, op_index(S, r, c + 1, Cp, Rp), ps, im);
    }
}

// FP32 grid rows whose north and south segments start at 16-byte boundaries
// and hold whole groups of 4 points (true of the octahedral rows 20 + 4i and
// of regular grids with nlon a multiple of 4): the grid side moves 4 points
// per access.
template <typename Rr>
__device__ inline bool grid_vec4(const void *grid, const RowPair &rp, long long npts)
{
    if (sizeof(Rr) != 4) return false;
    return ((rp.off_n | rp.off_s | npts | (long long)rp.N) & 3) == 0 && ((uintptr_t)grid & 15) == 0;
}

// Four consecutive values (two fields' re, im) of one row-major row starting
// at element idx, a multiple of 4: one 16-byte store (FP32) or one 8-byte
// store per plane (BF16 hi/lo).
template <int S, typename Rr>
__device__ inline void store_quad(void *base, long long idx, long long ps, const Rr *v)
{
    if (S == S_F32) {
        *(float4 *)((float *)base + idx) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    } else if (S == S_BF16_SPLIT) {
        __nv_bfloat162 hi[2], lo[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float a = (float)v[2 * h], b = (float)v[2 * h + 1];
            hi[h] = __floats2bfloat162_rn(a, b);
            lo[h] = __floats2bfloat162_rn(a - __low2float(hi[h]), b - __high2float(hi[h]));
        }
        uint2 uh, ul;
        uh.x = *(const unsigned *)&hi[0];
        uh.y = *(const unsigned *)&hi[1];
        ul.x = *(const unsigned *)&lo[0];
        ul.y = *(const unsigned *)&lo[1];
        *(uint2 *)((__nv_bfloat16 *)base + idx) = uh;
        *(uint2 *)((__nv_bfloat16 *)base + idx + ps) = ul;
    }
}

template <typename Rr, int MB> struct FftBounds { static constexpr int MINB = MB; };
template <int MB> struct FftBounds<double, MB> { static constexpr int MINB = 1; };

// The row's metadata is copied once per CTA into shared memory (a per-thread
// copy would live in local memory: the radix list is indexed at run time).
__device__ inline void load_rowpair(RowPair *dst, const RowPair *src)
{
    const int nw = (int)(sizeof(RowPair) / sizeof(int));
    for (int i = threadIdx.x; i < nw; i += blockDim.x) ((int *)dst)[i] = ((const int *)src)[i];
    __syncthreads();
}

// Storage mode chosen at run time (S_RT: the job's smode; FP32 kernels serve
// all three FP32 storage modes with one instance).
constexpr int S_RT = -1;
template <typename Rr>
__device__ inline void store_quad_rt(int sm, void *base, long long idx, long long ps, const Rr *v)
{
    if (sm == S_F32) store_quad<S_F32, Rr>(base, idx, ps, v);
    else if (sm == S_BF16_SPLIT) store_quad<S_BF16_SPLIT, Rr>(base, idx, ps, v);
}
template <typename Rr>
__device__ inline void store_pair_rt(int sm, void *base, long long r, int c, int Cp, long long Rp, long long ps, Rr re,
                                     Rr im)
{
    switch (sm) {
    case S_F64: store_pair<S_F64, Rr>(base, r, c, Cp, Rp, ps, re, im); break;
    case S_F32: store_pair<S_F32, Rr>(base, r, c, Cp, Rp, ps, re, im); break;
    case S_TF32_SPLIT: store_pair<S_TF32_SPLIT, Rr>(base, r, c, Cp, Rp, ps, re, im); break;
    default: store_pair<S_BF16_SPLIT, Rr>(base, r, c, Cp, Rp, ps, re, im); break;
    }
}

template <typename Rr, int S, class SW>
__device__ inline void fft_dir_body(const FftJob &J, const RowPair &rp, int j, int f0, void *tws)
{
    const int Sm = S >= 0 ? S : J.smode;
    typedef typename CT<Rr>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = J.G;
    const int N = rp.N, W = rp.fftlen, SL = J.Sslot;
    const int nfields = J.nfields, Cp = J.Cp, T = J.T, Jp = J.Jp;
    const long long npts = J.npts, Rp = J.Rp, plane_stride = J.ps;
    const Rr *grid = (const Rr *)J.src;
    void *fb = J.dst;
    C *x = (C *)smem_raw;
    const Tw<C> tw = make_tw<C>((const C *)J.tw + rp.tw_off, W, (C *)tws);
    const C *chirp = (const C *)J.chirp + rp.chirp_off;
    const SW sw;

    // FFT_U items per thread per round, all loads issued before any use
    const FastDiv dW(W);
    const int nt = blockDim.x;
    if (grid_vec4<Rr>(grid, rp, npts)) {
        // rows of 4-float multiples at 16-byte boundaries: 4 points per load
        const int W4 = W >> 2;
        const FastDiv dW4(W4);
        for (int base = threadIdx.x; base < G * W4; base += 2 * nt) {
            float4 vn[2], vs[2];
            C c[2][4];
            int f[2], k[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = base + u * nt;
                f[u] = dW4(idx);
                k[u] = 4 * (idx - f[u] * W4);
                vn[u] = vs[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    c[u][e].x = 1;
                    c[u][e].y = 0;
                }
                if (idx < G * W4 && f0 + f[u] < nfields && k[u] < N) {
                    const float *g = (const float *)grid + (long long)(f0 + f[u]) * npts;
                    vn[u] = __ldg((const float4 *)(g + rp.off_n + k[u]));
                    vs[u] = __ldg((const float4 *)(g + rp.off_s + k[u]));
                    if (rp.mode == 1) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) c[u][e] = __ldg(&chirp[k[u] + e]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (base + u * nt >= G * W4) break;
                const float re[4] = {vn[u].x, vn[u].y, vn[u].z, vn[u].w};
                const float im[4] = {vs[u].x, vs[u].y, vs[u].z, vs[u].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    C v;
                    v.x = re[e];
                    v.y = im[e];
                    x[f[u] * SL + sw(k[u] + e)] = rp.mode == 1 ? cmul(v, c[u][e]) : v;
                }
            }
        }
    } else
    for (int base = threadIdx.x; base < G * W; base += FFT_U * nt) {
        C v[FFT_U], c[FFT_U];
        int pos[FFT_U];
#pragma unroll
        for (int u = 0; u < FFT_U; ++u) {
            const int idx = base + u * nt;
            const int f = dW(idx), k = idx - f * W;
            const int fld = f0 + f;
            pos[u] = idx < G * W ? f * SL + sw(k) : -1;
            v[u].x = 0;
            v[u].y = 0;
            c[u].x = 1;
            c[u].y = 0;
            if (idx < G * W && fld < nfields && k < N) {
                const Rr *g = grid + (long long)fld * npts;
                v[u].x = g[rp.off_n + k];
                v[u].y = g[rp.off_s + k];
                if (rp.mode == 1) c[u] = __ldg(&chirp[k]);
            }
        }
#pragma unroll
        for (int u = 0; u < FFT_U; ++u)
            if (pos[u] >= 0) x[pos[u]] = rp.mode == 1 ? cmul(v[u], c[u]) : v[u];
    }
    __syncthreads();
    // slots past the last field hold zeros and need no transform
    fft_forward<C, SW>(x, tw, (const C *)J.kern + rp.kern_off, rp, min(G, nfields - f0), SL);

    const Rr inv = (Rr)1.0 / (Rr)N;
    const int M = rp.M;
    if ((Sm == S_BF16_SPLIT || Sm == S_F32) && (G & 1) == 0) {
        // two adjacent fields per item: their (re, im) columns are adjacent,
        // so E and O each take one 4-column store per plane; one chirp value
        // serves both fields and both signs of m (w_{-m} = w_m)
        const int G2 = G >> 1;
        const FastDiv dG2(G2);
        for (int idx = threadIdx.x; idx < (M + 1) * G2; idx += nt) {
            const int m = dG2(idx), f = 2 * (idx - m * G2);
            const int fld = f0 + f;
            if (fld >= nfields) continue;
            C cm;
            cm.x = 1;
            cm.y = 0;
            if (rp.mode == 1) cm = __ldg(&chirp[m]);
            Rr e4[4], o4[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const C *xf = x + (size_t)(f + h) * SL;
                C zm, zc;
                if (rp.mode == 1) {
                    zm = cmul(cm, cconj(xf[sw(m)]));
                    zc = m == 0 ? zm : cmul(cm, cconj(xf[sw(rp.fftlen - m)]));
                } else {
                    zm = xf[sw(dif_pos(m, rp))];
                    zc = m == 0 ? zm : xf[sw(dif_pos(N - m, rp))];
                }
                zc = cconj(zc);
                Rr ax = (zm.x + zc.x) * (Rr)0.5, ay = (zm.y + zc.y) * (Rr)0.5;
                Rr dx = (zm.x - zc.x) * (Rr)0.5, dy = (zm.y - zc.y) * (Rr)0.5;
                Rr bx = dy, by = -dx;
                Rr ex = (ax + bx) * inv, ey = (ay + by) * inv;
                Rr ox = (ax - bx) * inv, oy = (ay - by) * inv;
                if (m == 0) { ey = 0; oy = 0; }
                if (fld + h >= nfields) { ex = ey = ox = oy = 0; }  // padding columns stay zero
                e4[2 * h] = ex;
                e4[2 * h + 1] = ey;
                o4[2 * h] = ox;
                o4[2 * h + 1] = oy;
            }
            const long long rE = (long long)m * Jp + j, rO = ((long long)(T + 1) + m) * Jp + j;
            store_quad_rt<Rr>(Sm, fb, rE * Cp + 2 * fld, plane_stride, e4);
            store_quad_rt<Rr>(Sm, fb, rO * Cp + 2 * fld, plane_stride, o4);
        }
        return;
    }
    const FastDiv dG(G);
    for (int base = threadIdx.x; base < (M + 1) * G; base += FFT_U * nt) {
    C zmu[FFT_U], zcu[FFT_U];
#pragma unroll
    for (int u = 0; u < FFT_U; ++u) {
        const int idx = min(base + u * nt, (M + 1) * G - 1);
        const int m = dG(idx), f = idx - m * G;
        const C *xf = x + (size_t)f * SL;
        zmu[u] = fft_value<C, SW>(xf, chirp, rp, m);
        zcu[u] = m == 0 ? zmu[u] : fft_value_neg<C, SW>(xf, chirp, rp, m);
    }
#pragma unroll
    for (int u = 0; u < FFT_U; ++u) {
        const int idx = base + u * nt;
        if (idx >= (M + 1) * G) break;
        const int m = dG(idx), f = idx - m * G;
        const int fld = f0 + f;
        if (fld >= nfields) continue;
        const C zm = zmu[u];
        const C zc = cconj(zcu[u]);
        // north spectrum A = (zm + zc)/2, south spectrum B = -i (zm - zc)/2
        Rr ax = (zm.x + zc.x) * (Rr)0.5, ay = (zm.y + zc.y) * (Rr)0.5;
        Rr dx = (zm.x - zc.x) * (Rr)0.5, dy = (zm.y - zc.y) * (Rr)0.5;
        Rr bx = dy, by = -dx;
        Rr ex = (ax + bx) * inv, ey = (ay + by) * inv;
        Rr ox = (ax - bx) * inv, oy = (ay - by) * inv;
        if (m == 0) { ey = 0; oy = 0; }
        const long long rE = (long long)m * Jp + j, rO = ((long long)(T + 1) + m) * Jp + j;
        store_pair_rt<Rr>(Sm, fb, rE, 2 * fld, Cp, Rp, plane_stride, ex, ey);
        store_pair_rt<Rr>(Sm, fb, rO, 2 * fld, Cp, Rp, plane_stride, ox, oy);
    }
    }
}

template <typename Rr, int S, int MAXJ, int NT, int MB>
__global__ void __launch_bounds__(NT, (FftBounds<Rr, MB>::MINB)) k_fft_dir(const __grid_constant__ FftBatch<MAXJ> B)
{
    __shared__ RowPair rp;
    __shared__ __align__(16) typename CT<Rr>::T tws[2 * TW_SPLIT];
    const int q = find_job<MAXJ>(B.prefix, B.njobs, blockIdx.x);
    const FftJob &J = B.job[q];
    const int b = (int)(blockIdx.x - B.prefix[q]);
    const int rr = b / J.nfg;
    const int f0 = (b - rr * J.nfg) * J.G;
    load_rowpair(&rp, J.rps + J.r0 + rr);
    const int j = rp.j;
    switch (rp.swz) {
    case 1: fft_dir_body<Rr, S, Swz<1>>(J, rp, j, f0, tws); break;
    case 2: fft_dir_body<Rr, S, Swz<2>>(J, rp, j, f0, tws); break;
    case 3: fft_dir_body<Rr, S, Swz<3>>(J, rp, j, f0, tws); break;
    default: fft_dir_body<Rr, S, Swz<0>>(J, rp, j, f0, tws); break;
    }
}

template <typename Rr, class SW>
__device__ inline void fft_inv_body(const FftJob &J, const RowPair &rp, int j, int f0, void *tws)
{
    typedef typename CT<Rr>::T C;
    typedef typename CT<Rr>::T C2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = J.G;
    const int N = rp.N, S = J.Sslot;
    const int nfields = J.nfields, Cp = J.Cp, T = J.T, Jp = J.Jp;
    const long long npts = J.npts;
    const Rr *fb = (const Rr *)J.src;
    Rr *grid = (Rr *)J.dst;
    C *x = (C *)smem_raw;
    const Tw<C> tw = make_tw<C>((const C *)J.tw + rp.tw_off, rp.fftlen, (C *)tws);
    const C *chirp = (const C *)J.chirp + rp.chirp_off;
    const SW sw;

    for (int idx = threadIdx.x; idx < G * S; idx += blockDim.x) {
        C v;
        v.x = 0;
        v.y = 0;
        x[idx] = v;
    }
    __syncthreads();
    // conj(Z): Z[m] = Xn + i Xs, Z[N-m] = conj(Xn) + i conj(Xs), Z[0] = Re Xn + i Re Xs,
    // times the chirp at the same place for Bluestein rows
    const int M = rp.M;
    const int nt = blockDim.x;
    if (sizeof(Rr) == 4 && (G & 1) == 0) {
        // two adjacent fields per item: one 16-byte load each of S and A (the
        // column pair of an odd last field is padding, read but not used)
        const int G2 = G >> 1;
        const FastDiv dG2(G2);
        for (int base = threadIdx.x; base < (M + 1) * G2; base += 2 * nt) {
            float4 sv[2], av[2];
            C cw[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = base + u * nt;
                const int m = dG2(idx), fld = f0 + 2 * (idx - m * G2);
                sv[u] = av[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                cw[u].x = 1;
                cw[u].y = 0;
                if (idx < (M + 1) * G2 && fld < nfields) {
                    const long long rS = ((long long)m * Jp + j) * Cp + 2 * fld;
                    const long long rA = (((long long)(T + 1) + m) * Jp + j) * Cp + 2 * fld;
                    sv[u] = *(const float4 *)((const float *)fb + rS);
                    if (m < T || J.a_top) av[u] = *(const float4 *)((const float *)fb + rA);
                    if (rp.mode == 1) cw[u] = __ldg(&chirp[m]);  // w_{-m} = w_m
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = base + u * nt;
                if (idx >= (M + 1) * G2) break;
                const int m = dG2(idx), f = 2 * (idx - m * G2);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (f0 + f + h >= nfields) break;
                    const Rr sx = h ? sv[u].z : sv[u].x, sy = h ? sv[u].w : sv[u].y;
                    const Rr axx = h ? av[u].z : av[u].x, ayy = h ? av[u].w : av[u].y;
                    const Rr nx = sx + axx, ny = sy + ayy;  // north F_m
                    const Rr qx = sx - axx, qy = sy - ayy;  // south F_m
                    C *xf = x + (size_t)(f + h) * S;
                    if (m == 0) {
                        C v;
                        v.x = nx;
                        v.y = -qx;
                        if (rp.mode == 1) v = cmul(v, cw[u]);
                        xf[sw(0)] = v;
                    } else {
                        C a, bb;
                        a.x = nx - qy;
                        a.y = -(ny + qx);
                        bb.x = nx + qy;
                        bb.y = ny - qx;
                        if (rp.mode == 1) {
                            a = cmul(a, cw[u]);
                            bb = cmul(bb, cw[u]);
                        }
                        xf[sw(m)] = a;
                        xf[sw(rp.mode == 1 ? rp.fftlen - m : N - m)] = bb;
                    }
                }
            }
        }
    } else {
    const FastDiv dG(G);
    for (int base = threadIdx.x; base < (M + 1) * G; base += FFT_U * nt) {
        C2 sv[FFT_U], av[FFT_U];
        C ca[FFT_U], cb[FFT_U];
#pragma unroll
        for (int u = 0; u < FFT_U; ++u) {
            const int idx = base + u * nt;
            const int m = dG(idx), f = idx - m * G;
            const int fld = f0 + f;
            sv[u].x = sv[u].y = av[u].x = av[u].y = 0;
            ca[u].x = cb[u].x = 1;
            ca[u].y = cb[u].y = 0;
            if (idx < (M + 1) * G && fld < nfields) {
                const long long rS = ((long long)m * Jp + j) * Cp + 2 * fld;
                const long long rA = (((long long)(T + 1) + m) * Jp + j) * Cp + 2 * fld;
                sv[u] = *(const C2 *)(fb + rS);
                // the odd-parity half of m = T is empty (no n = T + 1), so its
                // rows are never written by the Legendre stage: A = 0 there
                if (m < T || J.a_top) av[u] = *(const C2 *)(fb + rA);
                if (rp.mode == 1) {
                    ca[u] = __ldg(&chirp[m]);  // w_{-m} = w_m
                    cb[u] = ca[u];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < FFT_U; ++u) {
            const int idx = base + u * nt;
            const int m = dG(idx), f = idx - m * G;
            if (idx >= (M + 1) * G || f0 + f >= nfields) continue;
            const Rr sx = sv[u].x, sy = sv[u].y, axx = av[u].x, ayy = av[u].y;
            const Rr nx = sx + axx, ny = sy + ayy;  // north F_m
            const Rr qx = sx - axx, qy = sy - ayy;  // south F_m
            C *xf = x + (size_t)f * S;
            if (m == 0) {
                C v;
                v.x = nx;
                v.y = -qx;
                if (rp.mode == 1) v = cmul(v, ca[u]);
                xf[sw(0)] = v;
            } else {
                C a, bb;
                a.x = nx - qy;
                a.y = -(ny + qx);
                bb.x = nx + qy;
                bb.y = ny - qx;
                if (rp.mode == 1) {
                    a = cmul(a, ca[u]);
                    bb = cmul(bb, cb[u]);
                }
                xf[sw(m)] = a;
                // wavenumber -m: at N - m for the N-point FFT, at L - m for Bluestein
                xf[sw(rp.mode == 1 ? rp.fftlen - m : N - m)] = bb;
            }
        }
    }
    }
    __syncthreads();
    const int Gv = min(G, nfields - f0);
    fft_forward<C, SW>(x, tw, (const C *)J.kern + rp.kern_off, rp, Gv, S);
    if (grid_vec4<Rr>(grid, rp, npts)) {
        const int N4 = N >> 2;
        const FastDiv dN4(N4);
        for (int idx = threadIdx.x; idx < Gv * N4; idx += nt) {
            const int f = dN4(idx), k = 4 * (idx - f * N4);
            const C *xf = x + (size_t)f * S;
            C v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = fft_value<C, SW>(xf, chirp, rp, k + e);
            float *g = (float *)grid + (long long)(f0 + f) * npts;
            *(float4 *)(g + rp.off_n + k) = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
            *(float4 *)(g + rp.off_s + k) = make_float4(-v[0].y, -v[1].y, -v[2].y, -v[3].y);
        }
        return;
    }
    const FastDiv dN(N);
    for (int base = threadIdx.x; base < Gv * N; base += FFT_U * nt) {
        C v[FFT_U];
#pragma unroll
        for (int u = 0; u < FFT_U; ++u) {
            const int idx = min(base + u * nt, Gv * N - 1);
            const int f = dN(idx), k = idx - f * N;
            v[u] = fft_value<C, SW>(x + (size_t)f * S, chirp, rp, k);
        }
#pragma unroll
        for (int u = 0; u < FFT_U; ++u) {
            const int idx = base + u * nt;
            if (idx >= Gv * N) break;
            const int f = dN(idx), k = idx - f * N;
            Rr *g = grid + (long long)(f0 + f) * npts;
            g[rp.off_n + k] = v[u].x;
            g[rp.off_s + k] = -v[u].y;
        }
    }
}

template <typename Rr, int MAXJ, int NT, int MB>
__global__ void __launch_bounds__(NT, (FftBounds<Rr, MB>::MINB)) k_fft_inv(const __grid_constant__ FftBatch<MAXJ> B)
{
    __shared__ RowPair rp;
    __shared__ __align__(16) typename CT<Rr>::T tws[2 * TW_SPLIT];
    const int q = find_job<MAXJ>(B.prefix, B.njobs, blockIdx.x);
    const FftJob &J = B.job[q];
    const int b = (int)(blockIdx.x - B.prefix[q]);
    const int rr = b / J.nfg;
    const int f0 = (b - rr * J.nfg) * J.G;
    load_rowpair(&rp, J.rps + J.r0 + rr);
    const int j = rp.j;
    switch (rp.swz) {
    case 1: fft_inv_body<Rr, Swz<1>>(J, rp, j, f0, tws); break;
    case 2: fft_inv_body<Rr, Swz<2>>(J, rp, j, f0, tws); break;
    case 3: fft_inv_body<Rr, Swz<3>>(J, rp, j, f0, tws); break;
    default: fft_inv_body<Rr, Swz<0>>(J, rp, j, f0, tws); break;
    }
}

template <typename K>
inline st_status set_smem(K kern, size_t smem)
{
    if (smem > 48 * 1024) ST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return ST_OK;
}

template <int MAXJ, class K>
inline st_status run_fft_batch(K kern, int threads, const FftJob *jobs, int n, size_t smem, cudaStream_t s)
{
    FftBatch<MAXJ> B;
    B.njobs = n;
    long long tot = 0;
    for (int q = 0; q < n; ++q) {
        B.prefix[q] = tot;
        B.job[q] = jobs[q];
        tot += (long long)jobs[q].J * jobs[q].nfg;
    }
    B.prefix[n] = tot;
    if (tot == 0) return ST_OK;
    if (tot > 0x7fffffffLL) return ST_ERR_UNSUPPORTED;
    st_status r = set_smem(kern, smem);
    if (r) return r;
    kern<<<(unsigned)tot, threads, smem, s>>>(B);
    ++kernel_launches();
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

}  // namespace st
