// FP32 row FFTs with compile-time radix plans (the Fourier stage of ESCAPE
// D3.3 section 4.4.1; the custom variable-size batched FFT that section 4.2.5
// names as the way past batched library FFTs of one length).
//
// Every FFT length L used here is R1 x R2 (x R3 (x R4)) with R1 in
// {2,3,4,5,6,8,10,12,16} and every later radix 16 (a few short plans excepted),
// at most 8192.  A plan is a type, so each pass is straight-line code with
// constant strides: a thread loads R elements, runs an R-point DFT in
// registers (composite radices as two small DFTs with constant twiddles), and
// stores them back.  Fields of one CTA live in shared memory at slot f * SL
// with one pad element per 16 (address e + e / 16): with the radix-16 passes
// last, every pass of these plans is free of bank conflicts.
//
// Two kinds of rows (both map the two rows of a Gaussian row pair onto one
// complex sequence z = north + i south, as the generic kernel does):
//  mode 0: N = L, one L-point FFT.
//  mode 1: Bluestein, L >= N + 2M: a DIF FFT, the product with the row's
//          kernel spectrum (stored in the DIF output order), and a DIT FFT.
//          The last DIF stage, the product and the first DIT stage act on the
//          same contiguous groups of R_P elements and run as one pass, so a
//          Bluestein row with P stages costs 2P - 1 passes.
// The outer passes read and write HBM straight from registers where the
// element order allows: the direct transform reads the grid rows in pass 1,
// the inverse writes them in its last pass.
#pragma once

#include "st_internal.cuh"

#include <type_traits>
#include <utility>

namespace st {
// FF_NS: the namespace of this instantiation (the persistent batch kernel
// compiles the same bodies at its own CTA width in a namespace of its own).
#ifndef FF_NS
#define FF_NS ff
#endif
#ifndef FF_NT
#define FF_NT 256
#endif
// Whole CTA or half CTA: a translation unit that runs the bodies in one half
// of a 512-thread CTA (the persistent batch kernel: two row-FFT items per SM
// at a time, as two 256-thread CTAs would) defines FF_HALVES; each half then
// has its own thread index, barrier and FF_HALF_BYTES of shared memory.
#ifdef FF_HALVES
#define FF_HALF (threadIdx.x >> 8)
#define FF_TID (threadIdx.x & 255)
#define FF_SYNC() asm volatile("bar.sync %0, 256;" ::"r"(4 + FF_HALF) : "memory")
#define FF_SMEM_OFF (FF_HALF * FF_HALF_BYTES)
#define FF_NHALF 2
#else
#define FF_HALF 0
#define FF_TID threadIdx.x
#define FF_SYNC() __syncthreads()
#define FF_SMEM_OFF 0
#define FF_NHALF 1
#endif
namespace FF_NS {

typedef float2 C;

#ifndef FF_MINB
#error "define FF_MINB (CTAs per SM the register budget is sized for)"
#endif
constexpr int NT = FF_NT;      // threads per CTA
constexpr int MINB = FF_MINB;  // CTAs per SM the register budget is sized for

__device__ __forceinline__ C cadd(C a, C b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ C csub(C a, C b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ C cmul(C a, C b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ C cconj(C a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ C cneg(C a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ C cmul_mi(C a) { return make_float2(a.y, -a.x); }   // times -i
__device__ __forceinline__ C cmul_pi(C a) { return make_float2(-a.y, a.x); }   // times +i

// ---- compile-time roots of unity W_R^K = e^{-2 pi i K / R}: Taylor series of
// cos and sin at the angle reduced to (-pi, pi], evaluated in double by the
// compiler and rounded once to float.
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double tcos(double x)
{
    double t = 1.0, s = 1.0;
    for (int i = 1; i <= 16; ++i) {
        t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        s += t;
    }
    return s;
}
constexpr double tsin(double x)
{
    double t = x, s = x;
    for (int i = 1; i <= 16; ++i) {
        t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        s += t;
    }
    return s;
}
constexpr double angle(int K, int R)
{
    int k = ((K % R) + R) % R;
    if (2 * k > R) k -= R;
    return 2.0 * kPi * (double)k / (double)R;
}
template <int K, int R>
struct Root {
    static constexpr float c = (float)tcos(angle(K, R));
    static constexpr float s = (float)-tsin(angle(K, R));
};

// v * W_R^K; multiples of an eighth turn use their exact forms.
template <int K, int R>
__device__ __forceinline__ C twc(C v)
{
    constexpr int k = ((K % R) + R) % R;
    constexpr float h = 0.70710678118654752440f;
    if constexpr (k == 0) return v;
    else if constexpr (4 * k == R) return cmul_mi(v);
    else if constexpr (2 * k == R) return cneg(v);
    else if constexpr (4 * k == 3 * R) return cmul_pi(v);
    else if constexpr (8 * k == R) return make_float2((v.x + v.y) * h, (v.y - v.x) * h);
    else if constexpr (8 * k == 3 * R) return make_float2((v.y - v.x) * h, -(v.x + v.y) * h);
    else if constexpr (8 * k == 5 * R) return make_float2(-(v.x + v.y) * h, (v.x - v.y) * h);
    else if constexpr (8 * k == 7 * R) return make_float2((v.x - v.y) * h, (v.x + v.y) * h);
    else {
        constexpr float c = Root<K, R>::c, s = Root<K, R>::s;
        return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
    }
}

// Compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1.
template <class F, int... I>
__device__ __forceinline__ void sfor_(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    sfor_(f, std::make_integer_sequence<int, N>{});
}

// ---- small forward DFTs in registers, X_k = sum_n x_n W_R^{n k}, in place.
__device__ __forceinline__ void dft2(C *v)
{
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
__device__ __forceinline__ void dft3(C *v)
{
    const float c = -0.5f, s = -0.86602540378443864676f;  // W_3 = c + i s
    const C t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    const C a = make_float2(v[0].x + c * t1.x, v[0].y + c * t1.y);
    const C b = make_float2(-s * t2.y, s * t2.x);  // i s t2
    v[0] = cadd(v[0], t1);
    v[1] = cadd(a, b);
    v[2] = csub(a, b);
}
__device__ __forceinline__ void dft4(C *v)
{
    const C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const C c = cadd(v[1], v[3]), d = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
}
__device__ __forceinline__ void dft5(C *v)
{
    // W_5^k = c_k + i s_k
    const float c1 = 0.30901699437494742410f, s1 = -0.95105651629515357212f;
    const float c2 = -0.80901699437494742410f, s2 = -0.58778525229247312917f;
    const C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const C d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    const C v0 = v[0];
    const C a1 = make_float2(v0.x + c1 * t1.x + c2 * t2.x, v0.y + c1 * t1.y + c2 * t2.y);
    const C a2 = make_float2(v0.x + c2 * t1.x + c1 * t2.x, v0.y + c2 * t1.y + c1 * t2.y);
    // b1 = i (s1 d1 + s2 d2), b2 = i (s2 d1 - s1 d2)
    const float u1x = s1 * d1.x + s2 * d2.x, u1y = s1 * d1.y + s2 * d2.y;
    const float u2x = s2 * d1.x - s1 * d2.x, u2y = s2 * d1.y - s1 * d2.y;
    const C b1 = make_float2(-u1y, u1x), b2 = make_float2(-u2y, u2x);
    v[0] = cadd(v0, cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <int R>
__device__ __forceinline__ void dft(C *v);

// R = RA RB as RA-point DFTs over n1 (n = RB n1 + n2), constant twiddles
// W_R^{n2 k1}, then RB-point DFTs over n2; X[k1 + RA k2] comes out of
// DFT k1's output k2.
template <int RA, int RB>
__device__ __forceinline__ void dft_ct(C *v)
{
    C y[RA][RB];
    sfor<RB>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        C u[RA];
        sfor<RA>([&](auto n1c) { u[decltype(n1c)::value] = v[RB * decltype(n1c)::value + n2]; });
        dft<RA>(u);
        sfor<RA>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            y[k1][n2] = twc<n2 * k1, RA * RB>(u[k1]);
        });
    });
    sfor<RA>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        dft<RB>(y[k1]);
        sfor<RB>([&](auto k2c) { v[k1 + RA * decltype(k2c)::value] = y[k1][decltype(k2c)::value]; });
    });
}

template <int R>
__device__ __forceinline__ void dft(C *v)
{
    if constexpr (R == 1) return;
    else if constexpr (R == 2) dft2(v);
    else if constexpr (R == 3) dft3(v);
    else if constexpr (R == 4) dft4(v);
    else if constexpr (R == 5) dft5(v);
    else if constexpr (R == 6) dft_ct<2, 3>(v);
    else if constexpr (R == 8) dft_ct<2, 4>(v);
    else if constexpr (R == 10) dft_ct<2, 5>(v);
    else if constexpr (R == 12) dft_ct<4, 3>(v);
    else if constexpr (R == 16) dft_ct<4, 4>(v);
    else static_assert(R == 2, "radix not provided");
}

// v[q] *= w^q, q = 1 .. R-1, with w^q = w^{4a} w^b (q = 4a + b): only w, w^2,
// w^3 and the current w^{4a} are live, and every power is at most five
// roundings deep.
template <int R>
__device__ __forceinline__ void twiddle_pow(C *v, C w)
{
    const C w2 = cmul(w, w);
    const C w3 = cmul(w2, w);
    if constexpr (R >= 2) v[1] = cmul(v[1], w);
    if constexpr (R >= 3) v[2] = cmul(v[2], w2);
    if constexpr (R >= 4) v[3] = cmul(v[3], w3);
    if constexpr (R > 4) {
        const C w4 = cmul(w2, w2);
        C wa = w4;
        sfor<(R + 3) / 4>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            if constexpr (a >= 1) {
                if constexpr (a == 2) wa = cmul(w4, w4);
                if constexpr (a == 3) wa = cmul(wa, w4);
                if constexpr (4 * a < R) v[4 * a] = cmul(v[4 * a], wa);
                if constexpr (4 * a + 1 < R) v[4 * a + 1] = cmul(v[4 * a + 1], cmul(wa, w));
                if constexpr (4 * a + 2 < R) v[4 * a + 2] = cmul(v[4 * a + 2], cmul(wa, w2));
                if constexpr (4 * a + 3 < R) v[4 * a + 3] = cmul(v[4 * a + 3], cmul(wa, w3));
            }
        });
    }
}

// ---- asynchronous global -> shared copies (no registers held, no waits
// that can spin: cp.async.wait_all blocks in hardware until the copies land)
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---- bulk copies (TMA engine) into shared memory, completion on an mbarrier.
// Every wait is bounded: past FF_WAIT_NS the CTA records bit 8 in the plan's
// error word, drains its copies (again bounded) and gives up the row.
constexpr unsigned long long FF_WAIT_NS = 2000000000ull;  // 2 s; a legitimate wait takes microseconds
constexpr int FF_ERR_WAIT = 8;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity)
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
// true once phase `parity` of the barrier completed; false when it did not
// within FF_WAIT_NS or another thread of the CTA gave up (*abort set)
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int *abort)
{
    if (bar_test(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    while (!bar_test(bar, parity)) {
        if (*abort) return false;
        if (gtime() - t0 > FF_WAIT_NS) {
            *abort = 1;
            return false;
        }
    }
    return true;
}
// One thread: set the barrier up for `bytes` of copies and arrive.
__device__ __forceinline__ void bar_init_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// ---- plans
template <int A, int B, int Cc = 1, int D = 1>
struct Plan {
    static constexpr int P = Cc > 1 ? (D > 1 ? 4 : 3) : 2;
    static constexpr int L = A * B * Cc * D;
    static constexpr int SL = L + (L >> 4) + 1;  // slot of one field (pad-16 layout, one spare)
    // every base root a stage needs is W_L^t with t < L / R1; up to 512 of
    // them are copied to shared memory per CTA (longer tables stay in L2)
    static constexpr int TWN = L / A;
    static constexpr bool TW_SMEM = TWN <= 512;
    template <int s>
    static constexpr int R()
    {
        return s == 1 ? A : (s == 2 ? B : (s == 3 ? Cc : D));
    }
    // block size a stage-s butterfly works in
    template <int s>
    static constexpr int NS()
    {
        return s == 1 ? L : (s == 2 ? L / A : (s == 3 ? L / (A * B) : L / (A * B * Cc)));
    }
};

__device__ __forceinline__ int sw(int e) { return e + (e >> 4); }

// Slot index of element e0 + q ST for q = 0 .. R-1 as base + q * step: the
// pad-16 map is linear along a stride that is a multiple of 16, and along
// stride 1 inside a block of R elements when R divides 16 and the block
// starts at a multiple of R.
template <int ST, int R>
struct Lin {
    static constexpr bool ok = (ST % 16 == 0) || (ST == 1 && 16 % R == 0);
    static constexpr int step = ST % 16 == 0 ? ST + ST / 16 : 1;
};
template <int ST, int R>
__device__ __forceinline__ int slot_of(int e0, int q)
{
    if constexpr (Lin<ST, R>::ok) return sw(e0) + q * Lin<ST, R>::step;
    else return sw(e0 + q * ST);
}

// Mixed-radix digit reversal of the plan: where frequency m sits after the
// DIF stages (m = d1 + R1 (d2 + R2 (...)), place = sum_s d_s NS_s / R_s).
template <class PL>
__device__ __forceinline__ int dif_place(int m)
{
    int pos = 0;
    sfor<PL::P>([&](auto sc) {
        constexpr int s = decltype(sc)::value + 1;
        constexpr int R = PL::template R<s>();
        constexpr int ST = PL::template NS<s>() / R;
        const int d = m % R;
        m /= R;
        pos += d * ST;
    });
    return pos;
}

// One in-place stage in shared memory on G fields.  DIF: R-point DFT, then
// output q times W_NS^{n1 q}; DIT: the transpose (twiddle first).  KERN: the
// last DIF stage fused with the Bluestein product and the first DIT stage.
template <class PL, int s, bool DIT, bool KERN = false>
__device__ __forceinline__ void stage(C *x, int G, const C *__restrict__ tw, const C *__restrict__ kern)
{
    constexpr int L = PL::L, R = PL::template R<s>(), NS = PL::template NS<s>();
    constexpr int ST = NS / R, NB = L / R, TWS = L / NS, SL = PL::SL;
    for (int i = FF_TID; i < G * NB; i += NT) {
        const int f = i / NB, u = i - f * NB;
        const int b = u / ST, n1 = u - b * ST;
        C *xf = x + f * SL;
        const int e0 = b * NS + n1;
        C v[R];
        C kq[KERN ? R : 1];
        if constexpr (KERN) {
            // value q of block b of the kernel spectrum sits at q NB + b
            // (consecutive threads, consecutive blocks: coalesced)
#pragma unroll
            for (int q = 0; q < R; ++q) kq[q] = __ldg(&kern[q * NB + b]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = xf[slot_of<ST, R>(e0, q)];
        if constexpr (KERN) {
            // ST == 1 here: no twiddles on either side of the product
            dft<R>(v);
#pragma unroll
            for (int q = 0; q < R; ++q) v[q] = cconj(cmul(v[q], kq[q]));
            dft<R>(v);
        } else if constexpr (ST == 1) {
            dft<R>(v);
        } else {
            const C w = tw[n1 * TWS];
            if constexpr (DIT) {
                twiddle_pow<R>(v, w);
                dft<R>(v);
            } else {
                dft<R>(v);
                twiddle_pow<R>(v, w);
            }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) xf[slot_of<ST, R>(e0, q)] = v[q];
    }
}

// Stages 2 .. P-1 of the DIF (a = 2) or, in reverse, of the DIT.
template <class PL, bool DIT>
__device__ __forceinline__ void middle_stages(C *x, int G, const C *tw)
{
    if constexpr (!DIT) {
        if constexpr (PL::P >= 3) { stage<PL, 2, false>(x, G, tw, nullptr); FF_SYNC(); }
        if constexpr (PL::P >= 4) { stage<PL, 3, false>(x, G, tw, nullptr); FF_SYNC(); }
    } else {
        if constexpr (PL::P >= 4) { stage<PL, 3, true>(x, G, tw, nullptr); FF_SYNC(); }
        if constexpr (PL::P >= 3) { stage<PL, 2, true>(x, G, tw, nullptr); FF_SYNC(); }
    }
}

// Stage 1 of the DIF reading its R1 inputs from `in(f, e)` (zero outside the
// row), writing shared memory.
template <class PL, class IN>
__device__ __forceinline__ void stage1_in(C *x, int G, const C *__restrict__ tw, IN in)
{
    constexpr int L = PL::L, R = PL::template R<1>(), ST = L / R, SL = PL::SL;
    for (int i = FF_TID; i < G * ST; i += NT) {
        const int f = i / ST, n = i - f * ST;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = in(f, n + q * ST, f * SL + slot_of<ST, R>(n, q));
        dft<R>(v);
        twiddle_pow<R>(v, tw[n]);
        C *xf = x + f * SL;
#pragma unroll
        for (int q = 0; q < R; ++q) xf[slot_of<ST, R>(n, q)] = v[q];
    }
}

// Element of field f's slot where its raw rows are staged: the slot start
// rounded up to an even element, so 16-byte aligned; the N + N floats end
// inside the slot because N + 1 <= SL.
__device__ __forceinline__ int raw_at(int f, int SL) { return (f * SL + 1) & ~1; }

// Stage 1 of the DIF on rows staged raw in shared memory: field f's north
// row (N floats) then south row sit at element raw_at(f, SL) of its own
// slot.  One item per thread per field (L / R1 <= NT); each field's raw
// values are read by every thread before any thread overwrites the slot.
// cz holds the thread's R1 chirp factors (ones on mode-0 rows), loaded once
// for all fields.
template <class PL>
__device__ __forceinline__ void stage1_raw(C *x, int G, const C *__restrict__ tw, int N, const C *cz,
                                           const C *__restrict__ chirp, bool blue)
{
    constexpr int L = PL::L, R = PL::template R<1>(), ST = L / R, SL = PL::SL;
    const int n = FF_TID;
    if constexpr (ST <= NT) {
        // one item per thread per field; cz holds the thread's R chirp
        // factors (ones on mode-0 rows), loaded once for all fields
        for (int f = 0; f < G; ++f) {
            const float *raw = (const float *)(x + raw_at(f, SL));
            C v[R];
            if (n < ST) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int e = n + q * ST;
                    v[q] = e < N ? cmul(cz[q], make_float2(raw[e], raw[N + e])) : make_float2(0.f, 0.f);
                }
            }
            FF_SYNC();
            if (n < ST) {
                dft<R>(v);
                twiddle_pow<R>(v, tw[n]);
                C *xf = x + f * SL;
#pragma unroll
                for (int q = 0; q < R; ++q) xf[slot_of<ST, R>(n, q)] = v[q];
            }
        }
    } else {
        // ST / NT items per thread per field, all read before the barrier;
        // the chirp factors are loaded per field, ahead of the reads
        static_assert(ST % NT == 0, "whole items per thread");
        constexpr int IT = ST / NT;
        for (int f = 0; f < G; ++f) {
            const float *raw = (const float *)(x + raw_at(f, SL));
            C v[IT][R];
#pragma unroll
            for (int i = 0; i < IT; ++i)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int e = n + i * NT + q * ST;
                    v[i][q] = make_float2(1.f, 0.f);
                    if (blue && e < N) v[i][q] = __ldg(&chirp[e]);
                }
#pragma unroll
            for (int i = 0; i < IT; ++i)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int e = n + i * NT + q * ST;
                    v[i][q] = e < N ? cmul(v[i][q], make_float2(raw[e], raw[N + e])) : make_float2(0.f, 0.f);
                }
            FF_SYNC();
            C *xf = x + f * SL;
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int ni = n + i * NT;
                dft<R>(v[i]);
                twiddle_pow<R>(v[i], tw[ni]);
#pragma unroll
                for (int q = 0; q < R; ++q) xf[slot_of<ST, R>(ni, q)] = v[i][q];
            }
        }
    }
}

// Stage 1 of the DIT (natural order out), handing output e of field f to
// out(f, e, value).
// pre(e) is read for every output before the pass's shared-memory loads (a
// global load issued early, so that its latency overlaps the arithmetic) and
// handed to out(f, e, slot index, value, pre(e)).
template <class PL, class PRE, class OUT>
__device__ __forceinline__ void stage1_out(C *x, int G, const C *__restrict__ tw, PRE pre, OUT out)
{
    constexpr int L = PL::L, R = PL::template R<1>(), ST = L / R, SL = PL::SL;
    for (int i = FF_TID; i < G * ST; i += NT) {
        const int f = i / ST, n = i - f * ST;
        C pv[R];
#pragma unroll
        for (int q = 0; q < R; ++q) pv[q] = pre(n + q * ST);
        const C *xf = x + f * SL;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = xf[slot_of<ST, R>(n, q)];
        twiddle_pow<R>(v, tw[n]);
        dft<R>(v);
#pragma unroll
        for (int q = 0; q < R; ++q) out(f, n + q * ST, f * SL + slot_of<ST, R>(n, q), v[q], pv[q]);
    }
}

__device__ __forceinline__ float round_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// E/O values of two adjacent fields (columns 2 fld .. 2 fld + 3) of Fourier-
// buffer row r in storage mode sm (FP32, split TF32 column-major, or split
// BF16 row-major); `two` false: one field only.
__device__ __forceinline__ void store_cols(void *base, int sm, long long r, int col, int Cp, long long Rp,
                                           long long ps, const float *v, bool two)
{
    if (sm == S_BF16_SPLIT) {
        __nv_bfloat162 hi[2], lo[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            hi[h] = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
            lo[h] = __floats2bfloat162_rn(v[2 * h] - __low2float(hi[h]), v[2 * h + 1] - __high2float(hi[h]));
        }
        __nv_bfloat16 *b = (__nv_bfloat16 *)base + r * Cp + col;
        if (two) {
            uint2 uh, ul;
            uh.x = *(const unsigned *)&hi[0];
            uh.y = *(const unsigned *)&hi[1];
            ul.x = *(const unsigned *)&lo[0];
            ul.y = *(const unsigned *)&lo[1];
            *(uint2 *)b = uh;
            *(uint2 *)(b + ps) = ul;
        } else {
            *(__nv_bfloat162 *)b = hi[0];
            *(__nv_bfloat162 *)(b + ps) = lo[0];
        }
    } else if (sm == S_F32) {
        float *b = (float *)base + r * Cp + col;
        if (two) *(float4 *)b = make_float4(v[0], v[1], v[2], v[3]);
        else *(float2 *)b = make_float2(v[0], v[1]);
    } else {
        // split TF32, column-major (element (r, c) at c Rp + r)
        float *b = (float *)base;
        const int nc = two ? 4 : 2;
        for (int k = 0; k < nc; ++k) {
            const float hi = round_tf32(v[k]), lo = round_tf32(v[k] - hi);
            b[(long long)(col + k) * Rp + r] = hi;
            b[(long long)(col + k) * Rp + r + ps] = lo;
        }
    }
}

// Start the asynchronous copy of a row's base roots W_L^t, t < L / R1, into
// shared memory (when the plan keeps them there).
template <class PL>
__device__ __forceinline__ void load_tables(C *tws, const C *twg)
{
    if constexpr (PL::TW_SMEM)
        for (int t = FF_TID; t < PL::TWN; t += NT) cp_async8(&tws[t], &twg[t]);
    cp_async_commit();
}

// ---------------------------------------------------------------- direct
//
// Grid rows -> E = F(north) + F(south), O = F(north) - F(south) for m <= M,
// scaled by 1/N, in the storage the direct Legendre GEMM reads.
template <class PL>
__device__ __noinline__ void dir_body(const FftJob &J, const RowPair &rp, int f0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *x = (C *)(smem_raw + FF_SMEM_OFF);
    constexpr int L = PL::L, SL = PL::SL;
    const int N = rp.N, M = rp.M;
    // fields of this CTA (the last CTA of a row may hold fewer than J.G)
    const int G = max(0, min(J.G, J.nfields - f0));
    const bool blue = rp.mode == 1;
    const C *twg = (const C *)J.tw + rp.tw_off;
    const C *chirp = (const C *)J.chirp + rp.chirp_off;
    const C *kern = (const C *)J.kern + rp.kern_off;
    // shared memory: J.G field slots, then the base roots, which arrive by
    // an asynchronous copy while stage 1 runs on the roots in L2
    C *tws = x + ((J.G * SL + 1) & ~1);
    const C *tw = twg;
    if constexpr (PL::TW_SMEM) tw = tws;
    if (G > 0) load_tables<PL>(tws, twg);
    const float *grid = (const float *)J.src + (long long)f0 * J.npts;
    const long long npts = J.npts;
    const long long on = rp.off_n, os = rp.off_s;

    // Rows whose offsets, length and field stride are multiples of four
    // floats arrive by bulk copies into the fields' slots (one per row and
    // field, tracked by one barrier) instead of per-thread loads.
    constexpr int kST1 = PL::L / PL::template R<1>();
    constexpr bool kRawFits = kST1 <= NT || kST1 % NT == 0;
    const bool raw = kRawFits && G > 0 && ((on | os | (long long)N | npts) & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(J.src) & 15) == 0 && (smem_addr(x) & 15) == 0;
    if (raw) {
        __shared__ __align__(8) unsigned long long rbar_[FF_NHALF];
        __shared__ int abort_[FF_NHALF];
        unsigned long long &rbar = rbar_[FF_HALF];
        int &abort_raw = abort_[FF_HALF];
        const uint32_t bar = smem_addr(&rbar);
        if (FF_TID == 0) {
            abort_raw = 0;
            bar_init_expect(bar, (uint32_t)(G * 8 * N));
            for (int f = 0; f < G; ++f) {
                float *d = (float *)(x + raw_at(f, SL));
                bulk_copy(d, grid + f * npts + on, 4u * N, bar);
                bulk_copy(d + N, grid + f * npts + os, 4u * N, bar);
            }
        }
        FF_SYNC();
        // the chirp factors of this thread's stage-1 elements, loaded while
        // the rows are in flight
        constexpr int R1 = PL::template R<1>(), ST1 = PL::L / R1;
        C cz[R1];
#pragma unroll
        for (int q = 0; q < R1; ++q) {
            const int e = FF_TID + q * ST1;
            cz[q] = make_float2(1.f, 0.f);
            if (ST1 <= NT && blue && FF_TID < ST1 && e < N) cz[q] = __ldg(&chirp[e]);
        }
        cp_async_wait_all();
        bar_wait(bar, 0, &abort_raw);
        FF_SYNC();
        // every thread has seen the phase complete: the barrier may be
        // retired (a persistent CTA sets it up again for its next row)
        if (FF_TID == 0 && !abort_raw) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
        if (abort_raw) {
            // give the copies in flight a bounded chance to land before the
            // shared memory is released
            if (FF_TID == 0) {
                atomicOr(J.err, FF_ERR_WAIT);
                const unsigned long long t0 = gtime();
                while (!bar_test(bar, 0) && gtime() - t0 < FF_WAIT_NS) {
                }
            }
            return;
        }
        if constexpr (kRawFits) stage1_raw<PL>(x, G, tw, N, cz, chirp, blue);
    } else {
        stage1_in<PL>(x, G, twg, [&](int f, int e, int) -> C {
            C z = make_float2(0.f, 0.f);
            if (e < N) {
                const float *g = grid + f * npts;
                z = make_float2(__ldg(g + on + e), __ldg(g + os + e));
                if (blue) z = cmul(z, __ldg(&chirp[e]));
            }
            return z;
        });
    }
    cp_async_wait_all();
    FF_SYNC();
    middle_stages<PL, false>(x, G, tw);
    constexpr int P = PL::P;
    if (blue) {
        stage<PL, P, false, true>(x, G, tw, kern);
        FF_SYNC();
        middle_stages<PL, true>(x, G, tw);
        // y at natural places; keep 0 .. M and L - M .. L - 1
        stage1_out<PL>(
            x, G, tw, [](int) { return make_float2(0.f, 0.f); },
            [&](int, int e, int si, C v, C) {
                if (e <= M || e >= L - M) x[si] = v;
            });
    } else {
        stage<PL, P, false>(x, G, tw, nullptr);
    }
    FF_SYNC();

    // Z_m and Z_{-m}; north spectrum (Z_m + conj Z_{-m}) / 2, south
    // -i (Z_m - conj Z_{-m}) / 2; E, O their sum and difference over N.
    const float inv = 1.0f / (float)N;
    const int G2 = (G + 1) >> 1;
    const int Cp = J.Cp, Jp = J.Jp, T = J.T, j = rp.j;
    // job fields in registers: after a global store the compiler would
    // otherwise have to read them again from the parameter block
    void *const dst = J.dst;
    const int smode = J.smode;
    const long long Rp = J.Rp, ps = J.ps;
    // four items per thread per round, their chirp loads issued first
    const int nitems = (M + 1) * G2;
    for (int base = FF_TID; base < nitems; base += 4 * NT) {
    C cmu[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int idx = base + u * NT;
        cmu[u] = make_float2(1.f, 0.f);
        if (blue && idx < nitems) cmu[u] = __ldg(&chirp[idx / G2]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int idx = base + u * NT;
        if (idx >= nitems) break;
        const int m = idx / G2, f = 2 * (idx - m * G2);
        const bool two = f + 1 < G;
        const C cm = cmu[u];
        float e4[4] = {0.f, 0.f, 0.f, 0.f}, o4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;  // no slot beyond the CTA's last field
            const C *xf = x + (f + h) * SL;
            C zm, zc;
            if (blue) {
                zm = cmul(cm, cconj(xf[sw(m)]));
                zc = m == 0 ? zm : cmul(cm, cconj(xf[sw(L - m)]));
            } else {
                zm = xf[sw(dif_place<PL>(m))];
                zc = m == 0 ? zm : xf[sw(dif_place<PL>(N - m))];
            }
            zc = cconj(zc);
            const float ax = (zm.x + zc.x) * 0.5f, ay = (zm.y + zc.y) * 0.5f;
            const float dx = (zm.x - zc.x) * 0.5f, dy = (zm.y - zc.y) * 0.5f;
            const float bx = dy, by = -dx;
            float ex = (ax + bx) * inv, ey = (ay + by) * inv;
            float ox = (ax - bx) * inv, oy = (ay - by) * inv;
            if (m == 0) ey = oy = 0.f;
            e4[2 * h] = ex;
            e4[2 * h + 1] = ey;
            o4[2 * h] = ox;
            o4[2 * h + 1] = oy;
        }
        const long long rE = (long long)m * Jp + j, rO = ((long long)(T + 1) + m) * Jp + j;
        const int col = 2 * (f0 + f);
        store_cols(dst, smode, rE, col, Cp, Rp, ps, e4, two);
        store_cols(dst, smode, rO, col, Cp, Rp, ps, o4, two);
    }
    }
}

// ---------------------------------------------------------------- inverse
//
// S, A -> F(north) = S + A, F(south) = S - A -> one complex FFT of
// conj(Z) (Z = north + i south spectrum, Hermitian halves folded) -> rows.
template <class PL>
__device__ __noinline__ void inv_body(const FftJob &J, const RowPair &rp, int f0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *x = (C *)(smem_raw + FF_SMEM_OFF);
    constexpr int L = PL::L, SL = PL::SL;
    const int N = rp.N, M = rp.M;
    const int G = max(0, min(J.G, J.nfields - f0));
    const bool blue = rp.mode == 1;
    const C *twg = (const C *)J.tw + rp.tw_off;
    const C *chirp = (const C *)J.chirp + rp.chirp_off;
    const C *kern = (const C *)J.kern + rp.kern_off;
    // shared memory as in dir_body; the roots arrive during the staging
    C *tws = x + ((J.G * SL + 1) & ~1);
    const C *tw = twg;
    if constexpr (PL::TW_SMEM) tw = tws;
    if (G > 0) load_tables<PL>(tws, twg);
    const float *fb = (const float *)J.src;
    const int Cp = J.Cp, Jp = J.Jp, T = J.T, j = rp.j;


    // staging: Bluestein rows keep the inputs at their natural places (0 .. M
    // and L - M .. L - 1, the rest is zero by index in stage 1); mode-0 rows
    // run DIT passes only, so every place 0 .. N - 1 is written, in the
    // digit-reversed order.
    const int G2 = (G + 1) >> 1;
    const int mtop = blue ? M : N / 2;
    // four items per thread per round: every global load of the round is
    // issued before the first is used
    const int nitems = (mtop + 1) * G2;
    for (int base = FF_TID; base < nitems; base += 4 * NT) {
        float4 sv[4], av[4];
        C cw[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = base + u * NT;
            const int m = idx / G2, f = 2 * (idx - m * G2);
            sv[u] = av[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            cw[u] = make_float2(1.f, 0.f);
            if (idx < nitems && m <= M) {
                const bool two = f + 1 < G;
                const long long rS = ((long long)m * Jp + j) * Cp + 2 * (f0 + f);
                const long long rA = (((long long)(T + 1) + m) * Jp + j) * Cp + 2 * (f0 + f);
                // two fields: 16-byte loads (f0 + f is even then); one: 8 bytes.
                // The odd-parity half of m = T is empty (no n = T + 1): A = 0 there.
                if (two) {
                    sv[u] = *(const float4 *)(fb + rS);
                    if (m < T || J.a_top) av[u] = *(const float4 *)(fb + rA);
                } else {
                    const float2 s2 = *(const float2 *)(fb + rS);
                    sv[u].x = s2.x;
                    sv[u].y = s2.y;
                    if (m < T || J.a_top) {
                        const float2 a2 = *(const float2 *)(fb + rA);
                        av[u].x = a2.x;
                        av[u].y = a2.y;
                    }
                }
                if (blue) cw[u] = __ldg(&chirp[m]);  // w_{-m} = w_m
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = base + u * NT;
            if (idx >= nitems) break;
            const int m = idx / G2, f = 2 * (idx - m * G2);
            const bool two = f + 1 < G;
            const int pa = blue ? m : dif_place<PL>(m);
            const int pb = blue ? L - m : dif_place<PL>(N - m);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && !two) break;
                const float sx = h ? sv[u].z : sv[u].x, sy = h ? sv[u].w : sv[u].y;
                const float ax = h ? av[u].z : av[u].x, ay = h ? av[u].w : av[u].y;
                const float nx = sx + ax, ny = sy + ay;  // north F_m
                const float qx = sx - ax, qy = sy - ay;  // south F_m
                C *xf = x + (f + h) * SL;
                if (m == 0) {
                    C v = make_float2(nx, -qx);
                    if (blue) v = cmul(v, cw[u]);
                    xf[sw(pa)] = v;
                } else {
                    C a = make_float2(nx - qy, -(ny + qx));
                    C bb = make_float2(nx + qy, ny - qx);
                    if (blue) {
                        a = cmul(a, cw[u]);
                        bb = cmul(bb, cw[u]);
                    }
                    xf[sw(pa)] = a;
                    // m = N / 2 (zero beyond M) maps to one place on mode-0 rows
                    if (!(pa == pb)) xf[sw(pb)] = bb;
                }
            }
        }
    }
    cp_async_wait_all();
    FF_SYNC();

    constexpr int P = PL::P;
    if (blue) {
        stage1_in<PL>(x, G, tw, [&](int, int e, int si) -> C {
            C z = make_float2(0.f, 0.f);
            if (e <= M || e >= L - M) z = x[si];
            return z;
        });
        // stage 1 reads and writes only its own butterfly's places, so it can
        // run in place; every place is written (zeros where the input was zero)
        FF_SYNC();
        middle_stages<PL, false>(x, G, tw);
        stage<PL, P, false, true>(x, G, tw, kern);
        FF_SYNC();
    } else {
        stage<PL, P, true>(x, G, tw, nullptr);
        FF_SYNC();
    }
    middle_stages<PL, true>(x, G, tw);
    float *grid = (float *)J.dst + (long long)f0 * J.npts;
    const long long npts = J.npts, on = rp.off_n, os = rp.off_s;
    stage1_out<PL>(
        x, G, tw,
        [&](int e) {
            C w = make_float2(1.f, 0.f);
            if (blue && e < N) w = __ldg(&chirp[e]);
            return w;
        },
        [&](int f, int e, int, C v, C w) {
            if (e < N) {
                if (blue) v = cmul(w, cconj(v));
                float *g = grid + f * npts;
                g[on + e] = v.x;
                g[os + e] = -v.y;
            }
        });
}

}  // namespace FF_NS
}  // namespace st
