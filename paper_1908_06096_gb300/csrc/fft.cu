// Ragged real FFTs along the latitude rows (the Fourier stage of ESCAPE D3.3
// section 4.4.1; section 4.2.5 notes that batched library FFTs cannot mix row
// lengths and that a custom variable-size batched FFT would lift that limit:
// this is that FFT).
//
// One CTA takes one northern row j and its mirror row (same length N) for a
// group of G fields.  The two real rows of a field are packed as one complex
// sequence z = north + i south, so a single complex FFT of length N serves
// both.  The transform runs as Stockham autosort passes in shared memory, one
// pass per prime-power factor: radix 2, 3, 4 and 5 butterflies are written
// out; any other prime factor is evaluated as a direct DFT over that factor
// (one output per thread).
//
// Direct stage: grid rows -> E = F(north) + F(south), O = F(north) - F(south)
// for m <= M_j, scaled by 1/N, written in the storage the direct Legendre
// GEMM reads.  Inverse stage: S, A -> F(north) = S + A, F(south) = S - A ->
// Hermitian spectra -> one complex inverse FFT -> both rows.
#include "st_internal.cuh"

#include <algorithm>

namespace st {

constexpr int FFT_THREADS = 512;

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
// multiply by -i
template <typename C> __device__ inline C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

// Radix-R butterfly on v[0..R-1] with W = e^{-2 pi i / R}.
template <int R, typename C> __device__ inline void dft_small(C *v);

template <> __device__ inline void dft_small<2, double2>(double2 *v)
{
    double2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <> __device__ inline void dft_small<2, float2>(float2 *v)
{
    float2 a = v[0], b = v[1];
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

// W = c + i s with c = -1/2, s = -sqrt(3)/2
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

// One Stockham pass of radix R (2, 3, 4 or 5) over G sequences of length N in
// shared memory: src -> dst, L = product of the radices of earlier passes.
template <int R, typename C>
__device__ inline void pass_small(const C *src, C *dst, const C *tw, int N, int S, int L, int G)
{
    int nb = N / R;
    int step = N / (L * R);
    for (int idx = threadIdx.x; idx < G * nb; idx += blockDim.x) {
        int f = idx / nb, b = idx - f * nb;
        int k = b % L, grp = b / L;
        const C *s = src + (size_t)f * S;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[b + r * nb];
        if (k) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * k * step]);
        }
        if (R == 2) dft_small<2, C>(v);
        if (R == 3) dft3(v);
        if (R == 4) dft4(v);
        if (R == 5) dft5(v);
        C *d = dst + (size_t)f * S + (size_t)grp * L * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[r * L] = v[r];
    }
}

// Stockham pass of any radix R as a direct DFT over the factor, one output
// per thread: out[grp L R + s L + k] = sum_r src[b + r N/R] W_N^{r (k + s L) N/(L R)}.
template <typename C>
__device__ inline void pass_generic(const C *src, C *dst, const C *tw, int N, int S, int L, int R, int G)
{
    int nb = N / R;
    int step = N / (L * R);
    for (int idx = threadIdx.x; idx < G * N; idx += blockDim.x) {
        int f = idx / N, o = idx - f * N;
        int k = o % L;
        int s_ = (o / L) % R;
        int grp = o / (L * R);
        int b = grp * L + k;
        const C *s = src + (size_t)f * S;
        int e = (k + s_ * L) * step;  // < N
        int ex = 0;
        C acc;
        acc.x = 0;
        acc.y = 0;
        for (int r = 0; r < R; ++r) {
            C x = s[b + r * nb];
            C t = tw[ex];
            acc.x += x.x * t.x - x.y * t.y;
            acc.y += x.x * t.y + x.y * t.x;
            ex += e;
            if (ex >= N) ex -= N;
        }
        dst[(size_t)f * S + o] = acc;
    }
}

// Runs all passes of length n = rp.fftlen over G sequences spaced S apart;
// returns the buffer that holds the result.
template <typename C>
__device__ C *fft_passes(C *x, C *y, const C *tw, const RowPair &rp, int G, int S)
{
    int L = 1;
    const int n = rp.fftlen;
    for (int q = 0; q < rp.nrad; ++q) {
        int R = rp.rad[q];
        switch (R) {
        case 2: pass_small<2, C>(x, y, tw, n, S, L, G); break;
        case 3: pass_small<3, C>(x, y, tw, n, S, L, G); break;
        case 4: pass_small<4, C>(x, y, tw, n, S, L, G); break;
        case 5: pass_small<5, C>(x, y, tw, n, S, L, G); break;
        default: pass_generic<C>(x, y, tw, n, S, L, R, G); break;
        }
        __syncthreads();
        C *t = x;
        x = y;
        y = t;
        L *= R;
    }
    return x;
}

// Forward N-point DFT of the G sequences in x (each in the first N slots of
// a stride-S slot); returns the buffer holding Z_0 .. Z_{N-1} per field.
// Mode 1 (Bluestein): Z_m = w_m conj(FFT_L(conj(FFT_L(z w) * kern)))_m with
// kern = FFT_L(b) / L, which is the circular convolution with b written
// through the conjugation identity IFFT(v) = conj(FFT(conj(v))) / L.
template <typename C>
__device__ C *fft_forward(C *x, C *y, const C *tw, const C *chirp, const C *__restrict__ kern, const RowPair &rp,
                          int G, int S)
{
    if (rp.mode == 0) return fft_passes<C>(x, y, tw, rp, G, S);
    const int N = rp.N, L = rp.fftlen;
    for (int idx = threadIdx.x; idx < G * L; idx += blockDim.x) {
        int f = idx / L, k = idx - f * L;
        C *v = x + (size_t)f * S + k;
        if (k < N) {
            *v = cmul(*v, chirp[k]);
        } else {
            C z;
            z.x = 0;
            z.y = 0;
            *v = z;
        }
    }
    __syncthreads();
    C *a = fft_passes<C>(x, y, tw, rp, G, S);
    C *other = a == x ? y : x;
    for (int idx = threadIdx.x; idx < G * L; idx += blockDim.x) {
        int f = idx / L, k = idx - f * L;
        C *v = a + (size_t)f * S + k;
        C t = cmul(*v, kern[k]);
        t.y = -t.y;
        *v = t;
    }
    __syncthreads();
    C *q = fft_passes<C>(a, other, tw, rp, G, S);
    for (int idx = threadIdx.x; idx < G * N; idx += blockDim.x) {
        int f = idx / N, m = idx - f * N;
        C *v = q + (size_t)f * S + m;
        C t = *v;
        t.y = -t.y;
        *v = cmul(chirp[m], t);
    }
    __syncthreads();
    return q;
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

template <typename Rr, int S>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_dir(const RowPair *__restrict__ rps,
                                                         const typename CT<Rr>::T *__restrict__ tw_all,
                                                         const typename CT<Rr>::T *__restrict__ chirp_all,
                                                         const typename CT<Rr>::T *__restrict__ kern_all,
                                                         const Rr *__restrict__ grid, long long npts, int nfields, int G,
                                                         void *fb, int Cp, long long Rp, long long plane_stride, int T,
                                                         int Jp)
{
    typedef typename CT<Rr>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int j = blockIdx.y;
    const RowPair rp = rps[j];
    const int N = rp.N, W = rp.fftlen;
    C *tw = (C *)smem_raw;
    C *ch = tw + W;
    C *x = ch + (rp.mode ? N : 0);
    C *y = x + (size_t)G * W;
    const int f0 = blockIdx.x * G;

    for (int t = threadIdx.x; t < W; t += blockDim.x) tw[t] = tw_all[rp.tw_off + t];
    if (rp.mode)
        for (int t = threadIdx.x; t < N; t += blockDim.x) ch[t] = chirp_all[rp.chirp_off + t];
    for (int idx = threadIdx.x; idx < G * N; idx += blockDim.x) {
        int f = idx / N, k = idx - f * N;
        int fld = f0 + f;
        C v;
        v.x = 0;
        v.y = 0;
        if (fld < nfields) {
            const Rr *g = grid + (long long)fld * npts;
            v.x = g[rp.off_n + k];
            v.y = g[rp.off_s + k];
        }
        x[(size_t)f * W + k] = v;
    }
    __syncthreads();
    C *z = fft_forward<C>(x, y, tw, ch, kern_all + rp.kern_off, rp, G, W);

    const Rr inv = (Rr)1.0 / (Rr)N;
    const int M = rp.M;
    for (int idx = threadIdx.x; idx < (M + 1) * G; idx += blockDim.x) {
        int m = idx / G, f = idx - m * G;
        int fld = f0 + f;
        if (fld >= nfields) continue;
        const C *zf = z + (size_t)f * W;
        C zm = zf[m];
        C zc = zf[m == 0 ? 0 : N - m];
        zc.y = -zc.y;
        // north spectrum A = (zm + zc)/2, south spectrum B = -i (zm - zc)/2
        Rr ax = (zm.x + zc.x) * (Rr)0.5, ay = (zm.y + zc.y) * (Rr)0.5;
        Rr dx = (zm.x - zc.x) * (Rr)0.5, dy = (zm.y - zc.y) * (Rr)0.5;
        Rr bx = dy, by = -dx;
        Rr ex = (ax + bx) * inv, ey = (ay + by) * inv;
        Rr ox = (ax - bx) * inv, oy = (ay - by) * inv;
        if (m == 0) { ey = 0; oy = 0; }
        const long long rE = (long long)m * Jp + j, rO = ((long long)(T + 1) + m) * Jp + j;
        store_val<S, Rr>(fb, op_index(S, rE, 2 * fld, Cp, Rp), plane_stride, ex);
        store_val<S, Rr>(fb, op_index(S, rE, 2 * fld + 1, Cp, Rp), plane_stride, ey);
        store_val<S, Rr>(fb, op_index(S, rO, 2 * fld, Cp, Rp), plane_stride, ox);
        store_val<S, Rr>(fb, op_index(S, rO, 2 * fld + 1, Cp, Rp), plane_stride, oy);
    }
}

template <typename Rr>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_inv(const RowPair *__restrict__ rps,
                                                         const typename CT<Rr>::T *__restrict__ tw_all,
                                                         const typename CT<Rr>::T *__restrict__ chirp_all,
                                                         const typename CT<Rr>::T *__restrict__ kern_all,
                                                         const Rr *__restrict__ fb, int Cp, Rr *__restrict__ grid,
                                                         long long npts, int nfields, int G, int T, int Jp)
{
    typedef typename CT<Rr>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int j = blockIdx.y;
    const RowPair rp = rps[j];
    const int N = rp.N, W = rp.fftlen;
    C *tw = (C *)smem_raw;
    C *ch = tw + W;
    C *x = ch + (rp.mode ? N : 0);
    C *y = x + (size_t)G * W;
    const int f0 = blockIdx.x * G;

    for (int t = threadIdx.x; t < W; t += blockDim.x) tw[t] = tw_all[rp.tw_off + t];
    if (rp.mode)
        for (int t = threadIdx.x; t < N; t += blockDim.x) ch[t] = chirp_all[rp.chirp_off + t];
    for (int idx = threadIdx.x; idx < G * W; idx += blockDim.x) {
        C v;
        v.x = 0;
        v.y = 0;
        x[idx] = v;
    }
    __syncthreads();
    // conj(Z): Z[m] = Xn + i Xs, Z[N-m] = conj(Xn) + i conj(Xs), Z[0] = Re Xn + i Re Xs
    const int M = rp.M;
    for (int idx = threadIdx.x; idx < (M + 1) * G; idx += blockDim.x) {
        int m = idx / G, f = idx - m * G;
        int fld = f0 + f;
        if (fld >= nfields) continue;
        long long rS = ((long long)m * Jp + j) * Cp + 2 * fld;
        long long rA = (((long long)(T + 1) + m) * Jp + j) * Cp + 2 * fld;
        // the odd-parity half of m = T is empty (no n = T + 1), so its rows are
        // never written by the Legendre stage: A = 0 there
        Rr sx = fb[rS], sy = fb[rS + 1];
        Rr axx = m < T ? fb[rA] : (Rr)0, ayy = m < T ? fb[rA + 1] : (Rr)0;
        Rr nx = sx + axx, ny = sy + ayy;   // north F_m
        Rr qx = sx - axx, qy = sy - ayy;   // south F_m
        C *xf = x + (size_t)f * W;
        if (m == 0) {
            C v;
            v.x = nx;
            v.y = -qx;
            xf[0] = v;
        } else {
            C a, b;
            a.x = nx - qy;
            a.y = -(ny + qx);
            b.x = nx + qy;
            b.y = ny - qx;
            xf[m] = a;
            xf[N - m] = b;
        }
    }
    __syncthreads();
    C *z = fft_forward<C>(x, y, tw, ch, kern_all + rp.kern_off, rp, G, W);
    for (int idx = threadIdx.x; idx < G * N; idx += blockDim.x) {
        int f = idx / N, k = idx - f * N;
        int fld = f0 + f;
        if (fld >= nfields) continue;
        C v = z[(size_t)f * W + k];
        Rr *g = grid + (long long)fld * npts;
        g[rp.off_n + k] = v.x;
        g[rp.off_s + k] = -v.y;
    }
}

// Fields per CTA so that roots, chirp and two work buffers of every row fit
// in shared memory.
static int fft_fields_per_cta(const st_plan *p, int nfields, size_t *smem)
{
    const size_t cs = p->prec == P_FP64 ? 16 : 8;
    size_t fixed = 0, per = 0;
    for (const auto &r : p->rowpairs_h) {
        fixed = std::max(fixed, (size_t)(r.fftlen + (r.mode ? r.N : 0)) * cs);
        per = std::max(per, (size_t)r.fftlen * cs);
    }
    const size_t budget = 110 * 1024;
    int G = budget > fixed ? (int)((budget - fixed) / (2 * per)) : 1;
    if (G < 1) G = 1;
    if (G > 8) G = 8;
    if (G > nfields) G = nfields;
    *smem = fixed + 2 * per * (size_t)G;
    return G;
}

template <typename K>
static st_status set_smem(K kern, size_t smem)
{
    if (smem > 48 * 1024) ST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return ST_OK;
}

st_status launch_fft_dir(st_plan *p, const void *grid, int nfields, cudaStream_t s)
{
    size_t smem;
    int G = fft_fields_per_cta(p, nfields, &smem);
    if (smem > 227 * 1024) return ST_ERR_UNSUPPORTED;
    dim3 g((nfields + G - 1) / G, p->J);
    int Cp = cols_padded(nfields);
    const long long Rp = fb_rows(p);
    const long long ps = Rp * Cp;
    st_status r = ST_OK;
    switch (p->prec) {
    case P_FP64: {
        auto k = k_fft_dir<double, S_F64>;
        if ((r = set_smem(k, smem))) return r;
        k<<<g, FFT_THREADS, smem, s>>>(p->rowpairs, (const double2 *)p->tw, (const double2 *)p->chirp,
                                       (const double2 *)p->kern, (const double *)grid, p->npts, nfields, G,
                               p->fbop, Cp, Rp, ps, p->T, p->Jp);
        break;
    }
    case P_FP32: {
        auto k = k_fft_dir<float, S_F32>;
        if ((r = set_smem(k, smem))) return r;
        k<<<g, FFT_THREADS, smem, s>>>(p->rowpairs, (const float2 *)p->tw, (const float2 *)p->chirp,
                                       (const float2 *)p->kern, (const float *)grid, p->npts, nfields, G,
                               p->fbop, Cp, Rp, ps, p->T, p->Jp);
        break;
    }
    case P_TF32X3: {
        auto k = k_fft_dir<float, S_TF32_SPLIT>;
        if ((r = set_smem(k, smem))) return r;
        k<<<g, FFT_THREADS, smem, s>>>(p->rowpairs, (const float2 *)p->tw, (const float2 *)p->chirp,
                                       (const float2 *)p->kern, (const float *)grid, p->npts, nfields, G,
                               p->fbop, Cp, Rp, ps, p->T, p->Jp);
        break;
    }
    default: {
        auto k = k_fft_dir<float, S_BF16_SPLIT>;
        if ((r = set_smem(k, smem))) return r;
        k<<<g, FFT_THREADS, smem, s>>>(p->rowpairs, (const float2 *)p->tw, (const float2 *)p->chirp,
                                       (const float2 *)p->kern, (const float *)grid, p->npts, nfields, G,
                               p->fbop, Cp, Rp, ps, p->T, p->Jp);
        break;
    }
    }
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

st_status launch_fft_inv(st_plan *p, void *grid, int nfields, cudaStream_t s)
{
    size_t smem;
    int G = fft_fields_per_cta(p, nfields, &smem);
    if (smem > 227 * 1024) return ST_ERR_UNSUPPORTED;
    dim3 g((nfields + G - 1) / G, p->J);
    int Cp = cols_padded(nfields);
    st_status r = ST_OK;
    if (p->prec == P_FP64) {
        auto k = k_fft_inv<double>;
        if ((r = set_smem(k, smem))) return r;
        k<<<g, FFT_THREADS, smem, s>>>(p->rowpairs, (const double2 *)p->tw, (const double2 *)p->chirp,
                                       (const double2 *)p->kern, (const double *)p->fb, Cp, (double *)grid,
                               p->npts, nfields, G, p->T, p->Jp);
    } else {
        auto k = k_fft_inv<float>;
        if ((r = set_smem(k, smem))) return r;
        k<<<g, FFT_THREADS, smem, s>>>(p->rowpairs, (const float2 *)p->tw, (const float2 *)p->chirp,
                                       (const float2 *)p->kern, (const float *)p->fb, Cp, (float *)grid,
                               p->npts, nfields, G, p->T, p->Jp);
    }
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

}  // namespace st
