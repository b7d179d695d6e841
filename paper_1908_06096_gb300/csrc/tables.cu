// Plan-time kernels, all in FP64: Gaussian nodes and weights, normalised
// associated Legendre values, the Legendre tables in the layout each
// precision's GEMM reads, and the FFT roots of unity.
//
// Gaussian quadrature and the normalised associated Legendre functions are
// the ingredients of the transform of ESCAPE D3.3 section 4.4.1 (synthesis
// equation) and section 4.4.2 (coefficients as inner products); the paper
// does not spell out how they are computed.  Here: Newton iteration on
// P_nlat for the nodes, and the standard three-term recurrence in n for
// Pbar_n^m, both in FP64, once per plan.
#include "st_internal.cuh"

namespace st {

// ---------------------------------------------------------------- nodes

__device__ static void leg_p_and_prev(int n, double x, double &pn, double &pnm1)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { pn = 1.0; pnm1 = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    pn = p1;
    pnm1 = p0;
}

// One thread per northern root; Newton from cos(pi (j - 1/4) / (nlat + 1/2)),
// until the step is below 1e-15, plus one more step.  w = 2 / ((1 - x^2) P'^2).
__global__ void k_gauss(int nlat, double *mu, double *w)
{
    int half = (nlat + 1) / 2;
    int j = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (j > half) return;
    double x = cospi((j - 0.25) / (nlat + 0.5));
    double pn, pnm1, dp;
    bool extra = false;
    for (int it = 0; it < 100; ++it) {
        leg_p_and_prev(nlat, x, pn, pnm1);
        dp = nlat * (x * pn - pnm1) / (x * x - 1.0);
        double dx = pn / dp;
        x -= dx;
        if (extra) break;
        if (fabs(dx) < 1e-15) extra = true;
    }
    leg_p_and_prev(nlat, x, pn, pnm1);
    dp = nlat * (x * pn - pnm1) / (x * x - 1.0);
    double wj = 2.0 / ((1.0 - x * x) * dp * dp);
    if ((nlat & 1) && j == half) x = 0.0;
    mu[j - 1] = x;
    w[j - 1] = wj;
    mu[nlat - j] = -x;
    w[nlat - j] = wj;
}

st_status launch_gauss(int nlat, double *mu, double *w, cudaStream_t s)
{
    int half = (nlat + 1) / 2;
    k_gauss<<<(half + 127) / 128, 128, 0, s>>>(nlat, mu, w);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

// ---------------------------------------------------------------- Pbar recurrence

// Walks n = m .. T for one (m, mu) and hands each Pbar_n^m(mu) to `emit`.
//   Pbar_0^0 = 1/sqrt(2);  Pbar_m^m = sqrt((2m+1)/(2m)) sin(theta) Pbar_{m-1}^{m-1}
//   Pbar_{m+1}^m = sqrt(2m+3) mu Pbar_m^m
//   Pbar_n^m = sqrt((4n^2-1)/(n^2-m^2)) (mu Pbar_{n-1}^m
//              - sqrt(((n-1)^2-m^2)/(4(n-1)^2-1)) Pbar_{n-2}^m)
template <class F>
__device__ inline void pbar_column(int T, int m, double x, F emit)
{
    double s = sqrt((1.0 - x) * (1.0 + x));
    double pmm = 0.70710678118654752440;  // 1/sqrt(2)
    for (int k = 1; k <= m; ++k) pmm = sqrt((2.0 * k + 1.0) / (2.0 * k)) * s * pmm;
    emit(m, pmm);
    if (m + 1 > T) return;
    double p1 = sqrt(2.0 * m + 3.0) * x * pmm;
    emit(m + 1, p1);
    double p0 = pmm;
    double mm = (double)m * m;
    for (int n = m + 2; n <= T; ++n) {
        double dn = n, dn1 = n - 1.0;
        double a = sqrt((4.0 * dn * dn - 1.0) / (dn * dn - mm));
        double b = sqrt((dn1 * dn1 - mm) / (4.0 * dn1 * dn1 - 1.0));
        double p2 = a * (x * p1 - b * p0);
        emit(n, p2);
        p0 = p1;
        p1 = p2;
    }
}

__device__ inline long long tri_index(int T, int m, int n)
{
    return (long long)m * (T + 1) - (long long)m * (m - 1) / 2 + (n - m);
}

__global__ void k_legendre_values(int T, const double *mu, int nmu, double *out)
{
    int m = blockIdx.y;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmu || m > T) return;
    long long ns = (long long)(T + 1) * (T + 2) / 2;
    double *o = out + (long long)i * ns;
    pbar_column(T, m, mu[i], [&](int n, double v) { o[tri_index(T, m, n)] = v; });
}

st_status launch_legendre_values(int T, const double *mu, int nmu, double *out, cudaStream_t s)
{
    dim3 grid((nmu + 127) / 128, T + 1);
    k_legendre_values<<<grid, 128, 0, s>>>(T, mu, nmu, out);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

// ---------------------------------------------------------------- GEMM tables

// Byte address, inside a group's table, of element (col, r) of plane `plane`
// in the tensor-core layout: per (column tile, reduction chunk) one image of
// 2 planes x nt rows x 128 bytes, rows grouped by 8 into 1024-byte atoms with
// the 16-byte chunks of row i XOR-permuted by (i mod 8) (the 128-byte
// swizzle the tensor-core shared-memory descriptor expects for K-major data).
__device__ inline size_t tc_table_byte(const LegGroup &g, int col, int r, int plane, int es, int kc_len)
{
    int ct = col / g.nt, rr = col - ct * g.nt;
    int kc = r / kc_len, kk = r - kc * kc_len;
    size_t img = (size_t)g.tab_off + ((size_t)(ct * g.nkc + kc) * 2 + plane) * (size_t)g.nt * 128;
    int byte = kk * es;
    return img + (size_t)(rr >> 3) * 1024 + (size_t)(rr & 7) * 128 +
           (size_t)((((byte >> 4) ^ (rr & 7)) << 4) | (byte & 15));
}

__device__ inline float round_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int PREC>
__device__ inline void put_table(void *tab, const LegGroup &g, int col, int r, double v)
{
    if (PREC == P_FP64) {
        ((double *)tab)[g.tab_off + (long long)col * g.K + r] = v;
    } else if (PREC == P_FP32) {
        ((float *)tab)[g.tab_off + (long long)col * g.K + r] = (float)v;
    } else if (PREC == P_TF32X3) {
        float hi = round_tf32((float)v);
        float lo = round_tf32((float)(v - (double)hi));
        char *b = (char *)tab;
        *(float *)(b + tc_table_byte(g, col, r, 0, 4, 32)) = hi;
        *(float *)(b + tc_table_byte(g, col, r, 1, 4, 32)) = lo;
    } else {
        __nv_bfloat16 hi = __double2bfloat16(v);
        __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
        char *b = (char *)tab;
        *(__nv_bfloat16 *)(b + tc_table_byte(g, col, r, 0, 2, 64)) = hi;
        *(__nv_bfloat16 *)(b + tc_table_byte(g, col, r, 1, 2, 64)) = lo;
    }
}

// One thread per (m, northern row j): the inverse table gets Pbar_n^m(mu_j)
// at (col j, r k), the direct table w_j Pbar_n^m(mu_j) at (col k, r j), with
// n = m + p + 2k.  Rows that do not keep m (m > M_j) get zeros.
template <int PREC>
__global__ void k_tables(int T, int J, int max_m, const double *mu, const double *w, const int *Mrow,
                         const LegGroup *ginv, const LegGroup *gdir, void *tab_inv, void *tab_dir)
{
    int m = blockIdx.y;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J || m > max_m) return;
    bool keep = m <= Mrow[j];
    double x = mu[j], wj = w[j];
    LegGroup gi[2] = {ginv[2 * m], ginv[2 * m + 1]};
    LegGroup gd[2] = {gdir[2 * m], gdir[2 * m + 1]};
    pbar_column(T, m, x, [&](int n, double v) {
        int p = (n - m) & 1, k = (n - m) >> 1;
        if (!keep) v = 0.0;
        if (gi[p].K > 0) put_table<PREC>(tab_inv, gi[p], j, k, v);
        if (gd[p].ncol > 0) put_table<PREC>(tab_dir, gd[p], k, j, wj * v);
    });
}

st_status launch_tables(st_plan *p, cudaStream_t s)
{
    int *Mrow_d = nullptr;
    ST_CUDA(cudaMallocAsync(&Mrow_d, sizeof(int) * p->J, s));
    ST_CUDA(cudaMemcpyAsync(Mrow_d, p->Mrow.data(), sizeof(int) * p->J, cudaMemcpyHostToDevice, s));
    dim3 grid((p->J + 63) / 64, p->max_m + 1);
    switch (p->prec) {
    case P_FP64:
        k_tables<P_FP64><<<grid, 64, 0, s>>>(p->T, p->J, p->max_m, p->mu, p->w, Mrow_d, p->groups[0],
                                             p->groups[1], p->tab[0], p->tab[1]);
        break;
    case P_FP32:
        k_tables<P_FP32><<<grid, 64, 0, s>>>(p->T, p->J, p->max_m, p->mu, p->w, Mrow_d, p->groups[0],
                                             p->groups[1], p->tab[0], p->tab[1]);
        break;
    case P_TF32X3:
        k_tables<P_TF32X3><<<grid, 64, 0, s>>>(p->T, p->J, p->max_m, p->mu, p->w, Mrow_d, p->groups[0],
                                               p->groups[1], p->tab[0], p->tab[1]);
        break;
    default:
        k_tables<P_BF16X3><<<grid, 64, 0, s>>>(p->T, p->J, p->max_m, p->mu, p->w, Mrow_d, p->groups[0],
                                               p->groups[1], p->tab[0], p->tab[1]);
        break;
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(Mrow_d, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_tables");
    return ST_OK;
}

// ---------------------------------------------------------------- derivative tables
//
// H_n^m = (1 - mu^2) dPbar_n^m/dmu = (n+1) eps_n^m Pbar_{n-1}^m - n eps_{n+1}^m Pbar_{n+1}^m,
// eps_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)) (0 for n <= m).  One thread per
// (m, northern row j) walks the Pbar recurrence to T + 1 and writes, for
// n = m + p + 2k <= T:
//   set SYN_H  (synthesis layout): H_n^m(mu_j)                      at (col j, r k)
//   set ANA_P1 (analysis layout):  w_j / (1 - mu_j^2) Pbar_n^m(mu_j) at (col k, r j)
//   set ANA_H1 (analysis layout):  w_j / (1 - mu_j^2) H_n^m(mu_j)    at (col k, r j)
// (zeros on rows that do not keep m).
__device__ inline double eps_nm(int n, int m)
{
    if (n <= m) return 0.0;
    const double dn = n, dm = m;
    return sqrt((dn * dn - dm * dm) / (4.0 * dn * dn - 1.0));
}

template <int PREC>
__global__ void k_tables_deriv(int T, int J, int max_m, const double *mu, const double *w, const int *Mrow,
                               const LegGroup *gh, const LegGroup *gp1, const LegGroup *gh1, void *tab_h,
                               void *tab_p1, void *tab_h1)
{
    int m = blockIdx.y;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J || m > max_m) return;
    const bool keep = m <= Mrow[j];
    const double x = mu[j], c = w[j] / ((1.0 - x) * (1.0 + x));
    const LegGroup g0[2] = {gh[2 * m], gh[2 * m + 1]};
    const LegGroup g1[2] = {gp1[2 * m], gp1[2 * m + 1]};
    const LegGroup g2[2] = {gh1[2 * m], gh1[2 * m + 1]};
    double pa = 0.0, pb = 0.0;  // Pbar_{n-2}, Pbar_{n-1}
    pbar_column(T + 1, m, x, [&](int n, double v) {
        // v = Pbar_n: now H_{n-1} is known
        const int nn = n - 1;
        if (nn >= m) {
            double h = (nn + 1.0) * eps_nm(nn, m) * pa - (double)nn * eps_nm(nn + 1, m) * v;
            double pv = pb;
            if (!keep) h = pv = 0.0;
            const int p = (nn - m) & 1, k = (nn - m) >> 1;
            if (g0[p].K > 0) put_table<PREC>(tab_h, g0[p], j, k, h);
            if (g1[p].ncol > 0) put_table<PREC>(tab_p1, g1[p], k, j, c * pv);
            if (g2[p].ncol > 0) put_table<PREC>(tab_h1, g2[p], k, j, c * h);
        }
        pa = pb;
        pb = v;
    });
}

st_status launch_tables_deriv(st_plan *p, cudaStream_t s)
{
    int *Mrow_d = nullptr;
    ST_CUDA(cudaMallocAsync(&Mrow_d, sizeof(int) * p->J, s));
    ST_CUDA(cudaMemcpyAsync(Mrow_d, p->Mrow.data(), sizeof(int) * p->J, cudaMemcpyHostToDevice, s));
    dim3 grid((p->J + 63) / 64, p->max_m + 1);
#define ST_TD(PR)                                                                                              \
    k_tables_deriv<PR><<<grid, 64, 0, s>>>(p->T, p->J, p->max_m, p->mu, p->w, Mrow_d, p->groups[SET_SYN_H],  \
                                           p->groups[SET_ANA_P1], p->groups[SET_ANA_H1], p->tab[SET_SYN_H],    \
                                           p->tab[SET_ANA_P1], p->tab[SET_ANA_H1])
    switch (p->prec) {
    case P_FP64: ST_TD(P_FP64); break;
    case P_FP32: ST_TD(P_FP32); break;
    case P_TF32X3: ST_TD(P_TF32X3); break;
    default: ST_TD(P_BF16X3); break;
    }
#undef ST_TD
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(Mrow_d, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_tables_deriv");
    return ST_OK;
}

// ---------------------------------------------------------------- FFT roots

template <typename C>
__global__ void k_twiddles(const RowPair *rp, int J, C *tw)
{
    int j = blockIdx.y;
    if (j >= J) return;
    RowPair r = rp[j];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < r.fftlen; t += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)t / (double)r.fftlen, &sn, &cs);
        C v;
        v.x = (decltype(v.x))cs;
        v.y = (decltype(v.y))-sn;
        tw[r.tw_off + t] = v;
    }
}

// ---------------------------------------------------------------- Bluestein set-up
//
// Bluestein's identity m k = (m^2 + k^2 - (m - k)^2) / 2 turns the N-point DFT
//   Z_m = sum_k z_k e^{-2 pi i m k / N}
// into Z_m = w_m sum_k (z_k w_k) conj(w_{m-k}) with the chirp
// w_k = e^{-i pi k^2 / N}, for every integer m: a convolution with the
// conjugate chirp b_d = conj(w_d) over the offsets d = m - k that occur, done
// circularly at a length L that holds them all.
//   direct:  inputs k in [0, N), outputs m in [-M, M]  -> d in [-(N-1+M), M]
//   inverse: inputs m in [-M, M], outputs k in [0, N)  -> d in [-M, N-1+M]
// so L >= N + 2M and each direction's b is the other's mirror image
// (b_inv[i] = b_dir[-i mod L], hence FFT(b_inv)[k] = FFT(b_dir)[-k mod L]).
// The plan keeps w and both FFT_L(b) / L; all computed here in FP64 (k^2
// reduced mod 2N exactly in integers before the angle is formed).

__device__ inline void chirp_val(long long k, int N, double &c, double &s)
{
    long long t = (k * k) % (2LL * N);
    double sn, cs;
    sincospi((double)t / (double)N, &sn, &cs);
    c = cs;
    s = -sn;  // e^{-i pi t / N}
}

template <typename C>
__global__ void k_chirp(const RowPair *rps, int J, C *chirp)
{
    int j = blockIdx.y;
    if (j >= J) return;
    RowPair r = rps[j];
    if (r.mode != 1) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < r.N; k += gridDim.x * blockDim.x) {
        double c, s;
        chirp_val(k, r.N, c, s);
        C v;
        v.x = (decltype(v.x))c;
        v.y = (decltype(v.y))s;
        chirp[r.chirp_off + k] = v;
    }
}

// One CTA per Bluestein row: b in FP64, Stockham passes (one output per
// thread, roots by sincospi) in a global scratch buffer, result / L.
template <typename C>
__global__ void k_bluestein_kern(const RowPair *rps, int J, double2 *scratch, long long nkern, C *kern)
{
    int j = blockIdx.x;
    if (j >= J) return;
    const RowPair r = rps[j];
    if (r.mode != 1) return;
    const int N = r.N, L = r.fftlen;
    double2 *x = scratch + r.kern_off, *y = scratch + nkern + r.kern_off;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        long long d = -1;  // direct offsets: [0, M] at i = d, [-(N-1+M), -1] at i = L + d
        if (i <= r.M) d = i;
        else if (i >= L - (N - 1 + r.M)) d = L - i;
        if (d >= 0) {
            double c, s;
            chirp_val(d, N, c, s);
            v = make_double2(c, -s);  // conj(w_d)
        }
        x[i] = v;
    }
    __syncthreads();
    int Lc = 1;
    for (int q = 0; q < r.nrad; ++q) {
        const int R = r.rad[q], nb = L / R, step = L / (Lc * R);
        for (int o = threadIdx.x; o < L; o += blockDim.x) {
            int k = o % Lc, s_ = (o / Lc) % R, grp = o / (Lc * R);
            int b = grp * Lc + k;
            long long e = (long long)(k + s_ * Lc) * step;
            double ax = 0, ay = 0;
            for (int rr = 0; rr < R; ++rr) {
                double2 v = x[b + rr * nb];
                long long t = (e * rr) % L;
                double sn, cs;
                sincospi(2.0 * (double)t / (double)L, &sn, &cs);
                // v * e^{-2 pi i t / L}
                ax += v.x * cs + v.y * sn;
                ay += v.y * cs - v.x * sn;
            }
            y[o] = make_double2(ax, ay);
        }
        __syncthreads();
        double2 *t = x;
        x = y;
        y = t;
        Lc *= R;
    }
    // stored in the digit-reversed order the DIF passes leave their output
    // in, so the pointwise product needs no permutation.  Rows of the
    // compile-time plans transpose each block of R (the last radix) places:
    // place b R + q sits at q (L / R) + b, so that the threads of the fused
    // product pass, one block each, read consecutive values.
    const double inv = 1.0 / (double)L;
    const int RP = r.rad[r.nrad - 1], NBP = L / RP;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const double2 vd = x[i], vi = x[i == 0 ? 0 : L - i];
        int pos = dif_pos(i, r);
        if (r.fast >= 0) pos = (pos % RP) * NBP + pos / RP;
        C v;
        v.x = (decltype(v.x))(vd.x * inv);
        v.y = (decltype(v.y))(vd.y * inv);
        kern[r.kern_off + pos] = v;
        v.x = (decltype(v.x))(vi.x * inv);
        v.y = (decltype(v.y))(vi.y * inv);
        kern[nkern + r.kern_off + pos] = v;
    }
}

st_status launch_bluestein_setup(st_plan *p, cudaStream_t s)
{
    double2 *scratch = nullptr;
    ST_CUDA(cudaMallocAsync(&scratch, sizeof(double2) * 2 * (size_t)p->nkern, s));
    dim3 g1((p->max_chirp + 255) / 256, p->J);
    if (p->prec == P_FP64) {
        k_chirp<double2><<<g1, 256, 0, s>>>(p->rowpairs, p->J, (double2 *)p->chirp);
        k_bluestein_kern<double2><<<p->J, 256, 0, s>>>(p->rowpairs, p->J, scratch, p->nkern, (double2 *)p->kern);
    } else {
        k_chirp<float2><<<g1, 256, 0, s>>>(p->rowpairs, p->J, (float2 *)p->chirp);
        k_bluestein_kern<float2><<<p->J, 256, 0, s>>>(p->rowpairs, p->J, scratch, p->nkern, (float2 *)p->kern);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "bluestein set-up");
    return ST_OK;
}

st_status launch_twiddles(st_plan *p, cudaStream_t s)
{
    dim3 grid((p->max_fft + 255) / 256, p->J);
    if (p->prec == P_FP64)
        k_twiddles<double2><<<grid, 256, 0, s>>>(p->rowpairs, p->J, (double2 *)p->tw);
    else
        k_twiddles<float2><<<grid, 256, 0, s>>>(p->rowpairs, p->J, (float2 *)p->tw);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

}  // namespace st
