// Legendre stage on the SIMT cores (the plain FP64 form and the FP32 SIMT
// form), the spectral pack/unpack that lay the coefficients out as GEMM
// operands, and the Fourier-buffer export used by the parity tests.
//
// The Legendre transform of ESCAPE D3.3 section 4.2.4 is one matrix product
// per zonal wavenumber m.  Splitting n - m into even and odd halves (using
// Pbar_n^m(-mu) = (-1)^(n-m) Pbar_n^m(mu)) gives two products per m over the
// northern rows only, which halves the work; all (m, parity) products run in
// one launch, each tile looking up its group (the grouped form of section
// 4.2.4's batched GEMM, without zero padding to a common size).
#include "pack_dev.cuh"

namespace st {

// ---------------------------------------------------------------- SIMT GEMM

// out[col][c] = sum_r tab[col][r] * data[r][c] for one (group, column tile,
// data tile) per CTA; 64 x 64 outputs, 256 threads with 4 x 4 each.
template <typename Rr, int MAXJ>
__global__ void __launch_bounds__(256) k_leg_simt(const __grid_constant__ SimtBatch<MAXJ> B)
{
    constexpr int TB = SIMT_TILE, KB = 16;
    __shared__ Rr As[KB][TB + 1];
    __shared__ Rr Bs[KB][TB];
    const int q = find_job<MAXJ>(B.prefix, B.njobs, blockIdx.x);
    const SimtJob &J = B.job[q];
    const int tile = (int)(blockIdx.x - B.prefix[q]);
    const int ncm = J.ncm, C = J.C, Cp = J.Cp;
    const LegTile lt = J.tiles[tile / ncm];
    const int cm = tile % ncm;
    const LegGroup g = J.groups[lt.g];
    const Rr *tab = (const Rr *)J.tab;
    const Rr *data = (const Rr *)J.data;
    Rr *out = (Rr *)J.out;
    const int col0 = lt.ct * TB, c0 = cm * TB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    Rr acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;

    const Rr *tg = tab + g.tab_off;
    for (int r = g.r0; r < g.K; r += KB) {
        for (int e = threadIdx.x; e < TB * KB; e += 256) {
            int cc = e / KB, kk = e % KB;
            int col = col0 + cc, rr = r + kk;
            As[kk][cc] = (col < g.ncol && rr < g.K) ? tg[(long long)col * g.K + rr] : (Rr)0;
        }
        for (int e = threadIdx.x; e < TB * KB; e += 256) {
            int kk = e / TB, c = e % TB;
            int rr = r + kk, cg = c0 + c;
            Bs[kk][c] = (rr < g.K && cg < C) ? data[(g.data_row0 + rr) * (long long)Cp + cg] : (Rr)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KB; ++kk) {
            Rr a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[kk][ty * 4 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = Bs[kk][tx * 4 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int col = col0 + ty * 4 + u;
        if (col >= g.ncol) continue;
        Rr *o = out + (g.out_row0 + col) * (long long)Cp;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int c = c0 + tx * 4 + v;
            if (c < C) o[c] = acc[u][v];
        }
    }
}

st_status simt_job(st_plan *p, int set, int nfields, const void *data, void *out, SimtJob *job, long long *blocks,
                   int cp)
{
    const int td = set_dir(set);
    job->groups = p->groups[set];
    job->tiles = p->tiles[td];
    job->tab = p->tab[set];
    job->data = data;
    job->out = out;
    job->C = 2 * nfields;
    job->Cp = cp ? cp : cols_padded(nfields);
    job->ncm = (job->C + SIMT_TILE - 1) / SIMT_TILE;
    *blocks = (long long)p->ntiles[td] * job->ncm;
    return ST_OK;
}

template <int MAXJ, class K>
static st_status run_simt_batch(K kern, const SimtJob *jobs, const long long *blocks, int n, cudaStream_t s)
{
    SimtBatch<MAXJ> B;
    B.njobs = n;
    long long tot = 0;
    for (int q = 0; q < n; ++q) {
        B.prefix[q] = tot;
        B.job[q] = jobs[q];
        tot += blocks[q];
    }
    B.prefix[n] = tot;
    if (tot == 0) return ST_OK;
    if (tot > 0x7fffffffLL) return ST_ERR_UNSUPPORTED;
    kern<<<(unsigned)tot, 256, 0, s>>>(B);
    ++kernel_launches();
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

st_status launch_simt_jobs(int prec, const SimtJob *jobs, const long long *blocks, int n, cudaStream_t s)
{
    if (n <= 0) return ST_OK;
    if (n > MAX_JOBS) return ST_ERR_ARG;
    if (n == 1)
        return prec == P_FP64 ? run_simt_batch<1>(k_leg_simt<double, 1>, jobs, blocks, n, s)
                              : run_simt_batch<1>(k_leg_simt<float, 1>, jobs, blocks, n, s);
    return prec == P_FP64 ? run_simt_batch<MAX_JOBS>(k_leg_simt<double, MAX_JOBS>, jobs, blocks, n, s)
                          : run_simt_batch<MAX_JOBS>(k_leg_simt<float, MAX_JOBS>, jobs, blocks, n, s);
}

st_status launch_leg_set(st_plan *p, int set, int nfields, cudaStream_t s, void *data, void *out, int cp)
{
    if (prec_is_tc(p->prec)) {
        TcJob J;
        st_status r = tc_job(p, set, nfields, data, out, &J, cp);
        if (r) return r;
        return launch_tc_jobs(p->prec, &J, 1, p->sm_count, s);
    }
    SimtJob J;
    long long blocks = 0;
    simt_job(p, set, nfields, data, out, &J, &blocks, cp);
    return launch_simt_jobs(p->prec, &J, &blocks, 1, s);
}

st_status launch_leg_simt(st_plan *p, int dir, int nfields, cudaStream_t s, void *data_in, void *out_in)
{
    // inverse: data = packed spectra, out = Fourier buffer; direct: the reverse
    void *data = data_in ? data_in : (dir == 0 ? p->sop : p->fbop);
    void *out = out_in ? out_in : (dir == 0 ? p->fb : p->sout);
    SimtJob J;
    long long blocks = 0;
    simt_job(p, dir, nfields, data, out, &J, &blocks);
    return launch_simt_jobs(p->prec, &J, &blocks, 1, s);
}

// ---------------------------------------------------------------- pack / unpack

template <typename Rr, int S, int MAXJ>
__global__ void __launch_bounds__(256) k_pack(const __grid_constant__ PackBatch<MAXJ> B)
{
    __shared__ Rr tile[32][65];
    const int q = find_job<MAXJ>(B.prefix, B.njobs, blockIdx.x);
    pack_block<Rr, S>(B.job[q], (int)(blockIdx.x - B.prefix[q]), tile, threadIdx.x >> 5, threadIdx.x & 31,
                      [] { __syncthreads(); });
}

// Operand rows (direct GEMM output, FP32/FP64) -> spectra (pack_dev.cuh).
template <typename Rr, int MAXJ>
__global__ void __launch_bounds__(256) k_unpack(const __grid_constant__ PackBatch<MAXJ> B)
{
    __shared__ Rr tile[32][65];
    const int q = find_job<MAXJ>(B.prefix, B.njobs, blockIdx.x);
    unpack_block<Rr>(B.job[q], (int)(blockIdx.x - B.prefix[q]), tile, threadIdx.x >> 5, threadIdx.x & 31,
                     [] { __syncthreads(); });
}

// dir 0: pack (spectra -> operand), 1: unpack (GEMM output -> spectra).
st_status pack_job(st_plan *p, int dir, int nfields, const void *src, void *dst, PackJob *job, int scale, int cp)
{
    PackJob &J = *job;
    J.src = src;
    J.dst = dst;
    J.srow = p->srow;
    J.nspec = p->nspec;
    J.scale = scale;
    J.Cp = cp ? cp : cols_padded(nfields);
    J.Rp = p->srow_total;
    J.ps = J.Rp * J.Cp;
    J.T = p->T;
    J.max_m = p->max_m;
    J.nfields = nfields;
    J.nft = (nfields + 31) / 32;
    J.nm = dir == 0 ? p->max_m + 1 : p->T + 1;
    return ST_OK;
}

template <int MAXJ, class K>
static st_status run_pack_batch(K kern, const PackJob *jobs, int n, cudaStream_t s)
{
    PackBatch<MAXJ> B;
    B.njobs = n;
    long long tot = 0;
    for (int q = 0; q < n; ++q) {
        B.prefix[q] = tot;
        B.job[q] = jobs[q];
        tot += (long long)jobs[q].nm * jobs[q].nft;
    }
    B.prefix[n] = tot;
    if (tot == 0) return ST_OK;
    kern<<<(unsigned)tot, 256, 0, s>>>(B);
    ++kernel_launches();
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

template <int MAXJ>
static st_status launch_pack_jobs_t(int dir, int prec, const PackJob *jobs, int n, cudaStream_t s)
{
    if (dir == 1)
        return prec == P_FP64 ? run_pack_batch<MAXJ>(k_unpack<double, MAXJ>, jobs, n, s)
                              : run_pack_batch<MAXJ>(k_unpack<float, MAXJ>, jobs, n, s);
    switch (prec) {
    case P_FP64: return run_pack_batch<MAXJ>(k_pack<double, S_F64, MAXJ>, jobs, n, s);
    case P_FP32: return run_pack_batch<MAXJ>(k_pack<float, S_F32, MAXJ>, jobs, n, s);
    case P_TF32X3: return run_pack_batch<MAXJ>(k_pack<float, S_TF32_SPLIT, MAXJ>, jobs, n, s);
    default: return run_pack_batch<MAXJ>(k_pack<float, S_BF16_SPLIT, MAXJ>, jobs, n, s);
    }
}

st_status launch_pack_jobs(int dir, int prec, const PackJob *jobs, int n, cudaStream_t s)
{
    if (n <= 0) return ST_OK;
    if (n > MAX_JOBS) return ST_ERR_ARG;
    if (n == 1) return launch_pack_jobs_t<1>(dir, prec, jobs, n, s);
    return launch_pack_jobs_t<MAX_JOBS>(dir, prec, jobs, n, s);
}

st_status launch_pack(st_plan *p, const void *spec, int nfields, cudaStream_t s, void *sop_in)
{
    PackJob J;
    pack_job(p, 0, nfields, spec, sop_in ? sop_in : p->sop, &J);
    return launch_pack_jobs(0, p->prec, &J, 1, s);
}

st_status launch_unpack(st_plan *p, void *spec, int nfields, cudaStream_t s)
{
    PackJob J;
    pack_job(p, 1, nfields, p->sout, spec, &J);
    return launch_pack_jobs(1, p->prec, &J, 1, s);
}

// ---------------------------------------------------------------- export (tests)

__global__ void k_fourier_export(int T, int J, int Jp, const int *Mrow, int store, const void *fb, int Cp, long long Rp,
                                 long long ps, int nfields, double *out)
{
    long long total = 2LL * (T + 1) * J * nfields;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int f = (int)(i % nfields);
        long long rest = i / nfields;
        int j = (int)(rest % J);
        long long pm = rest / J;          // p (T+1) + m
        int m = (int)(pm % (T + 1));
        long long r = pm * Jp + j;        // Fourier-buffer row
        double v[2] = {0.0, 0.0};
        if (m <= Mrow[j]) {
            for (int q = 0; q < 2; ++q) {
                long long idx = op_index(store, r, 2 * f + q, Cp, Rp);
                if (store == S_F64) v[q] = ((const double *)fb)[idx];
                else if (store == S_F32) v[q] = ((const float *)fb)[idx];
                else if (store == S_TF32_SPLIT)
                    v[q] = (double)((const float *)fb)[idx] + (double)((const float *)fb)[idx + ps];
                else
                    v[q] = (double)__bfloat162float(((const __nv_bfloat16 *)fb)[idx]) +
                           (double)__bfloat162float(((const __nv_bfloat16 *)fb)[idx + ps]);
            }
        }
        out[2 * i] = v[0];
        out[2 * i + 1] = v[1];
    }
}

st_status launch_fourier_export(st_plan *p, int dir, int nfields, double *out, cudaStream_t s)
{
    int *Mrow_d = nullptr;
    ST_CUDA(cudaMallocAsync(&Mrow_d, sizeof(int) * p->J, s));
    ST_CUDA(cudaMemcpyAsync(Mrow_d, p->Mrow.data(), sizeof(int) * p->J, cudaMemcpyHostToDevice, s));
    int Cp = cols_padded(nfields);
    int store = dir == 0 ? (p->prec == P_FP64 ? S_F64 : S_F32) : store_of(p->prec);
    const long long Rp = fb_rows(p);
    long long ps = Rp * Cp;
    k_fourier_export<<<1024, 256, 0, s>>>(p->T, p->J, p->Jp, Mrow_d, store, dir == 0 ? p->fb : p->fbop, Cp, Rp, ps,
                                          nfields, out);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(Mrow_d, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_fourier_export");
    return ST_OK;
}

}  // namespace st
