// Row-FFT stage, host side: the jobs of one stage (runs of rows that share a
// launch shape) and their dispatch to the compile-time FP32 plans
// (fft_fast.cuh) or the generic kernels (fft_generic.cuh).
#include "st_internal.cuh"

#include <algorithm>
#include <cstring>

namespace st {

// generic-kernel launchers (fft_gen_*.cu)
st_status launch_gen_dir_f64(const FftJob *jobs, int n, size_t smem, cudaStream_t s);
st_status launch_gen_dir_f32(const FftJob *jobs, int n, size_t smem, cudaStream_t s);
st_status launch_gen_inv_f64(const FftJob *jobs, int n, size_t smem, cudaStream_t s);
st_status launch_gen_inv_f32(const FftJob *jobs, int n, size_t smem, cudaStream_t s);

// Fields per CTA.  A CTA transforms G fields of one row pair, one shared-
// memory slot of the row's padded FFT length each, within the plan's per-CTA
// budget for this direction (autotuned).  G is the largest power of two (at
// most FFT_MAX_G and nfields) whose slots fit, so short rows near the poles
// take many fields per CTA and long rows few.
constexpr int FFT_MAX_G = 64;

static int fft_fields_for_slot(const st_plan *p, int dir, int nfields, int slot)
{
    const size_t cs = p->prec == P_FP64 ? 16 : 8;
    const size_t budget = p->prec == P_FP64 ? 110 * 1024 : (size_t)p->fft_kb[dir] * 1024;
    int G = 1;
    while (G < FFT_MAX_G && G < nfields && (size_t)(2 * G) * slot * cs <= budget) G *= 2;
    return std::min(G, nfields);
}
// The jobs of one FFT stage over all row pairs of `p` for `nfields` fields.
// The plan's device row-pair array holds the rows of the compile-time FP32
// plans first (entries 0 .. nfast-1, longest first), then the rows of the
// generic kernel ordered by padded FFT length, longest first.  Rows that
// share a launch shape form consecutive runs; one job per run.
//  - fast rows: a run shares (plan, fields per CTA); a CTA holds as many
//    fields as fit the per-CTA shared-memory budget (1 or an even number, so
//    that two adjacent fields always start on a 16-byte column boundary);
//  - generic rows: a run shares G (a power of two), its slot the longest
//    padded length in the run.
// *smem is the most any generic job needs (fast jobs carry their own).
st_status fft_jobs(st_plan *p, int dir, int nfields, const void *src, void *dst, std::vector<FftJob> &jobs,
                   size_t *smem, int kb)
{
    const size_t cs = p->prec == P_FP64 ? 16 : 8;
    const int J = p->J;
    FftJob base;
    memset(&base, 0, sizeof(base));
    base.rps = p->rowpairs;
    base.tw = p->tw;
    base.chirp = p->chirp;
    // the inverse's Bluestein kernel spectra follow all rows' direct ones
    base.kern = (const char *)p->kern + (dir == 0 ? cs * (size_t)p->nkern : 0);
    base.src = src;
    base.dst = dst;
    base.npts = p->npts;
    base.nfields = nfields;
    base.Cp = cols_padded(nfields);
    base.Rp = fb_rows(p);
    base.ps = base.Rp * base.Cp;
    base.T = p->T;
    base.Jp = p->Jp;
    base.smode = store_of(p->prec);
    base.err = p->err;

    // fast rows
    // launch variant 1 runs 512-thread CTAs: twice the budget of a
    // 256-thread CTA, within one SM's shared memory
    size_t budget = (size_t)(kb > 0 ? kb : p->fft_kb[dir]) * 1024;
    if (kb <= 0 && p->prec != P_FP64 && p->fft_var[dir] == 1) budget = std::min<size_t>(2 * budget, 216 * 1024);
    for (int r = 0; r < p->nfast;) {
        const RowPair &rp = p->rowpairs_h[p->row_order[r]];
        const int id = rp.fast;
        const bool blue = rp.mode == 1;
        const int SL = ff_slot(rp.fftlen);
        int e = r + 1;
        while (e < p->nfast && p->rowpairs_h[p->row_order[e]].fast == id &&
               (p->rowpairs_h[p->row_order[e]].mode == 1) == blue)
            ++e;
        const size_t tab = (size_t)ff_table_elems(id) * cs;
        int G = (int)std::min<size_t>(budget > tab ? (budget - tab) / ((size_t)SL * cs) : 1, 128);
        G = std::max(1, std::min(G, nfields));
        if (G > 1 && (G & 1)) --G;
        FftJob J1 = base;
        J1.kind = ff_group(id);
        J1.plan = id;
        J1.r0 = r;
        J1.J = e - r;
        J1.G = G;
        J1.Sslot = SL;
        J1.nfg = (nfields + G - 1) / G;
        J1.smem = (int)((size_t)((G * SL + 1) & ~1) * cs + tab);
        if (J1.smem > 227 * 1024) return ST_ERR_UNSUPPORTED;
        jobs.push_back(J1);
        r = e;
    }

    // generic rows
    std::vector<int> slot(J), G(J);
    for (int r = p->nfast; r < J; ++r) {
        const RowPair &rp = p->rowpairs_h[p->row_order[r]];
        slot[r] = fft_swz_size(rp.fftlen, rp.swz);
        G[r] = fft_fields_for_slot(p, dir, nfields, slot[r]);
    }
    size_t need = 0;
    for (int r = p->nfast; r < J;) {
        int e = r + 1;
        while (e < J && G[e] == G[r]) ++e;
        FftJob J1 = base;
        J1.kind = -1;
        J1.plan = -1;
        J1.r0 = r;
        J1.J = e - r;
        J1.G = G[r];
        J1.Sslot = *std::max_element(slot.begin() + r, slot.begin() + e);
        J1.nfg = (nfields + J1.G - 1) / J1.G;
        J1.smem = (int)std::min<size_t>((size_t)J1.G * J1.Sslot * cs, 1u << 30);
        need = std::max(need, (size_t)J1.G * J1.Sslot * cs);
        jobs.push_back(J1);
        r = e;
    }
    *smem = std::max(*smem, need);
    if (need > 227 * 1024) return ST_ERR_UNSUPPORTED;
    return ST_OK;
}

// dir 0: inverse (Fourier buffer -> grid), 1: direct (grid -> operand).  All
// jobs share the precision `prec`.  Jobs go to their kernel by kind: the
// generic kernel (smem: the most a generic job needs) or one of the
// compile-time plan groups; at most MAX_JOBS jobs per launch.
st_status launch_fft_jobs(int dir, int prec, const FftJob *jobs, int n, size_t smem, cudaStream_t s, int variant)
{
    if (n <= 0) return ST_OK;
    for (int kind = -1; kind < FF_NGROUPS; ++kind) {
        std::vector<FftJob> sel;
        for (int q = 0; q < n; ++q)
            if (jobs[q].kind == kind) sel.push_back(jobs[q]);
        for (size_t i = 0; i < sel.size(); i += MAX_JOBS) {
            const int m = (int)std::min<size_t>(MAX_JOBS, sel.size() - i);
            st_status r;
            if (kind < 0) {
                size_t need = 0;
                for (int q = 0; q < m; ++q) need = std::max(need, (size_t)sel[i + q].smem);
                if (dir == 1)
                    r = prec == P_FP64 ? launch_gen_dir_f64(sel.data() + i, m, need, s)
                                       : launch_gen_dir_f32(sel.data() + i, m, need, s);
                else
                    r = prec == P_FP64 ? launch_gen_inv_f64(sel.data() + i, m, need, s)
                                       : launch_gen_inv_f32(sel.data() + i, m, need, s);
            } else {
                r = launch_fftf(dir, kind, sel.data() + i, m, s, variant);
            }
            if (r) return r;
        }
    }
    (void)smem;
    return ST_OK;
}

st_status launch_fftf(int dir, int group, const FftJob *jobs, int n, cudaStream_t s, int variant)
{
    if (variant == 1) {
        switch (dir * 4 + group) {
        case 0: return launch_fftf_invw_g0(jobs, n, s);
        case 1: return launch_fftf_invw_g1(jobs, n, s);
        case 2: return launch_fftf_invw_g2(jobs, n, s);
        case 4: return launch_fftf_dirw_g0(jobs, n, s);
        case 5: return launch_fftf_dirw_g1(jobs, n, s);
        case 6: return launch_fftf_dirw_g2(jobs, n, s);
        }
        return ST_ERR_ARG;
    }
    switch (dir * 4 + group) {
    case 0: return launch_fftf_inv_g0(jobs, n, s);
    case 1: return launch_fftf_inv_g1(jobs, n, s);
    case 2: return launch_fftf_inv_g2(jobs, n, s);
    case 4: return launch_fftf_dir_g0(jobs, n, s);
    case 5: return launch_fftf_dir_g1(jobs, n, s);
    case 6: return launch_fftf_dir_g2(jobs, n, s);
    }
    return ST_ERR_ARG;
}

// The 3xTF32 direct GEMM reads its data operand K-major (latitude rows
// contiguous per data column), which a row FFT, one latitude row pair per
// CTA, could only write four bytes at a time.  So the row FFTs of 3xTF32
// plans write E/O row-major in FP32 into the plan's inverse Fourier buffer
// (free during a direct transform), and this kernel transposes 32 x 32
// tiles into the split operand: hi = tf32(v), lo = tf32(v - hi), column c
// of each plane at c Rp + r.  Rows the row FFTs did not write carry older
// finite values, which meet zero table entries in the GEMM.
__global__ void __launch_bounds__(256) k_fb_tf32split(const float *__restrict__ src, float *__restrict__ dst,
                                                      long long rows, int C, int Cp, long long Rp, long long ps)
{
    __shared__ float t[32][33];
    const long long r0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const long long r = r0 + k;
        const int c = c0 + tx;
        t[k][tx] = (r < rows && c < C) ? src[r * Cp + c] : 0.f;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k;
        const long long r = r0 + tx;
        if (c < C && r < rows) {
            const float v = t[tx][k];
            uint32_t h, l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(v - __uint_as_float(h)));
            dst[(long long)c * Rp + r] = __uint_as_float(h);
            dst[(long long)c * Rp + r + ps] = __uint_as_float(l);
        }
    }
}

st_status launch_fb_tf32split(st_plan *p, int nfields, cudaStream_t s)
{
    const long long rows = fb_rows(p);
    const int C = 2 * nfields, Cp = cols_padded(nfields);
    const dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((C + 31) / 32));
    k_fb_tf32split<<<grid, 256, 0, s>>>((const float *)p->fb, (float *)p->fbop, rows, C, Cp, rows,
                                       rows * (long long)Cp);
    ++kernel_launches();
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

// Jobs of the direct row FFTs of `p` into the operand of its direct GEMM
// (3xTF32 plans: row-major FP32 into the inverse Fourier buffer, for
// launch_fb_tf32split).
st_status fft_dir_jobs(st_plan *p, int nfields, const void *grid, std::vector<FftJob> &jobs, size_t *smem, int kb)
{
    const bool tf32 = p->prec == P_TF32X3;
    st_status r = fft_jobs(p, 1, nfields, grid, tf32 ? p->fb : p->fbop, jobs, smem, kb);
    if (r == ST_OK && tf32)
        for (auto &J : jobs) J.smode = S_F32;
    return r;
}

st_status launch_fft_dir(st_plan *p, const void *grid, int nfields, cudaStream_t s)
{
    std::vector<FftJob> jobs;
    size_t smem = 0;
    st_status r = fft_dir_jobs(p, nfields, grid, jobs, &smem);
    if (r) return r;
    if ((r = launch_fft_jobs(1, p->prec, jobs.data(), (int)jobs.size(), smem, s, p->fft_var[1]))) return r;
    return p->prec == P_TF32X3 ? launch_fb_tf32split(p, nfields, s) : ST_OK;
}

st_status launch_fft_inv(st_plan *p, void *grid, int nfields, cudaStream_t s, const void *fb_in, int a_top)
{
    std::vector<FftJob> jobs;
    size_t smem = 0;
    st_status r = fft_jobs(p, 0, nfields, fb_in ? fb_in : p->fb, grid, jobs, &smem);
    if (r) return r;
    for (auto &J : jobs) J.a_top = a_top;
    return launch_fft_jobs(0, p->prec, jobs.data(), (int)jobs.size(), smem, s, p->fft_var[0]);
}

}  // namespace st
