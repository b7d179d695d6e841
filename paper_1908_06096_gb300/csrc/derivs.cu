// Derivative and wind transforms (include/st.h: st_plan_enable_derivatives,
// st_inv_trans_deriv, st_inv_trans_uv, st_dir_trans_vordiv).
//
// The SH dwarf's time step (ESCAPE D3.3 sections 4.2.2-4.2.3) takes, besides
// scalar fields, the horizontal derivatives of fields and the wind from
// vorticity and divergence, and the reverse.  On the unit sphere, with phi the
// latitude, mu = sin(phi) and H_n^m = (1 - mu^2) dPbar_n^m/dmu:
//   d/dlambda:            coefficient i m a_n^m, Pbar synthesis;
//   (1 - mu^2) d/dmu:     coefficient a_n^m,     H synthesis;
//   psi = -zeta / (n (n+1)), chi = -D / (n (n+1));
//   U = u cos(phi) = dchi/dlambda - (1 - mu^2) dpsi/dmu,
//   V = v cos(phi) = dpsi/dlambda + (1 - mu^2) dchi/dmu;
//   zeta_n^m = sum_j w_j / (1 - mu_j^2) (i m V_m Pbar + U_m H),
//   D_n^m    = sum_j w_j / (1 - mu_j^2) (i m U_m Pbar - V_m H).
// The factor i m depends on m only, so it commutes with the Legendre sums: the
// P and H Legendre stages run as ordinary grouped GEMMs on the same operand,
// and a small kernel combines their outputs per (m, row) before the FFT (or
// per coefficient before the unpack).  Everything else is the scalar path.
#include "st_internal.cuh"

#include <algorithm>

namespace st {

// One thread per (Fourier-buffer row, field f < F).  fb holds the P synthesis,
// fb2 the H synthesis, both with 2F column pairs (Cp of 2F):
//   mode 0 (winds, fields [psi | chi]):  U = i m P[chi] - H[psi] -> column pair f,
//                                        V = i m P[psi] + H[chi] -> column pair F + f;
//   mode 1 (scalar, field a in pair f):  i m P[a] -> pair f, H[a] -> pair F + f.
// Rows never written by a GEMM read as zero: the odd half of m = T has no
// n = T + 1, so the P synthesis leaves its A rows alone at m = T and the H
// synthesis (halves exchanged) its S rows.  The combined A rows at m = T do
// hold data (the H synthesis of n = T), so the FFT after this kernel reads
// them (FftJob::a_top).
template <typename Rr>
__global__ void k_deriv_combine(Rr *fb, const Rr *fb2, long long nrows, int T, int Jp, int Cp, int F, int mode)
{
    const long long total = nrows * F;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / F;
        const int f = (int)(i - r * F);
        const long long pm = r / Jp;
        const int m = (int)(pm % (T + 1)), half = (int)(pm / (T + 1));
        const bool zp = half == 1 && m == T, zh = half == 0 && m == T;
        Rr *a = fb + r * Cp;
        const Rr *h = fb2 + r * Cp;
        const Rr mm = (Rr)m;
        const Rr par = zp ? (Rr)0 : a[2 * f], pai = zp ? (Rr)0 : a[2 * f + 1];
        const Rr har = zh ? (Rr)0 : h[2 * f], hai = zh ? (Rr)0 : h[2 * f + 1];
        if (mode == 0) {
            const Rr pbr = zp ? (Rr)0 : a[2 * (F + f)], pbi = zp ? (Rr)0 : a[2 * (F + f) + 1];
            const Rr hbr = zh ? (Rr)0 : h[2 * (F + f)], hbi = zh ? (Rr)0 : h[2 * (F + f) + 1];
            // i m (x + i y) = (-m y, m x)
            a[2 * f] = -mm * pbi - har;
            a[2 * f + 1] = mm * pbr - hai;
            a[2 * (F + f)] = -mm * pai + hbr;
            a[2 * (F + f) + 1] = mm * par + hbi;
        } else {
            a[2 * f] = -mm * pai;
            a[2 * f + 1] = mm * par;
            a[2 * (F + f)] = har;
            a[2 * (F + f) + 1] = hai;
        }
    }
}

st_status launch_deriv_combine(st_plan *p, int mode, int nfields, void *fb, const void *fb2, cudaStream_t s)
{
    const int Cp = cols_padded(2 * nfields);
    const long long nrows = fb_rows(p);
    const long long total = nrows * nfields;
    const int threads = 256;
    const long long blocks = std::min<long long>((total + threads - 1) / threads, (long long)p->sm_count * 16);
    if (p->prec == P_FP64)
        k_deriv_combine<double><<<(unsigned)blocks, threads, 0, s>>>((double *)fb, (const double *)fb2, nrows,
                                                                     p->T, p->Jp, Cp, nfields, mode);
    else
        k_deriv_combine<float><<<(unsigned)blocks, threads, 0, s>>>((float *)fb, (const float *)fb2, nrows, p->T,
                                                                    p->Jp, Cp, nfields, mode);
    ++kernel_launches();
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

// Packed spectral rows (m, parity, k): sout holds the P analysis, sout2 the H
// analysis of the fields [U | V] (2F column pairs).  One CTA per m:
//   zeta = i m P[V] + H[U] -> column pair f,  D = i m P[U] - H[V] -> pair F + f.
template <typename Rr>
__global__ void k_vordiv_combine(Rr *sout, const Rr *sout2, const long long *srow, int T, int Cp, int F)
{
    const int m = blockIdx.x;
    const Rr mm = (Rr)m;
    for (int par = 0; par < 2; ++par) {
        const int K = par ? (T - m + 1) / 2 : (T - m) / 2 + 1;
        const long long r0 = srow[2 * m + par];
        for (int i = threadIdx.x; i < K * F; i += blockDim.x) {
            const int k = i / F, f = i - k * F;
            Rr *a = sout + (r0 + k) * Cp;
            const Rr *h = sout2 + (r0 + k) * Cp;
            const Rr pur = a[2 * f], pui = a[2 * f + 1], pvr = a[2 * (F + f)], pvi = a[2 * (F + f) + 1];
            const Rr hur = h[2 * f], hui = h[2 * f + 1], hvr = h[2 * (F + f)], hvi = h[2 * (F + f) + 1];
            a[2 * f] = -mm * pvi + hur;
            a[2 * f + 1] = mm * pvr + hui;
            a[2 * (F + f)] = -mm * pui - hvr;
            a[2 * (F + f) + 1] = mm * pur - hvi;
        }
    }
}

st_status launch_vordiv_combine(st_plan *p, int nfields, void *sout, const void *sout2, cudaStream_t s)
{
    const int Cp = cols_padded(2 * nfields);
    if (p->prec == P_FP64)
        k_vordiv_combine<double><<<p->T + 1, 256, 0, s>>>((double *)sout, (const double *)sout2, p->srow, p->T, Cp,
                                                          nfields);
    else
        k_vordiv_combine<float><<<p->T + 1, 256, 0, s>>>((float *)sout, (const float *)sout2, p->srow, p->T, Cp,
                                                         nfields);
    ++kernel_launches();
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

}  // namespace st

using namespace st;

namespace {

st_status check_deriv(st_plan_t p, int nfields)
{
    if (!p) return ST_ERR_ARG;
    if (!p->deriv) {
        set_last_error("derivatives are not enabled on this plan (st_plan_enable_derivatives)");
        return ST_ERR_ARG;
    }
    if (nfields < 1 || 2 * nfields > p->max_fields) {
        set_last_error("derivative and wind transforms need 1 <= 2 nfields <= max_fields");
        return ST_ERR_ARG;
    }
    return ST_OK;
}

}  // namespace

extern "C" {

st_status st_plan_enable_derivatives(st_plan_t p, void *stream)
{
    if (!p) return ST_ERR_ARG;
    if (p->deriv) return ST_OK;
    cudaStream_t s = (cudaStream_t)stream;
    st_status r;
    for (int set = SET_SYN_H; set < NSETS; ++set) {
        build_groups_deriv(p, set);
        if ((r = plan_alloc(p, (void **)&p->groups[set], sizeof(LegGroup) * p->groups_h[set].size()))) return r;
        ST_CUDA(cudaMemcpyAsync(p->groups[set], p->groups_h[set].data(), sizeof(LegGroup) * p->groups_h[set].size(),
                                cudaMemcpyHostToDevice, s));
        if ((r = plan_alloc(p, &p->tab[set], p->tab_bytes[set]))) return r;
        ST_CUDA(cudaMemsetAsync(p->tab[set], 0, std::max<size_t>(p->tab_bytes[set], 16), s));
        p->table_bytes += p->tab_bytes[set];
    }
    if ((r = count_launch(p, K_TABLES, s, [&] { return launch_tables_deriv(p, s); }))) return r;
    if ((r = plan_alloc(p, &p->fb2, p->fb_bytes))) return r;
    if ((r = plan_alloc(p, &p->sout2, p->sout_bytes))) return r;
    ST_CUDA(cudaMemsetAsync(p->fb2, 0, p->fb_bytes, s));
    ST_CUDA(cudaMemsetAsync(p->sout2, 0, p->sout_bytes, s));
    p->workspace_bytes += p->fb_bytes + p->sout_bytes;
    // the host copies of the groups must outlive the asynchronous copies
    ST_CUDA(cudaStreamSynchronize(s));
    p->deriv = true;
    return ST_OK;
}

st_status st_inv_trans_deriv(st_plan_t p, const void *spec_dev, void *out_dev, int nfields, void *stream)
{
    st_status r = check_deriv(p, nfields);
    if (r) return r;
    if (!spec_dev || !out_dev) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // the operands and Fourier buffers carry 2 nfields column pairs throughout
    // (the FFT writes both derivative fields of every input field)
    const int cp = cols_padded(2 * nfields);
    if ((r = count_launch(p, K_PACK, s, [&] {
             PackJob J;
             pack_job(p, 0, nfields, spec_dev, p->sop, &J, 0, cp);
             return launch_pack_jobs(0, p->prec, &J, 1, s);
         })))
        return r;
    if ((r = count_launch(p, K_LEG_INV, s, [&] { return launch_leg_set(p, SET_SYN, nfields, s, p->sop, p->fb, cp); })))
        return r;
    if ((r = count_launch(p, K_LEG_INV, s,
                          [&] { return launch_leg_set(p, SET_SYN_H, nfields, s, p->sop, p->fb2, cp); })))
        return r;
    if ((r = count_launch(p, K_COMBINE, s, [&] { return launch_deriv_combine(p, 1, nfields, p->fb, p->fb2, s); })))
        return r;
    return count_launch(p, K_FFT_INV, s, [&] { return launch_fft_inv(p, out_dev, 2 * nfields, s, nullptr, 1); });
}

st_status st_inv_trans_uv(st_plan_t p, const void *vordiv_dev, void *uv_dev, int nfields, void *stream)
{
    st_status r = check_deriv(p, nfields);
    if (r) return r;
    if (!vordiv_dev || !uv_dev) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nf2 = 2 * nfields;
    // [zeta | D] -> [psi | chi] (inverse Laplacian) in the packed operand
    if ((r = count_launch(p, K_PACK, s, [&] {
             PackJob J;
             pack_job(p, 0, nf2, vordiv_dev, p->sop, &J, 1);
             return launch_pack_jobs(0, p->prec, &J, 1, s);
         })))
        return r;
    if ((r = count_launch(p, K_LEG_INV, s, [&] { return launch_leg_set(p, SET_SYN, nf2, s, p->sop, p->fb); })))
        return r;
    if ((r = count_launch(p, K_LEG_INV, s, [&] { return launch_leg_set(p, SET_SYN_H, nf2, s, p->sop, p->fb2); })))
        return r;
    if ((r = count_launch(p, K_COMBINE, s, [&] { return launch_deriv_combine(p, 0, nfields, p->fb, p->fb2, s); })))
        return r;
    return count_launch(p, K_FFT_INV, s, [&] { return launch_fft_inv(p, uv_dev, nf2, s, nullptr, 1); });
}

st_status st_dir_trans_vordiv(st_plan_t p, const void *uv_dev, void *vordiv_dev, int nfields, void *stream)
{
    st_status r = check_deriv(p, nfields);
    if (r) return r;
    if (!uv_dev || !vordiv_dev) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nf2 = 2 * nfields;
    if ((r = count_launch(p, K_FFT_DIR, s, [&] { return launch_fft_dir(p, uv_dev, nf2, s); }))) return r;
    if ((r = count_launch(p, K_LEG_DIR, s, [&] { return launch_leg_set(p, SET_ANA_P1, nf2, s, p->fbop, p->sout); })))
        return r;
    if ((r = count_launch(p, K_LEG_DIR, s,
                          [&] { return launch_leg_set(p, SET_ANA_H1, nf2, s, p->fbop, p->sout2); })))
        return r;
    if ((r = count_launch(p, K_COMBINE, s, [&] { return launch_vordiv_combine(p, nfields, p->sout, p->sout2, s); })))
        return r;
    return count_launch(p, K_UNPACK, s, [&] { return launch_unpack(p, vordiv_dev, nf2, s); });
}

}  // extern "C"
