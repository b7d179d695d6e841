// Autotuner (st_plan_autotune): times candidate launch shapes on the plan
// itself and keeps the fastest.
//  - FFT, per direction: the shared-memory budget per CTA, which sets how
//    many fields a CTA holds (FP32 plans), and the CTA width (256 threads,
//    or 512 with twice the budget).
//  - Tensor-core Legendre: the inverse column-tile width (the tile shape of
//    the per-m GEMMs; changing it re-lays out the tables), first for all m,
//    then for the upper half of the wavenumbers alone (their reductions are
//    shorter, so a different width can suit them).  The direct GEMMs take
//    one column tile per (m, parity) up to 256 columns by construction.
// The choice can be appended to a cache file; st_plan_create applies a
// matching entry from the file named by ST_TUNE_CACHE.
#include "st_internal.cuh"

#include <algorithm>
#include <cstdio>

using namespace st;

namespace {

template <class F>
st_status time_ms(cudaStream_t s, int reps, F f, float *ms)
{
    cudaEvent_t a, b;
    ST_CUDA(cudaEventCreate(&a));
    ST_CUDA(cudaEventCreate(&b));
    st_status r = f();  // warm-up (also sets kernel attributes)
    if (r == ST_OK) {
        cudaEventRecord(a, s);
        for (int i = 0; i < reps && r == ST_OK; ++i) r = f();
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(ms, a, b);
        *ms /= reps;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return r;
}

}  // namespace

extern "C" st_status st_plan_autotune(st_plan_t p, int nfields, const char *cache_path, void *stream)
{
    if (!p || nfields < 1 || nfields > p->max_fields) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t el = p->prec == P_FP64 ? 8 : 4;
    void *grid = nullptr;
    ST_CUDA(cudaMalloc(&grid, (size_t)p->npts * nfields * el));
    ST_CUDA(cudaMemsetAsync(grid, 0, (size_t)p->npts * nfields * el, s));
    st_status r = ST_OK;
    const int reps = 3;

    // FFT launch shapes, per direction
    // (FP64 plans size their CTAs by a fixed budget: nothing to choose)
    const int kbs[] = {36, 54, 72, 108, 144};
    // FP32: variant 1 runs 512-thread CTAs (twice the fields a CTA)
    const int nvar_dir = p->prec == P_FP64 ? 0 : 2, nvar_inv = nvar_dir;
    for (int dir = 0; dir < 2 && r == ST_OK; ++dir) {
        float best = 1e30f;
        int bv = p->fft_var[dir], bk = p->fft_kb[dir];
        const int nvar = dir == 1 ? nvar_dir : nvar_inv;
        for (int v = 0; v < nvar && r == ST_OK; ++v)
            for (int kb : kbs) {
                p->fft_var[dir] = v;
                p->fft_kb[dir] = kb;
                float ms = 0;
                r = time_ms(s, reps, [&] {
                    return dir == 0 ? launch_fft_inv(p, grid, nfields, s) : launch_fft_dir(p, grid, nfields, s);
                }, &ms);
                if (r == ST_ERR_UNSUPPORTED) { r = ST_OK; continue; }  // budget too small for a row
                if (r != ST_OK) break;
                if (ms < best) { best = ms; bv = v; bk = kb; }
            }
        p->fft_var[dir] = bv;
        p->fft_kb[dir] = bk;
    }

    // inverse Legendre column-tile width (tensor-core plans)
    if (r == ST_OK && prec_is_tc(p->prec)) {
        const int J = p->J, jmax = (J + 15) / 16 * 16;
        const int cand[] = {64, 96, 128, 160, 192, 224, 256};
        float best = 1e30f;
        int bnt = p->nt_inv;
        for (int nt : cand) {
            if (nt > jmax && nt != cand[0]) continue;
            p->nt_inv = nt;
            if ((r = rebuild_legendre(p, s)) != ST_OK) break;
            float ms = 0;
            if ((r = time_ms(s, reps, [&] { return launch_leg_tc(p, 0, nfields, s); }, &ms)) != ST_OK) break;
            if (ms < best) { best = ms; bnt = nt; }
        }
        p->nt_inv = bnt;
        // then the upper half of the wavenumbers alone
        int bhi = 0;
        for (int nt : cand) {
            if (r != ST_OK) break;
            if (nt > jmax && nt != cand[0]) continue;
            if (nt == bnt) continue;  // the width chosen for all m is timed already
            p->nt_inv_hi = nt;
            if ((r = rebuild_legendre(p, s)) != ST_OK) break;
            float ms = 0;
            if ((r = time_ms(s, reps, [&] { return launch_leg_tc(p, 0, nfields, s); }, &ms)) != ST_OK) break;
            if (ms < best) { best = ms; bhi = nt; }
        }
        if (r == ST_OK) {
            p->nt_inv_hi = bhi;
            r = rebuild_legendre(p, s);
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(grid);
    if (r == ST_OK && cache_path && *cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s | %d %d %d %d %d %d\n", tune_key(p, nfields).c_str(), p->fft_var[0], p->fft_kb[0],
                    p->fft_var[1], p->fft_kb[1], p->nt_inv, p->nt_inv_hi);
            fclose(f);
        }
    }
    return r;
}
