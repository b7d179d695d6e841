// Kernel and launcher of one direction for one group of compile-time FFT
// plans (fft_fast.cuh).  Each group is its own translation unit so that the
// plans compile in parallel; a translation unit defines FF_DIR (1 direct,
// 0 inverse), FF_GROUP, FF_KERNEL and FF_LAUNCH, then includes this file.
#include "fft_fast.cuh"

#if !defined(FF_DIR) || !defined(FF_GROUP) || !defined(FF_KERNEL) || !defined(FF_LAUNCH)
#error "define FF_DIR, FF_GROUP, FF_KERNEL and FF_LAUNCH before including fft_fast_inst.cuh"
#endif

namespace st {
namespace FF_NS {

// Plans outside this translation unit's group are never instantiated here.
template <int GRP, class PL>
__device__ __forceinline__ void run_body(const FftJob &J, const RowPair &rp, int f0)
{
    if constexpr (GRP == FF_GROUP) {
        if constexpr (FF_DIR) dir_body<PL>(J, rp, f0);
        else inv_body<PL>(J, rp, f0);
    }
}

// One CTA: one row pair (entry r0 + rr of the job's run) and fields
// f0 .. f0 + G - 1; the job's plan selects the compile-time body.
__global__ void __launch_bounds__(NT, MINB) FF_KERNEL(const __grid_constant__ FftBatch<MAX_JOBS> B)
{
    __shared__ RowPair rp;
    const int q = find_job<MAX_JOBS>(B.prefix, B.njobs, blockIdx.x);
    const FftJob &J = B.job[q];
    const int b = (int)(blockIdx.x - B.prefix[q]);
    const int rr = b / J.nfg;
    const int f0 = (b - rr * J.nfg) * J.G;
    {
        const int nw = (int)(sizeof(RowPair) / sizeof(int));
        const int *src = (const int *)(J.rps + J.r0 + rr);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) ((int *)&rp)[i] = src[i];
        __syncthreads();
    }
    switch (J.plan) {
#define X(id, grp, a, b_, c, d) \
    case id: run_body<grp, Plan<a, b_, c, d>>(J, rp, f0); break;
        ST_FF_PLANS(X)
#undef X
    default: break;
    }
}

}  // namespace FF_NS

st_status FF_LAUNCH(const FftJob *jobs, int n, cudaStream_t s)
{
    if (n <= 0) return ST_OK;
    if (n > MAX_JOBS) return ST_ERR_ARG;
    FftBatch<MAX_JOBS> B;
    B.njobs = n;
    long long tot = 0;
    int smem = 0;
    for (int q = 0; q < n; ++q) {
        if (jobs[q].kind != FF_GROUP) return ST_ERR_ARG;
        B.prefix[q] = tot;
        B.job[q] = jobs[q];
        tot += (long long)jobs[q].J * jobs[q].nfg;
        smem = smem > jobs[q].smem ? smem : jobs[q].smem;
    }
    B.prefix[n] = tot;
    if (tot == 0) return ST_OK;
    if (tot > 0x7fffffffLL) return ST_ERR_UNSUPPORTED;
    if (smem > 227 * 1024) return ST_ERR_UNSUPPORTED;
    if (smem > 48 * 1024)
        ST_CUDA(cudaFuncSetAttribute(FF_NS::FF_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FF_NS::FF_KERNEL<<<(unsigned)tot, FF_NS::NT, smem, s>>>(B);
    ++kernel_launches();
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

}  // namespace st
