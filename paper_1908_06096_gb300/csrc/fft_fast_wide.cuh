// Row-FFT bodies of one direction and plan group at the persistent batch
// kernel's CTA width (512 threads, batch_persistent.cu): the same bodies as
// fft_fast_inst.cuh instantiates for the per-stage kernels, in namespace
// st::ffw, behind one dispatch function per translation unit that the batch
// kernel links against (relocatable device code).  A translation unit defines
// FF_DIR, FF_GROUP and FF_WBODY, then includes this file.
#define FF_NS ffw
#define FF_NT 512
#define FF_MINB 1
#include "fft_fast.cuh"

#if !defined(FF_DIR) || !defined(FF_GROUP) || !defined(FF_WBODY)
#error "define FF_DIR, FF_GROUP and FF_WBODY before including fft_fast_wide.cuh"
#endif

namespace st {
namespace ffw {

template <int GRP, class PL>
__device__ __forceinline__ void run_wbody(const FftJob &J, const RowPair &rp, int f0)
{
    if constexpr (GRP == FF_GROUP) {
        if constexpr (FF_DIR) dir_body<PL>(J, rp, f0);
        else inv_body<PL>(J, rp, f0);
    }
}

// One 512-thread CTA's row pair rp (in shared memory) and fields f0 ..
// f0 + J.G - 1 of job J, whose plan belongs to this group.
__device__ void FF_WBODY(const FftJob &J, const RowPair &rp, int f0)
{
    switch (J.plan) {
#define X(id, grp, a, b_, c, d) \
    case id: run_wbody<grp, Plan<a, b_, c, d>>(J, rp, f0); break;
        ST_FF_PLANS(X)
#undef X
    default: break;
    }
}

}  // namespace ffw
}  // namespace st
