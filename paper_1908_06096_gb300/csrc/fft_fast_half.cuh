// Row-FFT bodies of one direction and plan group for one half of the
// persistent batch kernel's 512-thread CTA (batch_persistent.cu): the same
// bodies fft_fast_inst.cuh instantiates for the per-stage kernels, run by
// 256 threads with the half's own barrier and FF_HALF_BYTES of shared
// memory, in namespace st::ffh, behind one dispatch function per translation
// unit that the batch kernel links against (relocatable device code).  A
// translation unit defines FF_DIR, FF_GROUP and FF_HBODY, then includes this
// file.
#define FF_NS ffh
#define FF_NT 256
#define FF_MINB 1
#define FF_HALVES 1
#include "fft_fast.cuh"

#if !defined(FF_DIR) || !defined(FF_GROUP) || !defined(FF_HBODY)
#error "define FF_DIR, FF_GROUP and FF_HBODY before including fft_fast_half.cuh"
#endif

namespace st {
namespace ffh {

template <int GRP, class PL>
__device__ __forceinline__ void run_hbody(const FftJob &J, const RowPair &rp, int f0)
{
    if constexpr (GRP == FF_GROUP) {
        if constexpr (FF_DIR) dir_body<PL>(J, rp, f0);
        else inv_body<PL>(J, rp, f0);
    }
}

// One half's row pair rp (in shared memory) and fields f0 .. f0 + J.G - 1
// of job J, whose plan belongs to this group.
__device__ void FF_HBODY(const FftJob &J, const RowPair &rp, int f0)
{
    switch (J.plan) {
#define X(id, grp, a, b_, c, d) \
    case id: run_hbody<grp, Plan<a, b_, c, d>>(J, rp, f0); break;
        ST_FF_PLANS(X)
#undef X
    default: break;
    }
}

}  // namespace ffh
}  // namespace st
