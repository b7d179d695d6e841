// Generic row-FFT kernel instance: direct direction, FP32 (storage mode at run time).
#include "fft_generic.cuh"

namespace st {

st_status launch_gen_dir_f32(const FftJob *jobs, int n, size_t smem, cudaStream_t s)
{
    if (n <= 0) return ST_OK;
    if (n > MAX_JOBS) return ST_ERR_ARG;
    return run_fft_batch<MAX_JOBS>(k_fft_dir<float, S_RT, MAX_JOBS, 256, 2>, 256, jobs, n, smem, s);
}

}  // namespace st
