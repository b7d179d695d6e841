// Generic row-FFT kernel instance: direct direction, FP64.
#include "fft_generic.cuh"

namespace st {

st_status launch_gen_dir_f64(const FftJob *jobs, int n, size_t smem, cudaStream_t s)
{
    if (n <= 0) return ST_OK;
    if (n > MAX_JOBS) return ST_ERR_ARG;
    return run_fft_batch<MAX_JOBS>(k_fft_dir<double, S_F64, MAX_JOBS, 256, 2>, 256, jobs, n, smem, s);
}

}  // namespace st
