// Fast FP32 row FFTs, direct direction, plan group 0 (fft_fast_inst.cuh).
// the direct runs best at 128 registers a thread (2 CTAs per SM) since its rows
// arrive by bulk copies
#define FF_MINB 2
#define FF_DIR 1
#define FF_GROUP 0
#define FF_KERNEL k_fftf_dir_g0
#define FF_LAUNCH launch_fftf_dir_g0
#include "fft_fast_inst.cuh"
