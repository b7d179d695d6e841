// Fast FP32 row FFTs, inverse direction, plan group 1 (fft_fast_inst.cuh).
// the inverse runs best with 128 registers a thread (2 CTAs per SM)
#define FF_MINB 2
#define FF_DIR 0
#define FF_GROUP 1
#define FF_KERNEL k_fftf_inv_g1
#define FF_LAUNCH launch_fftf_inv_g1
#include "fft_fast_inst.cuh"
