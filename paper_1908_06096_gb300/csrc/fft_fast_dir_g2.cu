// Fast FP32 row FFTs, direct direction, plan group 2 (fft_fast_inst.cuh).
// the direct runs best at 80 registers a thread (3 CTAs per SM)
#define FF_MINB 3
#define FF_DIR 1
#define FF_GROUP 2
#define FF_KERNEL k_fftf_dir_g2
#define FF_LAUNCH launch_fftf_dir_g2
#include "fft_fast_inst.cuh"
