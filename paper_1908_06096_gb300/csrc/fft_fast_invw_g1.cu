// Fast FP32 row FFTs, inverse direction, plan group 1, 512-thread CTAs
// (launch variant 1: twice the fields per CTA of variant 0, so that each
// CTA's Fourier-buffer loads cover twice the columns) (fft_fast_inst.cuh).
#define FF_NS ffw
#define FF_NT 512
#define FF_MINB 1
#define FF_DIR 0
#define FF_GROUP 1
#define FF_KERNEL k_fftf_invw_g1
#define FF_LAUNCH launch_fftf_invw_g1
#include "fft_fast_inst.cuh"
