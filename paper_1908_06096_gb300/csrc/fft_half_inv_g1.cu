// Row FFTs in one half of the persistent batch kernel's CTA: inverse direction, plan
// group 1 (fft_fast_half.cuh).
#define FF_DIR 0
#define FF_GROUP 1
#define FF_HBODY half_inv_g1
#include "fft_fast_half.cuh"
