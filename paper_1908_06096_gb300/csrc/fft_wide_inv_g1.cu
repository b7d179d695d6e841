// Row FFTs at the persistent batch kernel's CTA width: inverse direction, plan group 1
// (fft_fast_wide.cuh).
#define FF_DIR 0
#define FF_GROUP 1
#define FF_WBODY wide_inv_g1
#include "fft_fast_wide.cuh"
