// Row FFTs at the persistent batch kernel's CTA width: inverse direction, plan group 0
// (fft_fast_wide.cuh).
#define FF_DIR 0
#define FF_GROUP 0
#define FF_WBODY wide_inv_g0
#include "fft_fast_wide.cuh"
