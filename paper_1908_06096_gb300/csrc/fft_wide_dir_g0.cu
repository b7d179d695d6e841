// Row FFTs at the persistent batch kernel's CTA width: direct direction, plan group 0
// (fft_fast_wide.cuh).
#define FF_DIR 1
#define FF_GROUP 0
#define FF_WBODY wide_dir_g0
#include "fft_fast_wide.cuh"
