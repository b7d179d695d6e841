// Row FFTs at the persistent batch kernel's CTA width: direct direction, plan group 1
// (fft_fast_wide.cuh).
#define FF_DIR 1
#define FF_GROUP 1
#define FF_WBODY wide_dir_g1
#include "fft_fast_wide.cuh"
