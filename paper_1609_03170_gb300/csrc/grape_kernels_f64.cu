// grape_kernels_f64.cu - the hot-path kernels instantiated in native FP64.
#include "grape_kernels.cuh"

GRAPE_DEFINE_LAUNCHERS(f64, grape_num::NumD)
