// grape_kernels_df.cu - the hot-path kernels instantiated in double-float
// arithmetic on the FP32 pipes (the default precision).
#include "grape_kernels.cuh"

GRAPE_DEFINE_LAUNCHERS(df, grape_num::NumF)
