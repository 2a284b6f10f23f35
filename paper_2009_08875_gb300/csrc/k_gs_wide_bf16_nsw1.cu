// Wide binary32 Gauss-Seidel sweeps (k_gs_wide.cuh): bfloat16 storage, one sweep per launch.
#include "k_gs_wide.cuh"

namespace st {
ST_WIDE_INSTANTIATE(__nv_bfloat16, 1, wide_attr_bf16_nsw1)
}  // namespace st
