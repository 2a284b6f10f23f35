// Wide binary32 Gauss-Seidel sweeps (k_gs_wide.cuh): binary32 storage, one sweep per launch.
#include "k_gs_wide.cuh"

namespace st {
ST_WIDE_INSTANTIATE(float, 1, wide_attr_f32_nsw1)
}  // namespace st
