// Wide binary32 Gauss-Seidel sweeps (k_gs_wide.cuh): bfloat16 storage, three fused sweeps.
#include "k_gs_wide.cuh"

namespace st {
ST_WIDE_INSTANTIATE(__nv_bfloat16, 3, wide_attr_bf16_nsw3)
}  // namespace st
