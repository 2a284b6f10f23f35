// Wide binary32 Gauss-Seidel sweeps (k_gs_wide.cuh): binary32 storage, three fused sweeps; the
// level test and the attribute setter of all four instantiation units.
#include "k_gs_wide.cuh"

namespace st {

ST_WIDE_INSTANTIATE(float, 3, wide_attr_f32_nsw3)
template cudaError_t wide_launch_scale_restrict<false>(const st_handle_s*, int, int, int, float*, const float*, float*,
                                                       float*);
template cudaError_t wide_launch_scale_restrict<true>(const st_handle_s*, int, int, int, float*, const float*, float*,
                                                      float*);

bool wide_fits(const st_handle_s* h, int /*shape*/, int k) {
  // the half-warp regions (96 x 96) below 192 columns, the whole-warp ones (192 x 96) above
  const int n = (1 << k) - 1;
  return h->domain == 0 && n >= 6 * WideShape<1>::NL && n >= (32 * WideShape<1>::NWARP / WideShape<1>::NL) * WideShape<1>::R;
}

cudaError_t wide_set_attributes() {
  cudaError_t e = wide_attr_f32_nsw3();
  if (e == cudaSuccess) e = wide_attr_f32_nsw1();
  if (e == cudaSuccess) e = wide_attr_bf16_nsw3();
  if (e == cudaSuccess) e = wide_attr_bf16_nsw1();
  return e;
}

}  // namespace st
