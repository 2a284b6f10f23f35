// Double-float arithmetic: a value is the unevaluated sum hi + lo of two binary32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  Built from the error-free transformations of
// Dekker (1971) and Knuth (TAOCP vol. 2, Sec. 4.2.2): TwoSum gives s + e = a + b exactly, the fused
// multiply-add gives p + e = a b exactly; the sum and product below follow the "double-double"
// recipes of Hida, Li and Bailey (2001) with binary32 halves.  On GB300 binary32 runs at ~58x the
// binary64 rate, so the multigrid's smoothing, which is bound by binary64 instruction issue, can
// run in this format at a fraction of the cost (ST_FP64_DF).
#pragma once

#include <cuda_runtime.h>

namespace st {

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ constexpr df64(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ explicit df64(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr df64(float h, float l, int) : hi(h), lo(l) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (no ordering assumption)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return df64(s, e, 0);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo, 0); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the leading product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s;
  fast_two_sum(p, e, s, e);
  return df64(s, e, 0);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }

// full-warp shuffles by d lanes for every element type of the multigrid (df64: both halves)
__device__ __forceinline__ double shfl_up(double v, unsigned d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float shfl_up(float v, unsigned d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ df64 shfl_up(df64 v, unsigned d) {
  return df64(__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d), 0);
}
__device__ __forceinline__ double shfl_down(double v, unsigned d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float shfl_down(float v, unsigned d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ df64 shfl_down(df64 v, unsigned d) {
  return df64(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d), 0);
}

}  // namespace st
