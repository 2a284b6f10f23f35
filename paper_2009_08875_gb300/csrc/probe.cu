// Measurement hook (not part of the method): the GPU's sustained fused multiply-add rates in
// binary64 and binary32, measured by a throughput kernel, to put the binary64 multigrid sweeps
// on an arithmetic roofline whose peak was measured on the same device and clocks.
//
// Each thread runs C independent multiply-add chains x <- x * a + c (a slightly below 1, so the
// values stay finite and normal; C = 4, 8 and 16 are tried and the best rate kept), with enough
// warps per SM to cover the pipeline latency, and the launch is timed with CUDA events.  The
// chain results are folded into one value per block and stored in a file-scope device array, so
// the compiler cannot drop the arithmetic; nothing is allocated.
#include <cuda_runtime.h>

#include "st_internal.cuh"

namespace st {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 8;
constexpr int kProbeMaxBlocks = 4096;

__device__ double g_probe_sink[kProbeMaxBlocks];

template <typename T, int kChains>
__global__ void __launch_bounds__(kProbeThreads) k_fma_rate(int iters, T a, T c) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  __shared__ T red[kProbeThreads];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = T(0);
    for (int i = 0; i < kProbeThreads; ++i) t += red[i];
    g_probe_sink[blockIdx.x] = (double)t;
  }
}

// fused multiply-adds per second of one timed launch (best of `reps` after one warm-up)
template <typename T, int kChains>
cudaError_t time_rate(int blocks, int iters, int reps, cudaStream_t s, double* rate) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = 1e30f;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, s);
    k_fma_rate<T, kChains><<<blocks, kProbeThreads, 0, s>>>(iters, T(0.999999), T(1e-6));
    e = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;  // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) *rate = (double)blocks * kProbeThreads * kChains * 16.0 * iters / (best * 1e-3);
  return e;
}

// the best of 4, 8 and 16 chains per thread, the same number of fmas per launch
template <typename T>
cudaError_t best_rate(int blocks, int iters8, cudaStream_t s, double* rate) {
  double r4 = 0.0, r8 = 0.0, r16 = 0.0;
  cudaError_t e = time_rate<T, 4>(blocks, 2 * iters8, 3, s, &r4);
  if (e == cudaSuccess) e = time_rate<T, 8>(blocks, iters8, 3, s, &r8);
  if (e == cudaSuccess) e = time_rate<T, 16>(blocks, iters8 / 2, 3, s, &r16);
  *rate = r4 > r8 ? (r4 > r16 ? r4 : r16) : (r8 > r16 ? r8 : r16);
  return e;
}

}  // namespace

}  // namespace st

using namespace st;

extern "C" st_status st_probe_fma_rates(void* cuda_stream, double* fp64_fma_per_s, double* fp32_fma_per_s) {
  if (!fp64_fma_per_s || !fp32_fma_per_s) {
    set_error("st_probe_fma_rates: null pointer");
    return ST_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail("st_probe_fma_rates: device query", e);
  int blocks = sms * kProbeBlocksPerSM;
  blocks = blocks < 1 ? 1 : (blocks > kProbeMaxBlocks ? kProbeMaxBlocks : blocks);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  // binary64: about 2.5e9 fmas (a few ms at ~6e11/s); binary32: 32x as many
  e = best_rate<double>(blocks, 64, s, fp64_fma_per_s);
  if (e == cudaSuccess) e = best_rate<float>(blocks, 2048, s, fp32_fma_per_s);
  if (e != cudaSuccess) return cuda_fail("st_probe_fma_rates", e);
  return ST_OK;
}
