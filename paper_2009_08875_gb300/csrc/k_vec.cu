// PCG vector kernels (Sec. 3.4): inner products with a fixed-shape two-pass reduction (the
// same grid, the same partition and the same summation order on every call, so results are
// bitwise reproducible), and the axpy updates of the Hestenes-Stiefel recurrences, which read
// their scalars from device memory so the loop needs no host round trip except the stop test.
#include <type_traits>

#include "st_internal.cuh"

namespace st {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0
}

// inner products accumulate in binary64 partial sums, whatever the vectors' storage type.  Problem
// blockIdx.y of a batch owns elements [y n, (y + 1) n); its partial sums go to
// partials[y * gridDim.x + blockIdx.x].  The partition depends only on n, so a problem gives the
// same bits alone and inside any batch.
template <typename Ta, typename Tb>
__global__ void __launch_bounds__(256) k_dot_partial(const Ta* __restrict__ a, const Tb* __restrict__ b, int64_t n,
                                                     double* __restrict__ partials) {
  a += (int64_t)blockIdx.y * n;
  b += (int64_t)blockIdx.y * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double t;
  if constexpr (std::is_same<Ta, float>::value && std::is_same<Tb, float>::value) {
    // binary32 vectors: a product of two floats is exactly p + e (p = fl(a b), e = fma(a, b, -p)),
    // summed in double-float (about 48 bits, well inside the binary64 partial sums it feeds) and
    // converted once per thread.  This keeps the loop off the binary64 pipe, which GB300 runs at
    // 1/58 of the binary32 rate: widening and a binary64 fma per element made the dot bound by it.
    df64 acc0(0.0f), acc1(0.0f);
    auto prod = [](float x, float y) {
      const float p = __fmul_rn(x, y);
      return df64(p, __fmaf_rn(x, y, -p), 0);
    };
    for (; i + stride < n; i += 2 * stride) {
      acc0 += prod(a[i], b[i]);
      acc1 += prod(a[i + stride], b[i + stride]);
    }
    if (i < n) acc0 += prod(a[i], b[i]);
    t = block_sum(double(acc0) + double(acc1));
  } else {
    double acc0 = 0.0, acc1 = 0.0;
    for (; i + stride < n; i += 2 * stride) {
      acc0 = fma((double)a[i], (double)b[i], acc0);
      acc1 = fma((double)a[i + stride], (double)b[i + stride], acc1);
    }
    if (i < n) acc0 = fma((double)a[i], (double)b[i], acc0);
    t = block_sum(acc0 + acc1);
  }
  if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// one block per problem: sum its partials and update its PCG scalars.  act (may be null) marks
// the problems still iterating; a finished problem gets alpha = beta = 0, so the updates leave
// its vectors unchanged while the others go on.
__global__ void __launch_bounds__(256) k_dot_final(const double* __restrict__ partials, int nb_per,
                                                   double* __restrict__ scal, const int* __restrict__ act, int slot,
                                                   int op) {
  const int prob = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb_per; i += blockDim.x) acc += partials[(int64_t)prob * nb_per + i];
  double t = block_sum(acc);
  if (threadIdx.x == 0) {
    double* sc = scal + (int64_t)prob * SC_COUNT;
    const bool on = act == nullptr || act[prob] != 0;
    switch (op) {
      case DOT_STORE:
        sc[slot] = t;
        break;
      case DOT_ALPHA:  // t = p^T q (a zero problem, r = p = 0, takes no step)
        sc[SC_PQ] = t;
        sc[SC_ALPHA] = (on && t != 0.0) ? sc[SC_RHO] / t : 0.0;
        break;
      case DOT_BETA:  // t = r^T z (new)
        sc[SC_RHO_NEW] = t;
        sc[SC_BETA] = (on && sc[SC_RHO] != 0.0) ? t / sc[SC_RHO] : 0.0;
        if (on) sc[SC_RHO] = t;
        break;
      case DOT_BETA_FLEX:  // t = r^T z (new); slot SC_RZOLD holds r^T z_old (Polak-Ribiere)
        sc[SC_RHO_NEW] = t;
        sc[SC_BETA] = (on && sc[SC_RHO] != 0.0) ? (t - sc[SC_RZOLD]) / sc[SC_RHO] : 0.0;
        if (on) sc[SC_RHO] = t;
        break;
      case DOT_INIT:  // t = r_0^T z_0; beta = 0 makes the first p = z + beta p (p = 0) equal z
        sc[SC_RHO] = t;
        sc[SC_RHO0] = t;
        sc[SC_RHO_NEW] = t;
        sc[SC_BETA] = 0.0;
        break;
    }
  }
}

// w += alpha p;  r -= alpha q  (problem blockIdx.y, elements [y n, (y+1) n))
template <typename T>
__global__ void __launch_bounds__(256) k_update_wr(T* __restrict__ w, T* __restrict__ r, const T* __restrict__ p,
                                                   const T* __restrict__ q, int64_t n, const double* __restrict__ sc) {
  const T alpha = (T)sc[(int64_t)blockIdx.y * SC_COUNT + SC_ALPHA];
  const int64_t off = (int64_t)blockIdx.y * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    w[off + i] = fma(alpha, p[off + i], w[off + i]);
    r[off + i] = fma(-alpha, q[off + i], r[off + i]);
  }
}

// p = z + beta p
template <typename T>
__global__ void __launch_bounds__(256) k_update_p(T* __restrict__ p, const T* __restrict__ z, int64_t n,
                                                  const double* __restrict__ sc) {
  const T beta = (T)sc[(int64_t)blockIdx.y * SC_COUNT + SC_BETA];
  const int64_t off = (int64_t)blockIdx.y * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    p[off + i] = fma(beta, p[off + i], z[off + i]);
}

// dst = src, converting the storage type (binary64 <-> binary32 rounds to nearest)
template <typename Td, typename Ts>
__global__ void __launch_bounds__(256) k_copy(Td* __restrict__ dst, const Ts* __restrict__ src, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = (Td)src[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_zero(T* __restrict__ dst, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = T(0);
}

// w += d (binary64 accumulation of a binary32 correction)
__global__ void __launch_bounds__(256) k_add_correction(double* __restrict__ w, const float* __restrict__ d,
                                                        int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) w[i] += (double)d[i];
}

// y = alpha x + beta y (binary64)
__global__ void __launch_bounds__(256) k_axpby(double* __restrict__ y, const double* __restrict__ x, double alpha,
                                               double beta, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = alpha * x[i] + beta * y[i];
}

// r = f - q (binary64) and, if rs is not null, rs = r rounded to binary32
__global__ void __launch_bounds__(256) k_residual_split(double* __restrict__ r, float* __restrict__ rs,
                                                        const double* __restrict__ f, const double* __restrict__ q,
                                                        int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = f[i] - q[i];
    r[i] = v;
    if (rs) rs[i] = (float)v;
  }
}

// ---------------------------------------------------------------------------------------
// Stop tests of the device-driven PCG loops (Sec. 3.4, Eq. 3.3).  They take, per problem, the
// same decisions as the host-driven loop from the same binary64 scalars, store the per-problem
// state in `ds` (DevState) and set the condition of the CUDA graph's WHILE node that repeats the
// iteration body: non-zero while some problem is active and the iteration limit is not reached,
// so a loop runs at most `maxit` times whatever the data.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool stop_breakdown(double pq, double rho, bool check_pq) {
  return (check_pq && (!(pq > 0.0) || !isfinite(pq))) || !isfinite(rho) || rho < 0.0;
}

// one block; all threads return whether any problem is active
__device__ __forceinline__ bool block_any(bool v) { return __syncthreads_or(v ? 1 : 0) != 0; }

// PCG (binary64 iteration, binary64 or binary32 preconditioner), and the outer loop of iterative
// refinement.  mode LOOP_INIT: start from rho_0 = scal[slot] (slot SC_RHO0, or SC_OUTER for the
// refinement); mode LOOP_ITER: after one iteration, rho = scal[slot] (SC_RHO_NEW, or SC_OUTER) and
// p^T q = scal[SC_PQ] when check_pq.  The refinement's outer test also ends a problem whose inner
// iterations reached maxit (ST_ERR_MAXIT) and stops the loop when no inner solve made progress.
__global__ void __launch_bounds__(256) k_loop_test(const double* __restrict__ scal, int* __restrict__ act,
                                                   DevState ds, int B, double tol, int tol_mode, int maxit,
                                                   int mode, int slot, int check_pq, int refine,
                                                   cudaGraphConditionalHandle hc) {
  const int it = mode == LOOP_INIT ? 0 : ds.ctr[0] + 1;
  bool any = false;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double* sc = scal + (int64_t)b * SC_COUNT;
    if (mode == LOOP_INIT) {
      const double r0 = sc[slot];
      ds.iters[b] = 0;
      ds.outer[b] = 0;
      ds.relres[b] = 0.0;
      ds.status[b] = ST_OK;
      ds.rho0[b] = r0;
      int a = 1;
      if (!isfinite(r0) || r0 < 0.0) {
        ds.status[b] = ST_ERR_BREAKDOWN;
        a = 0;
      } else if (r0 == 0.0 || (tol_mode == 1 && sqrt(r0) <= tol)) {
        a = 0;
      }
      act[b] = a;
      if (refine) ds.oact[b] = a;
      any = any || a;
      continue;
    }
    if (refine) {
      if (!ds.oact[b]) continue;
      act[b] = 1;
    } else {
      if (!act[b]) continue;
      ds.iters[b] = it;
    }
    const double rho = sc[slot], pq = sc[SC_PQ];
    int a = 1;
    if (stop_breakdown(pq, rho, check_pq != 0)) {
      ds.status[b] = ST_ERR_BREAKDOWN;
      a = 0;
    } else {
      const double rr = sqrt(rho / ds.rho0[b]);
      ds.relres[b] = rr;
      if (tol_mode == 1 ? sqrt(rho) <= tol : rr <= tol) a = 0;
    }
    act[b] = a;
    if (refine) {
      if (!a) ds.oact[b] = 0;
      if (a && ds.iters[b] >= maxit) {
        ds.status[b] = ST_ERR_MAXIT;
        ds.oact[b] = 0;
      }
      any = any || ds.oact[b];
    } else {
      any = any || a;
    }
  }
  any = block_any(any);
  if (threadIdx.x == 0) {
    ds.ctr[0] = it;
    bool go = any && it < maxit;
    if (refine && mode != LOOP_INIT) go = go && ds.ctr[1] != 0;  // some inner solve made progress
    cudaGraphSetConditional(hc, go ? 1u : 0u);
  }
}

// The refinement's inner binary32 PCG.  mode LOOP_INIT: problems active in the outer loop with
// rho_0 = scal[SC_RHO0] > 0 (finite) start; mode LOOP_ITER: a problem stops at a relative K_X-norm
// reduction of inner_tol or when binary32 can make no further progress.  ds.its counts each
// problem's inner iterations.
__global__ void __launch_bounds__(256) k_inner_test(const double* __restrict__ scal, int* __restrict__ act,
                                                    DevState ds, int B, double inner_tol, int inner_maxit, int mode,
                                                    cudaGraphConditionalHandle hc) {
  const int it = mode == LOOP_INIT ? 0 : ds.ctr[2] + 1;
  bool any = false;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double* sc = scal + (int64_t)b * SC_COUNT;
    if (mode == LOOP_INIT) {
      const double r0 = sc[SC_RHO0];
      ds.its[b] = 0;
      const int a = ds.oact[b] && r0 > 0.0 && isfinite(r0);
      act[b] = a;
      any = any || a;
      continue;
    }
    if (!act[b]) continue;
    ds.its[b] = it;
    const double pq = sc[SC_PQ], rho = sc[SC_RHO_NEW];
    const int a = !(stop_breakdown(pq, rho, true) || sqrt(rho / sc[SC_RHO0]) <= inner_tol);
    act[b] = a;
    any = any || a;
  }
  any = block_any(any);
  if (threadIdx.x == 0) {
    ds.ctr[2] = it;
    cudaGraphSetConditional(hc, (any && it < inner_maxit) ? 1u : 0u);
  }
}

// After an inner solve: every problem of the outer loop adds its inner iterations and one outer
// step; ds.ctr[1] records whether any inner solve made progress.
__global__ void __launch_bounds__(256) k_refine_count(DevState ds, int B) {
  bool prog = false;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (!ds.oact[b]) continue;
    ds.iters[b] += ds.its[b];
    ds.outer[b] += 1;
    prog = prog || ds.its[b] > 0;
  }
  prog = block_any(prog);
  if (threadIdx.x == 0) ds.ctr[1] = prog ? 1 : 0;
}

// blocks of the dot-product partition of one problem of n elements (depends on n only)
inline int dot_blocks(int64_t n) {
  int64_t g = (n + 8 * kThreads - 1) / (8 * kThreads);
  return (int)(g < 1 ? 1 : (g > kDotBlocks ? kDotBlocks : g));
}

// blocks per problem of a batched elementwise update, about kDotBlocks in total
inline unsigned per_problem_grid(int64_t n, int nb) {
  int64_t g = (n + kThreads - 1) / kThreads;
  int64_t cap = kDotBlocks / nb > 0 ? kDotBlocks / nb : 1;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

inline unsigned stream_grid(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  return (unsigned)(g < kDotBlocks ? (g > 0 ? g : 1) : kDotBlocks);
}

}  // namespace

template <typename Ta, typename Tb>
cudaError_t launch_dot(const st_handle_s* h, int b0, int nb, const Ta* a, const Tb* b, int64_t n, int slot, int op) {
  const int nblk = dot_blocks(n);
  k_dot_partial<Ta, Tb><<<dim3(nblk, nb), kThreads, 0, h->stream>>>(a, b, n, h->partials);
  k_dot_final<<<nb, kThreads, 0, h->stream>>>(h->partials, nblk, h->scal + (int64_t)b0 * SC_COUNT, h->act + b0, slot,
                                               op);
  count_launch(h, 2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_wr(const st_handle_s* h, int b0, int nb, T* w, T* r, const T* p, const T* q, int64_t n) {
  k_update_wr<T><<<dim3(per_problem_grid(n, nb), nb), kThreads, 0, h->stream>>>(w, r, p, q, n,
                                                                                 h->scal + (int64_t)b0 * SC_COUNT);
  count_launch(h);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_p(const st_handle_s* h, int b0, int nb, T* p, const T* z, int64_t n) {
  k_update_p<T><<<dim3(per_problem_grid(n, nb), nb), kThreads, 0, h->stream>>>(p, z, n,
                                                                                h->scal + (int64_t)b0 * SC_COUNT);
  count_launch(h);
  return cudaGetLastError();
}

template <typename Td, typename Ts>
cudaError_t launch_copy(const st_handle_s* h, Td* dst, const Ts* src, int64_t n) {
  k_copy<Td, Ts><<<stream_grid(n), kThreads, 0, h->stream>>>(dst, src, n);
  count_launch(h);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero(const st_handle_s* h, T* dst, int64_t n) {
  k_zero<T><<<stream_grid(n), kThreads, 0, h->stream>>>(dst, n);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_axpby(const st_handle_s* h, double* y, const double* x, double alpha, double beta, int64_t n) {
  k_axpby<<<stream_grid(n), kThreads, 0, h->stream>>>(y, x, alpha, beta, n);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_add_correction(const st_handle_s* h, double* w, const float* d, int64_t n) {
  k_add_correction<<<stream_grid(n), kThreads, 0, h->stream>>>(w, d, n);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_residual_split(const st_handle_s* h, double* r, float* rs, const double* f, const double* q,
                                  int64_t n) {
  k_residual_split<<<stream_grid(n), kThreads, 0, h->stream>>>(r, rs, f, q, n);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_loop_test(const st_handle_s* h, int mode, int slot, bool check_pq, bool refine,
                             cudaGraphConditionalHandle hc) {
  const st_config& c = h->cfg;
  k_loop_test<<<1, 256, 0, h->stream>>>(h->scal, h->act, h->ds, h->B, c.tol, c.tol_mode, c.maxit, mode, slot,
                                        check_pq ? 1 : 0, refine ? 1 : 0, hc);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_inner_test(const st_handle_s* h, int mode, cudaGraphConditionalHandle hc) {
  const st_config& c = h->cfg;
  k_inner_test<<<1, 256, 0, h->stream>>>(h->scal, h->act, h->ds, h->B, c.inner_tol, c.inner_maxit, mode, hc);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_refine_count(const st_handle_s* h) {
  k_refine_count<<<1, 256, 0, h->stream>>>(h->ds, h->B);
  count_launch(h);
  return cudaGetLastError();
}

template cudaError_t launch_dot<double, double>(const st_handle_s*, int, int, const double*, const double*, int64_t,
                                                int, int);
template cudaError_t launch_dot<float, float>(const st_handle_s*, int, int, const float*, const float*, int64_t, int,
                                              int);
template cudaError_t launch_dot<double, float>(const st_handle_s*, int, int, const double*, const float*, int64_t,
                                               int, int);
template cudaError_t launch_update_wr<double>(const st_handle_s*, int, int, double*, double*, const double*,
                                              const double*, int64_t);
template cudaError_t launch_update_wr<float>(const st_handle_s*, int, int, float*, float*, const float*, const float*,
                                             int64_t);
template cudaError_t launch_update_p<double>(const st_handle_s*, int, int, double*, const double*, int64_t);
template cudaError_t launch_update_p<float>(const st_handle_s*, int, int, float*, const float*, int64_t);
template cudaError_t launch_copy<double, double>(const st_handle_s*, double*, const double*, int64_t);
template cudaError_t launch_copy<float, float>(const st_handle_s*, float*, const float*, int64_t);
template cudaError_t launch_copy<float, double>(const st_handle_s*, float*, const double*, int64_t);
template cudaError_t launch_copy<double, float>(const st_handle_s*, double*, const float*, int64_t);
template cudaError_t launch_zero<double>(const st_handle_s*, double*, int64_t);
template cudaError_t launch_zero<float>(const st_handle_s*, float*, int64_t);

}  // namespace st
