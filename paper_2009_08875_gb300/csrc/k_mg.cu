// Time-slice-batched symmetric multigrid for C = a A_x + s M_x (K_x, K_l of Sec. 3.1 and
// Thm. 3.1; "2 V-cycles with 3 Gauss-Seidel steps per grid", Sec. 5.1).
//
// One launch processes every slice of a batch.  Level k has n = 2^k - 1 interior points
// per side, slices are contiguous n*n blocks.  Readings (the paper leaves them open):
// nested P1 prolongation, restriction = its transpose, rediscretised coarse operators,
// Gauss-Seidel in three colours c = (i + j) mod 3 of the grid indices (i, j) = (ix+1, iy+1),
// pre-sweeps in colour order 0,1,2 and post-sweeps 2,1,0 (a symmetric V-cycle), exact
// solve on level 1 (one unknown), every application starting from x = 0.
#include "st_internal.cuh"

namespace st {

namespace {

// ---------------------------------------------------------------------------------------
// coefficient table: class 0 -> (a, s) = (1, 0); class 1 + l -> (alpha, 2^l), l = 0..J
// ---------------------------------------------------------------------------------------
__global__ void k_make_coef(Coef<double>* coef, int K, int J, double alpha) {
  int nclass = J + 2;
  for (int e = threadIdx.x; e < nclass * (K + 1); e += blockDim.x) {
    int cls = e / (K + 1), k = e % (K + 1);
    double a = cls == 0 ? 1.0 : alpha;
    double s = cls == 0 ? 0.0 : ldexp(1.0, cls - 1);
    double h2 = ldexp(1.0, -2 * k);
    Coef<double> c;
    c.c = 4.0 * a + s * h2 / 2.0;
    c.ax = -a + s * h2 / 12.0;
    c.dg = s * h2 / 12.0;
    c.inv_c = 1.0 / c.c;
    coef[e] = c;
  }
}

template <typename T>
__device__ __forceinline__ Coef<T> slice_coef(const Coef<T>* coef, int coef_class, int slice, int J, int K,
                                              int level) {
  int cls = coef_class >= 0 ? coef_class : 1 + wavelet_row_level(slice, J);
  return coef[cls * (K + 1) + level];
}

// ---------------------------------------------------------------------------------------
// Gauss-Seidel: NSW full 3-colour sweeps of one slice tile, staged in shared memory.
// The block owns an interior tile of TX x TY points and loads a halo of H = 3 NSW points:
// colour step t (0-based) updates every point within H - 1 - t of the tile, so after the
// last step the interior is exactly what sequential colour-by-colour sweeps over the whole
// slice produce.  Each lane owns three consecutive columns, of which exactly one has the
// active colour in any row, so every lane does one update per row and step.
// ---------------------------------------------------------------------------------------
constexpr int kWR = 96;  // region width = 32 lanes x 3 columns

// The sweep is out of place (x_in -> x_out): a block's halo overlaps its neighbours' interiors,
// so reading and writing one buffer in the same launch would race.
template <typename T, int NSW, int HR, bool DIAG>
__global__ void __launch_bounds__(256) k_gs_sweep(T* __restrict__ x_out, const T* __restrict__ x_in,
                                                  const T* __restrict__ b, int n,
                                                  const Coef<T>* __restrict__ coef, int coef_class, int J,
                                                  int K, int level, int reverse, int zero_init) {
  constexpr int H = 3 * NSW;
  constexpr int TX = kWR - 2 * H;
  constexpr int TY = HR - 2 * H;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  T* bs = xs + HR * kWR;

  const int slice = blockIdx.z;
  const int64_t off = (int64_t)slice * n * n;
  T* xsl = x_out + off;
  const T* xin = x_in + off;
  const T* bsl = b + off;
  const int gx0 = blockIdx.x * TX - H;
  const int gy0 = blockIdx.y * TY - H;
  const Coef<T> cf = slice_coef(coef, coef_class, slice, J, K, level);

  for (int idx = threadIdx.x; idx < HR * kWR; idx += blockDim.x) {
    int ry = idx / kWR, rx = idx - ry * kWR;
    int gx = gx0 + rx, gy = gy0 + ry;
    bool in = gx >= 0 && gx < n && gy >= 0 && gy < n;
    int64_t gi = (int64_t)gy * n + gx;
    xs[idx] = (in && !zero_init) ? xin[gi] : T(0);
    bs[idx] = in ? bsl[gi] : T(0);
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll 1
  for (int t = 0; t < 3 * NSW; ++t) {
    const int tc = t % 3;
    const int colour = reverse ? 2 - tc : tc;
    const int lo = t + 1;
    const int ry_lo = max(lo, -gy0), ry_hi = min(HR - lo, n - gy0);
    const int rx_lo = max(lo, -gx0), rx_hi = min(kWR - lo, n - gx0);
    for (int ry = ry_lo + warp; ry < ry_hi; ry += nwarp) {
      const int gy = gy0 + ry;
      // colour (gx + gy + 2) mod 3 == colour  <=>  rx == colour - 2 - gy - gx0 (mod 3)
      int m = (colour - 2 - gy - gx0) % 3;
      m += (m < 0) ? 3 : 0;
      const int rx = 3 * lane + m;
      if (rx >= rx_lo && rx < rx_hi) {
        const int i = ry * kWR + rx;
        T s4 = (xs[i - 1] + xs[i + 1]) + (xs[i - kWR] + xs[i + kWR]);
        T v = bs[i] - cf.ax * s4;
        if (DIAG) v -= cf.dg * (xs[i + kWR + 1] + xs[i - kWR - 1]);
        xs[i] = v * cf.inv_c;
      }
    }
    __syncthreads();
  }

  for (int idx = threadIdx.x; idx < TY * TX; idx += blockDim.x) {
    int ty = idx / TX, tx = idx - ty * TX;
    int gx = gx0 + H + tx, gy = gy0 + H + ty;
    if (gx < n && gy < n) xsl[(int64_t)gy * n + gx] = xs[(ty + H) * kWR + tx + H];
  }
}

// r = b - C x on every point of every slice
template <typename T, bool DIAG>
__global__ void k_residual(T* __restrict__ r, const T* __restrict__ x, const T* __restrict__ b, int n,
                           const Coef<T>* __restrict__ coef, int coef_class, int J, int K, int level) {
  const int N = n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int slice = blockIdx.y;
  const int64_t off = (int64_t)slice * N;
  const T* xs = x + off;
  const Coef<T> cf = slice_coef(coef, coef_class, slice, J, K, level);
  const int iy = p / n, ix = p - iy * n;
  const T xw = ix > 0 ? xs[p - 1] : T(0);
  const T xe = ix < n - 1 ? xs[p + 1] : T(0);
  const T xsth = iy > 0 ? xs[p - n] : T(0);
  const T xn = iy < n - 1 ? xs[p + n] : T(0);
  T s4 = (xw + xe) + (xsth + xn);
  T v = b[off + p] - cf.ax * s4;
  if (DIAG) {
    const T xne = (ix < n - 1 && iy < n - 1) ? xs[p + n + 1] : T(0);
    const T xsw = (ix > 0 && iy > 0) ? xs[p - n - 1] : T(0);
    v -= cf.dg * (xne + xsw);
  }
  r[off + p] = v - cf.c * xs[p];
}

// coarse rhs = P^T r: coarse node (I, J) collects fine node (2I, 2J) with weight 1 and the
// midpoints of its six coarse edges (axis and (1,1) diagonal directions) with weight 1/2.
template <typename T>
__global__ void k_restrict(T* __restrict__ bc, const T* __restrict__ r, int nc) {
  const int Nc = nc * nc;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Nc) return;
  const int nf = 2 * nc + 1;
  const int slice = blockIdx.y;
  const T* rs = r + (int64_t)slice * nf * nf;
  const int cy = q / nc, cx = q - cy * nc;
  const int p = (2 * cy + 1) * nf + (2 * cx + 1);  // interior index of fine node (2I, 2J)
  T e = (rs[p - 1] + rs[p + 1]) + (rs[p - nf] + rs[p + nf]) + (rs[p + nf + 1] + rs[p - nf - 1]);
  bc[(int64_t)slice * Nc + q] = rs[p] + T(0.5) * e;
}

// x += P xc: nested P1 interpolation (coarse values at even-even fine nodes, averages of the
// two coarse end points at midpoints of horizontal, vertical and (1,1)-diagonal edges).
template <typename T>
__global__ void k_prolong_add(T* __restrict__ x, const T* __restrict__ xc, int nf) {
  const int N = nf * nf;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int nc = (nf - 1) / 2;
  const int slice = blockIdx.y;
  const T* cs = xc + (int64_t)slice * nc * nc;
  const int iy = p / nf, ix = p - iy * nf;
  const int i = ix + 1, j = iy + 1;  // fine grid indices
  // coarse value at coarse grid node (I, J) (zero on the boundary)
  auto cv = [&](int I, int Jc) -> T {
    return (I >= 1 && I <= nc && Jc >= 1 && Jc <= nc) ? cs[(Jc - 1) * nc + (I - 1)] : T(0);
  };
  T v;
  if ((i & 1) == 0 && (j & 1) == 0) {
    v = cv(i >> 1, j >> 1);
  } else if ((j & 1) == 0) {
    v = T(0.5) * (cv(i >> 1, j >> 1) + cv((i >> 1) + 1, j >> 1));
  } else if ((i & 1) == 0) {
    v = T(0.5) * (cv(i >> 1, j >> 1) + cv(i >> 1, (j >> 1) + 1));
  } else {
    v = T(0.5) * (cv(i >> 1, j >> 1) + cv((i >> 1) + 1, (j >> 1) + 1));
  }
  x[(int64_t)slice * N + p] += v;
}

// exact solve on level 1 (one unknown per slice)
template <typename T>
__global__ void k_coarse1(T* __restrict__ x, const T* __restrict__ b, int nslices, const Coef<T>* __restrict__ coef,
                          int coef_class, int J, int K) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  const Coef<T> cf = slice_coef(coef, coef_class, s, J, K, 1);
  x[s] = b[s] * cf.inv_c;
}

constexpr int kHR64 = 64;

template <bool DIAG>
cudaError_t gs_sweep(const st_handle_s* h, int k, int nslices, int cls, double* x_out, const double* x_in,
                     const double* b, bool reverse, bool zero_init) {
  constexpr int NSW = 1, HR = kHR64, H = 3 * NSW;
  const int n = (1 << k) - 1;
  const int TX = kWR - 2 * H, TY = HR - 2 * H;
  dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, nslices);
  const size_t smem = 2 * sizeof(double) * HR * kWR;
  // profiled: the finest level, which carries three quarters of the sweep work
  const bool prof = (k == h->K) && prof_start(h);
  k_gs_sweep<double, NSW, HR, DIAG><<<grid, 256, smem, h->stream>>>(x_out, x_in, b, n, h->coef, cls, h->J, h->K,
                                                                     k, reverse ? 1 : 0, zero_init ? 1 : 0);
  count_launch(h);
  if (prof) {
    // per point and sweep: 3 adds + 1 fma + 1 mul (+ 1 add + 1 fma with diagonal couplings);
    // bytes: read x and b, write x (x is not read on a zero-initialised sweep)
    const double pts = (double)n * n * nslices;
    prof_stop(h, pts * NSW * (DIAG ? 7.0 : 5.0), pts * sizeof(double) * (zero_init ? 2.0 : 3.0));
  }
  return cudaGetLastError();
}

// One V-cycle on level k.  xb[0], xb[1] are the level's two iterate buffers and *cur the one
// holding the iterate; every sweep moves it to the other buffer.
template <bool DIAG>
cudaError_t vcycle(const st_handle_s* h, int k, int nslices, int cls, double* const xb[2], int* cur,
                   const double* b, bool x_is_zero) {
  const st::MGLevels& L = h->mg;
  const int n = (1 << k) - 1;
  const int N = n * n;
  cudaError_t e;
  if (k == L.kmin) {
    k_coarse1<double><<<(nslices + 255) / 256, 256, 0, h->stream>>>(xb[*cur], b, nslices, h->coef, cls, h->J, h->K);
    count_launch(h);
    return cudaGetLastError();
  }
  for (int s = 0; s < h->cfg.n_pre; ++s) {
    if ((e = gs_sweep<DIAG>(h, k, nslices, cls, xb[*cur ^ 1], xb[*cur], b, false, x_is_zero && s == 0)) != cudaSuccess)
      return e;
    *cur ^= 1;
  }
  if (h->cfg.n_pre == 0 && x_is_zero) {
    // nothing smoothed yet: the iterate must hold zeros before the residual is formed
    if ((e = cudaMemsetAsync(xb[*cur], 0, sizeof(double) * (size_t)N * nslices, h->stream)) != cudaSuccess) return e;
  }
  double* x = xb[*cur];
  dim3 g1((N + 255) / 256, nslices);
  k_residual<double, DIAG><<<g1, 256, 0, h->stream>>>(L.res[k], x, b, n, h->coef, cls, h->J, h->K, k);
  const int nc = (1 << (k - 1)) - 1;
  dim3 g2((nc * nc + 255) / 256, nslices);
  k_restrict<double><<<g2, 256, 0, h->stream>>>(L.bc[k - 1], L.res[k], nc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  double* const xcb[2] = {L.xc[k - 1], L.xc2[k - 1]};
  int ccur = 0;
  if ((e = vcycle<DIAG>(h, k - 1, nslices, cls, xcb, &ccur, L.bc[k - 1], true)) != cudaSuccess) return e;
  k_prolong_add<double><<<g1, 256, 0, h->stream>>>(x, xcb[ccur], n);
  count_launch(h, 3);  // residual, restriction, prolongation
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int s = 0; s < h->cfg.n_post; ++s) {
    if ((e = gs_sweep<DIAG>(h, k, nslices, cls, xb[*cur ^ 1], xb[*cur], b, true, false)) != cudaSuccess) return e;
    *cur ^= 1;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_make_coef(Coef<double>* coef, int K, int J, double alpha, cudaStream_t s) {
  k_make_coef<<<1, 256, 0, s>>>(coef, K, J, alpha);
  return cudaGetLastError();
}

cudaError_t mg_set_attributes() {
  const int smem = 2 * sizeof(double) * kHR64 * kWR;
  cudaError_t e = cudaFuncSetAttribute(k_gs_sweep<double, 1, kHR64, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gs_sweep<double, 1, kHR64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem);
}

cudaError_t mg_apply(const st_handle_s* h, int nslices, int coef_class, const double* b, double* x) {
  // class 0 (K_x: s = 0) has no diagonal couplings; the K_l classes do
  const bool diag = coef_class != 0;
  double* const xb[2] = {x, h->Xalt};
  int cur = 0;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < h->cfg.n_vcycles; ++c) {
    e = diag ? vcycle<true>(h, h->K, nslices, coef_class, xb, &cur, b, c == 0)
             : vcycle<false>(h, h->K, nslices, coef_class, xb, &cur, b, c == 0);
    if (e != cudaSuccess) return e;
  }
  const size_t bytes = sizeof(double) * (size_t)h->Nx * nslices;
  if (h->cfg.n_vcycles == 0) return cudaMemsetAsync(x, 0, bytes, h->stream);
  // an odd total number of sweeps leaves the iterate in the alternate buffer
  if (cur == 1) return cudaMemcpyAsync(x, h->Xalt, bytes, cudaMemcpyDeviceToDevice, h->stream);
  return cudaSuccess;
}

}  // namespace st
