// Time-slice-batched multigrid for C = a A_x + s M_x on the unit cube (Sec. 5.2, the 3D problem).
//
// Mesh: 2^k cubes per side, each cut into the six Kuhn tetrahedra along its (0,0,0)-(1,1,1)
// diagonal.  P1 on it couples a node with its 6 axis neighbours, the 6 face-diagonal neighbours
// +-(1,1,0), +-(1,0,1), +-(0,1,1) and the 2 body-diagonal neighbours +-(1,1,1) (the stiffness
// part only with the axis neighbours).  The coefficient table holds, per slice class and level,
// the centre c, axis ax, face-diagonal ay and body-diagonal dg coefficients (Coef<T>).
//
// Gauss-Seidel in four colours (i + j + k) mod 4 of the 1-based grid indices (no two coupled
// nodes share a colour: the couplings' index sums are +-1, +-2, +-3), pre-sweeps in colour order
// 0..3, post-sweeps 3..0 (a symmetric V-cycle), in place: one launch per colour, one thread per
// point of that colour, whose neighbours all have other colours.  The binary64 3D update costs
// 6 (K_x) or 14 (K_l) FP64 instructions per point, well above the machine balance, so reading
// the neighbours through L1/L2 instead of staging tiles costs little (ncu: the K_l colour step
// keeps the FP64 pipe 84% busy).  Restriction is P^T of the
// nested P1 prolongation (weight 1/2 at the 14 neighbours), the coarse level 1 has one unknown.
// The multigrid works in the Jacobi-scaled form of the 2D kernels (right-hand sides b' = b / c),
// in binary64, binary32, or double-float (ST_FP64_DF: mg_apply3_df).
#include "st_internal.cuh"

namespace st {
namespace {

template <typename T>
const Coef<T>* coef3(const st_handle_s* h);
template <>
const Coef<double>* coef3<double>(const st_handle_s* h) {
  return h->coef;
}
template <>
const Coef<float>* coef3<float>(const st_handle_s* h) {
  return h->coef32;
}
template <>
const Coef<df64>* coef3<df64>(const st_handle_s* h) {
  return h->coefdf;
}

template <typename T>
__device__ __forceinline__ Coef<T> coef_of(const Coef<T>* coef, int cls, int slice, int J, int K, int level) {
  return coef[slice_class(cls, slice, J) * (K + 1) + level];
}

// neighbour sums of point (ix, iy, iz) of an n^3 slice (zero outside the grid)
template <typename T>
struct Sums3 {
  T axis, face, body;
};

template <typename T, bool DIAG>
__device__ __forceinline__ Sums3<T> sums3(const T* __restrict__ x, int ix, int iy, int iz, int n) {
  const int64_t nn = (int64_t)n * n;
  const int64_t p = iz * nn + (int64_t)iy * n + ix;
  const bool xm = ix > 0, xp = ix < n - 1, ym = iy > 0, yp = iy < n - 1, zm = iz > 0, zp = iz < n - 1;
  Sums3<T> s;
  s.axis = ((xm ? x[p - 1] : T(0)) + (xp ? x[p + 1] : T(0))) + ((ym ? x[p - n] : T(0)) + (yp ? x[p + n] : T(0))) +
           ((zm ? x[p - nn] : T(0)) + (zp ? x[p + nn] : T(0)));
  if (DIAG) {
    s.face = (((xp && yp) ? x[p + 1 + n] : T(0)) + ((xm && ym) ? x[p - 1 - n] : T(0))) +
             (((xp && zp) ? x[p + 1 + nn] : T(0)) + ((xm && zm) ? x[p - 1 - nn] : T(0))) +
             (((yp && zp) ? x[p + n + nn] : T(0)) + ((ym && zm) ? x[p - n - nn] : T(0)));
    s.body = ((xp && yp && zp) ? x[p + 1 + n + nn] : T(0)) + ((xm && ym && zm) ? x[p - 1 - n - nn] : T(0));
  } else {
    s.face = T(0);
    s.body = T(0);
  }
  return s;
}

// one colour step: x = b' - (ax/c) S_axis - (ay/c) S_face - (dg/c) S_body at the points of colour
// `colour`; thread t of slice blockIdx.y handles the (t mod q)-th point of that colour in grid row
// t / q (q = ceil(n / 4) candidates per row)
template <typename T, bool DIAG>
__global__ void __launch_bounds__(256) k_gs3(T* __restrict__ x, const T* __restrict__ b, int n,
                                             const Coef<T>* __restrict__ coef, int cls, int J, int K, int level,
                                             int colour) {
  const int q = (n + 3) >> 2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)q * n * n) return;
  // 32-bit unsigned division (t < q n^2 < 2^31 for the cube's levels): a fraction of 64-bit's cost
  const unsigned row = (unsigned)t / (unsigned)q;
  const int m = (int)((unsigned)t - row * (unsigned)q);
  const int iz = (int)(row / (unsigned)n), iy = (int)row - iz * n;
  // colour of (ix, iy, iz) is (ix + iy + iz + 3) mod 4
  int ix0 = (colour - 3 - iy - iz) % 4;
  ix0 += ix0 < 0 ? 4 : 0;
  const int ix = ix0 + 4 * m;
  if (ix >= n) return;
  const int slice = blockIdx.y;
  const int64_t off = (int64_t)slice * n * n * n;
  const Coef<T> cf = coef_of(coef, cls, slice, J, K, level);
  const Sums3<T> s = sums3<T, DIAG>(x + off, ix, iy, iz, n);
  const int64_t p = off + ((int64_t)iz * n + iy) * n + ix;
  T v = b[p] - cf.axs * s.axis;
  if (DIAG) {
    v -= cf.ays * s.face;
    v -= cf.dgs * s.body;
  }
  x[p] = v;
}

// scaled residual r' = b' - x - (ax/c) S_axis - (ay/c) S_face - (dg/c) S_body
template <typename T, bool DIAG>
__global__ void __launch_bounds__(256) k_residual3(T* __restrict__ r, const T* __restrict__ x,
                                                   const T* __restrict__ b, int n, const Coef<T>* __restrict__ coef,
                                                   int cls, int J, int K, int level) {
  const int64_t N3 = (int64_t)n * n * n;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= N3) return;
  const unsigned pq = (unsigned)p, un = (unsigned)n, rq = pq / un;  // p < n^3 < 2^31
  const int ix = (int)(pq - rq * un), iy = (int)(rq % un), iz = (int)(rq / un);
  const int slice = blockIdx.y;
  const int64_t off = (int64_t)slice * N3;
  const Coef<T> cf = coef_of(coef, cls, slice, J, K, level);
  const Sums3<T> s = sums3<T, DIAG>(x + off, ix, iy, iz, n);
  T v = b[off + p] - cf.axs * s.axis;
  if (DIAG) {
    v -= cf.ays * s.face;
    v -= cf.dgs * s.body;
  }
  r[off + p] = v - x[off + p];
}

// coarse scaled right-hand side: (c / c_coarse) P^T r' -- the fine residual at the coarse node
// plus half of it at the 14 neighbours along the mesh's edge directions
template <typename T>
__global__ void __launch_bounds__(256) k_restrict3(T* __restrict__ bc, const T* __restrict__ r, int nf,
                                                   const Coef<T>* __restrict__ coef, int cls, int J, int K,
                                                   int level) {
  const int nc = (nf - 1) / 2;
  const int64_t Nc = (int64_t)nc * nc * nc;
  const int64_t pc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pc >= Nc) return;
  const unsigned pq = (unsigned)pc, un = (unsigned)nc, rq = pq / un;  // pc < nc^3 < 2^31
  const int cx = (int)(pq - rq * un), cy = (int)(rq % un), cz = (int)(rq / un);
  const int slice = blockIdx.y;
  const Coef<T> cf = coef_of(coef, cls, slice, J, K, level);
  const int64_t nn = (int64_t)nf * nf;
  const T* rs = r + (int64_t)slice * nn * nf;
  const int64_t f = (int64_t)(2 * cz + 1) * nn + (int64_t)(2 * cy + 1) * nf + (2 * cx + 1);
  const T axis = ((rs[f - 1] + rs[f + 1]) + (rs[f - nf] + rs[f + nf])) + (rs[f - nn] + rs[f + nn]);
  const T face = ((rs[f + 1 + nf] + rs[f - 1 - nf]) + (rs[f + 1 + nn] + rs[f - 1 - nn])) +
                 (rs[f + nf + nn] + rs[f - nf - nn]);
  const T body = rs[f + 1 + nf + nn] + rs[f - 1 - nf - nn];
  bc[(int64_t)slice * Nc + pc] = cf.rho * rs[f] + (T(0.5) * cf.rho) * ((axis + face) + body);
}

// x += P xc (prolong_value3, st_internal.cuh)
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add3(T* __restrict__ x, const T* __restrict__ xc, int nf) {
  const int64_t N3 = (int64_t)nf * nf * nf;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= N3) return;
  const unsigned pq = (unsigned)p, un = (unsigned)nf, rq = pq / un;  // p < nf^3 < 2^31
  const int ix = (int)(pq - rq * un), iy = (int)(rq % un), iz = (int)(rq / un);
  const int nc = (nf - 1) / 2;
  const int slice = blockIdx.y;
  x[(int64_t)slice * N3 + p] += prolong_value3<T>(xc + (int64_t)slice * nc * nc * nc, nc, ix + 1, iy + 1, iz + 1);
}

template <typename T, typename Tin = T>
__global__ void __launch_bounds__(256) k_scale_rhs3(T* __restrict__ bs, const Tin* __restrict__ b, int64_t N3,
                                                    const Coef<T>* __restrict__ coef, int cls, int J, int K) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= N3) return;
  const int slice = blockIdx.y;
  const Coef<T> cf = coef_of(coef, cls, slice, J, K, K);
  const int64_t i = (int64_t)slice * N3 + p;
  bs[i] = T(b[i]) * cf.inv_c;
}

// element i of a buffer of 8-byte double-float values becomes the binary64 value it holds
__global__ void k_widen_df3(void* buf, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const df64 v = reinterpret_cast<const df64*>(buf)[i];
    reinterpret_cast<double*>(buf)[i] = double(v);
  }
}

template <typename T>
__global__ void k_coarse1_3(T* __restrict__ x, const T* __restrict__ b, int nslices) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nslices) x[s] = b[s];  // one unknown: the scaled right-hand side is the solution
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

template <typename T, bool DIAG>
cudaError_t colour_sweep(const st_handle_s* h, int k, int nslices, int cls, T* x, const T* b, int colour) {
  const int n = (1 << k) - 1;
  const int64_t threads = (int64_t)((n + 3) >> 2) * n * n;
  const bool prof = (k == h->K) && colour == 0 && prof_start(h);
  k_gs3<T, DIAG><<<dim3(blocks_for(threads), nslices), 256, 0, h->stream>>>(x, b, n, coef3<T>(h), cls, h->J, h->K,
                                                                           k, colour);
  count_launch(h);
  if (prof) {
    // one colour of the sweep is timed; its work is a quarter of the sweep's
    const double pts = (double)n * n * n * nslices / 4.0;
    // FP64 instructions per point: 5 adds and 1 fma (K_x); 11 adds and 3 fmas with the mass
    // couplings of K_l (counted by ncu: the add / fma ratio of the launch is 3.67)
    prof_stop(h, (DIAG ? 1 : 0) + (sizeof(T) == 4 ? 2 : 0), pts * (DIAG ? 14.0 : 6.0), pts * sizeof(T) * 3.0);
  }
  return cudaGetLastError();
}

// One V-cycle on level k for the iterate x (in place) and scaled right-hand side b.
template <typename T, bool DIAG>
cudaError_t vcycle3(const st_handle_s* h, int k, int nslices, int cls, T* x, const T* b, bool x_is_zero) {
  const MGLevels& L = h->mg;
  const int n = (1 << k) - 1;
  const int64_t N3 = (int64_t)n * n * n;
  cudaError_t e;
  if (k == 1) {
    k_coarse1_3<T><<<(nslices + 255) / 256, 256, 0, h->stream>>>(x, b, nslices);
    count_launch(h);
    return cudaGetLastError();
  }
  if (x_is_zero && (e = cudaMemsetAsync(x, 0, sizeof(T) * N3 * nslices, h->stream)) != cudaSuccess) return e;
  for (int s = 0; s < h->cfg.n_pre; ++s)
    for (int c = 0; c < 4; ++c)
      if ((e = colour_sweep<T, DIAG>(h, k, nslices, cls, x, b, c)) != cudaSuccess) return e;
  // residual into the level's scratch (the alternate buffer on the finest level)
  T* r = k == h->K ? reinterpret_cast<T*>(h->Xalt) : reinterpret_cast<T*>(L.xc2[k]);
  k_residual3<T, DIAG><<<dim3(blocks_for(N3), nslices), 256, 0, h->stream>>>(r, x, b, n, coef3<T>(h), cls, h->J,
                                                                           h->K, k);
  count_launch(h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nc = (1 << (k - 1)) - 1;
  const int64_t Nc = (int64_t)nc * nc * nc;
  T* bc = reinterpret_cast<T*>(L.bc[k - 1]);
  T* xc = reinterpret_cast<T*>(L.xc[k - 1]);
  k_restrict3<T><<<dim3(blocks_for(Nc), nslices), 256, 0, h->stream>>>(bc, r, n, coef3<T>(h), cls, h->J, h->K, k);
  count_launch(h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = vcycle3<T, DIAG>(h, k - 1, nslices, cls, xc, bc, true)) != cudaSuccess) return e;
  k_prolong_add3<T><<<dim3(blocks_for(N3), nslices), 256, 0, h->stream>>>(x, xc, n);
  count_launch(h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int s = 0; s < h->cfg.n_post; ++s)
    for (int c = 3; c >= 0; --c)
      if ((e = colour_sweep<T, DIAG>(h, k, nslices, cls, x, b, c)) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

template <typename T>
cudaError_t mg_apply3(const st_handle_s* h, int nslices, int coef_class, const T* b, T* x) {
  // K_x (class 0) couples only the axis neighbours unless c > 0; the K_l classes always have
  // the mass couplings
  const bool diag = coef_class != 0 || h->diag0;
  const int64_t N3 = h->Nx;
  T* bs = reinterpret_cast<T*>(h->Bs);
  k_scale_rhs3<T><<<dim3(blocks_for(N3), nslices), 256, 0, h->stream>>>(bs, b, N3, coef3<T>(h), coef_class, h->J,
                                                                       h->K);
  count_launch(h);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (h->cfg.n_vcycles == 0) return cudaMemsetAsync(x, 0, sizeof(T) * N3 * nslices, h->stream);
  for (int c = 0; c < h->cfg.n_vcycles; ++c) {
    e = diag ? vcycle3<T, true>(h, h->K, nslices, coef_class, x, bs, c == 0)
             : vcycle3<T, false>(h, h->K, nslices, coef_class, x, bs, c == 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// binary64 in and out, the multigrid in double-float (ST_FP64_DF): the iterate lives in x's memory
// (8 bytes a value either way) and is widened to binary64 in place at the end
cudaError_t mg_apply3_df(const st_handle_s* h, int nslices, int coef_class, const double* b, double* x) {
  using D = df64;
  const bool diag = coef_class != 0 || h->diag0;
  const int64_t N3 = h->Nx;
  D* bs = reinterpret_cast<D*>(h->Bs);
  D* xd = reinterpret_cast<D*>(x);
  k_scale_rhs3<D, double><<<dim3(blocks_for(N3), nslices), 256, 0, h->stream>>>(bs, b, N3, coef3<D>(h), coef_class,
                                                                              h->J, h->K);
  count_launch(h);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (h->cfg.n_vcycles == 0) return cudaMemsetAsync(x, 0, sizeof(double) * N3 * nslices, h->stream);
  for (int c = 0; c < h->cfg.n_vcycles; ++c) {
    e = diag ? vcycle3<D, true>(h, h->K, nslices, coef_class, xd, bs, c == 0)
             : vcycle3<D, false>(h, h->K, nslices, coef_class, xd, bs, c == 0);
    if (e != cudaSuccess) return e;
  }
  k_widen_df3<<<(unsigned)((N3 * nslices + 255) / 256), 256, 0, h->stream>>>(x, N3 * nslices);
  count_launch(h);
  return cudaGetLastError();
}

template cudaError_t mg_apply3<double>(const st_handle_s*, int, int, const double*, double*);
template cudaError_t mg_apply3<float>(const st_handle_s*, int, int, const float*, float*);

}  // namespace st
