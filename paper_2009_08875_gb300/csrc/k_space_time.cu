// Kronecker-structured operators of the Schur complement (Lemma 4.2, applied row-wise as in
// Eq. 5.1): P1 mass / stiffness stencils on each time slice fused with the tridiagonal time
// matrices, the S epilogue, and the three-point wavelet transform along time (Eq. 3.1).
#include "st_internal.cuh"

namespace st {

namespace {

// ---------------------------------------------------------------------------------------
// spatial stencils on one slice (outside the grid = 0), as neighbour sums (c, s1, s2, s3):
// 2D (interior index p = iy n + ix): s1 = west + east, s2 = south + north, s3 = (1,1) + (-1,-1)
//   M_x: h^2/12 [6 at p; 1 at the six neighbours]
//   A_x: the 7-point stencil of <D grad, grad> + c M_x (Stencil7 over (c, s1, s2, s3); the
//        heat equation's [4; -1 at (+-1,0), (0,+-1)] when D = Id, c = 0)
// 3D, the unit cube with Kuhn tetrahedra (p = (iz n + iy) n + ix): s1 = the 6 axis neighbours,
//   s2 = the 6 face-diagonal neighbours +-(1,1,0), +-(1,0,1), +-(0,1,1), s3 = the 2 body-diagonal
//   neighbours +-(1,1,1)
//   M_x: h^3 [2/5; 1/20 on s1, 1/30 on s2, 1/20 on s3];  A_x: h [6; -1 on s1] + c M_x
// ---------------------------------------------------------------------------------------
template <typename T>
struct Sums {
  T c, s1, s2, s3;
};

template <typename T, int DIM>
__device__ __forceinline__ Sums<T> load_nbr(const T* __restrict__ u, int64_t p, int ix, int iy, int iz, int n) {
  Sums<T> v;
  v.c = u[p];
  const bool xm = ix > 0, xp = ix < n - 1, ym = iy > 0, yp = iy < n - 1;
  if (DIM == 2) {
    v.s1 = (xm ? u[p - 1] : T(0)) + (xp ? u[p + 1] : T(0));
    v.s2 = (ym ? u[p - n] : T(0)) + (yp ? u[p + n] : T(0));
    v.s3 = ((xp && yp) ? u[p + n + 1] : T(0)) + ((xm && ym) ? u[p - n - 1] : T(0));
  } else {
    const int64_t nn = (int64_t)n * n;
    const bool zm = iz > 0, zp = iz < n - 1;
    v.s1 = ((xm ? u[p - 1] : T(0)) + (xp ? u[p + 1] : T(0))) + ((ym ? u[p - n] : T(0)) + (yp ? u[p + n] : T(0))) +
           ((zm ? u[p - nn] : T(0)) + (zp ? u[p + nn] : T(0)));
    v.s2 = (((xp && yp) ? u[p + 1 + n] : T(0)) + ((xm && ym) ? u[p - 1 - n] : T(0))) +
           (((xp && zp) ? u[p + 1 + nn] : T(0)) + ((xm && zm) ? u[p - 1 - nn] : T(0))) +
           (((yp && zp) ? u[p + n + nn] : T(0)) + ((ym && zm) ? u[p - n - nn] : T(0)));
    v.s3 = ((xp && yp && zp) ? u[p + 1 + n + nn] : T(0)) + ((xm && ym && zm) ? u[p - 1 - n - nn] : T(0));
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T stiff_of(const Sums<T>& v, const Stencil7<T>& a) {
  return a.c0 * v.c + a.cx * v.s1 + a.cy * v.s2 + a.cd * v.s3;
}

// mass stencil sm: 2D passes (6 mh, mh, mh, mh) and uses mh (6 c + ((s1 + s2) + s3)); 3D the
// general form
template <typename T, int DIM>
__device__ __forceinline__ T mass_of(const Sums<T>& v, const Stencil7<T>& sm) {
  if (DIM == 2) return sm.cx * (T(6) * v.c + ((v.s1 + v.s2) + v.s3));
  return stiff_of(v, sm);
}

// grid coordinates of interior index p (p < n^DIM < 2^31: 32-bit unsigned division, a fraction of
// the cost of 64-bit division)
template <int DIM>
__device__ __forceinline__ void coords_of(int64_t p, int n, int& ix, int& iy, int& iz) {
  const unsigned q = (unsigned)p, un = (unsigned)n;
  if (DIM == 2) {
    iy = (int)(q / un);
    ix = (int)(q - (unsigned)iy * un);
    iz = 0;
  } else {
    const unsigned r = q / un;
    ix = (int)(q - r * un);
    iz = (int)(r / un);
    iy = (int)(r - (unsigned)iz * un);
  }
}

// tridiagonal time matrices on the uniform P1 mesh (h = 2^-J), row i of N_t:
//   A_t = 1/h tridiag(-1, 2, -1), ends 1/h;   M_t = h/6 tridiag(1, 4, 1), ends h/3;
//   L[i,j] = int Phi_j' Phi_i: L[i,i-1] = -1/2, L[i,i+1] = 1/2, L[0,0] = -1/2, L[N-1,N-1] = 1/2.
template <typename T>
struct Tri {
  T m, c, p;  // coefficients of rows i-1, i, i+1
};

template <typename T>
struct TimeConsts {
  T inv_h, h6, h3, h23;  // 1/h, h/6, h/3, 2h/3
};

template <typename T>
__device__ __forceinline__ Tri<T> tri_At(int i, int Nt, const TimeConsts<T>& k) {
  bool end = (i == 0 || i == Nt - 1);
  return Tri<T>{i > 0 ? -k.inv_h : T(0), end ? k.inv_h : T(2) * k.inv_h, i < Nt - 1 ? -k.inv_h : T(0)};
}
template <typename T>
__device__ __forceinline__ Tri<T> tri_Mt(int i, int Nt, const TimeConsts<T>& k) {
  bool end = (i == 0 || i == Nt - 1);
  return Tri<T>{i > 0 ? k.h6 : T(0), end ? k.h3 : k.h23, i < Nt - 1 ? k.h6 : T(0)};
}
template <typename T>
__device__ __forceinline__ T L_diag(int i, int Nt) {
  return i == 0 ? T(-0.5) : (i == Nt - 1 ? T(0.5) : T(0));
}
template <typename T>
__device__ __forceinline__ Tri<T> tri_L(int i, int Nt) {
  return Tri<T>{i > 0 ? T(-0.5) : T(0), L_diag<T>(i, Nt), i < Nt - 1 ? T(0.5) : T(0)};
}
template <typename T>
__device__ __forceinline__ Tri<T> tri_LT(int i, int Nt) {
  // L^T[i, i-1] = L[i-1, i] = 1/2, L^T[i, i+1] = L[i+1, i] = -1/2
  return Tri<T>{i > 0 ? T(0.5) : T(0), L_diag<T>(i, Nt), i < Nt - 1 ? T(-0.5) : T(0)};
}

template <typename T>
__device__ __forceinline__ T tri_dot(const Tri<T>& t, T a, T b, T c) {
  return t.m * a + t.c * b + t.p * c;
}

// mode 0 (S):  Y1 = A_t (U M) + L^T (U A),  Y2 = L (U M) + M_t (U A)
// mode 1 (rhs): Y1 = L^T (G M),             Y2 = M_t (G M)
// One thread per spatial point walks a chunk of time rows, keeping the stencil results of
// rows i-1, i, i+1 in registers (the chunk edges recompute one halo row).  Output rows are the
// global rows row0 .. row0 + nrows - 1 of the N_t rows (Y row i - row0); U holds global row j at
// its row j - row0 + halo (halo = 1: a time-sharded block with one neighbour row each side).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_timemix(const T* __restrict__ U, T* __restrict__ Y1, T* __restrict__ Y2,
                                                 int n, int Nt, int row0, int nrows, int halo, int chunk,
                                                 Stencil7<T> sm, Stencil7<T> sa, TimeConsts<T> tk, int mode,
                                                 int lshape) {
  const int64_t N = DIM == 2 ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int64_t poff = (int64_t)blockIdx.z * Nt * N;  // problem blockIdx.z of the batch
  U += poff;
  Y1 += poff;
  Y2 += poff;
  // global row i lives at U row i - row0 + halo and is output at Y row i - row0
  auto urow = [&](int i) { return U + (int64_t)(i - row0 + halo) * N; };
  auto yoff = [&](int i) { return (int64_t)(i - row0) * N + p; };
  int ix, iy, iz;
  coords_of<DIM>(p, n, ix, iy, iz);
  const int i0 = row0 + blockIdx.y * chunk;
  const int i1 = min(row0 + nrows, i0 + chunk);
  if (DIM == 2 && outside_domain(ix, iy, n, lshape)) {  // nodes outside the domain stay zero
    for (int i = i0; i < i1; ++i) {
      Y1[yoff(i)] = T(0);
      Y2[yoff(i)] = T(0);
    }
    return;
  }
  T um_m = T(0), ua_m = T(0), um_c, ua_c, um_p = T(0), ua_p = T(0);
  if (i0 > 0) {
    Sums<T> v = load_nbr<T, DIM>(urow(i0 - 1), p, ix, iy, iz, n);
    um_m = mass_of<T, DIM>(v, sm);
    ua_m = stiff_of(v, sa);
  }
  {
    Sums<T> v = load_nbr<T, DIM>(urow(i0), p, ix, iy, iz, n);
    um_c = mass_of<T, DIM>(v, sm);
    ua_c = stiff_of(v, sa);
  }
  for (int i = i0; i < i1; ++i) {
    if (i + 1 < Nt) {
      Sums<T> v = load_nbr<T, DIM>(urow(i + 1), p, ix, iy, iz, n);
      um_p = mass_of<T, DIM>(v, sm);
      ua_p = mode == 0 ? stiff_of(v, sa) : T(0);
    } else {
      um_p = T(0);
      ua_p = T(0);
    }
    T y1, y2;
    if (mode == 0) {
      y1 = tri_dot(tri_At(i, Nt, tk), um_m, um_c, um_p) + tri_dot(tri_LT<T>(i, Nt), ua_m, ua_c, ua_p);
      y2 = tri_dot(tri_L<T>(i, Nt), um_m, um_c, um_p) + tri_dot(tri_Mt(i, Nt, tk), ua_m, ua_c, ua_p);
    } else {
      y1 = tri_dot(tri_LT<T>(i, Nt), um_m, um_c, um_p);
      y2 = tri_dot(tri_Mt(i, Nt, tk), um_m, um_c, um_p);
    }
    Y1[yoff(i)] = y1;
    Y2[yoff(i)] = y2;
    um_m = um_c;
    ua_m = ua_c;
    um_c = um_p;
    ua_c = ua_p;
  }
}

// Z_i = M X1_i + A X2_i (+ M row0 on row 0): the Schur epilogue (K_x already applied)
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_epilogue(const T* __restrict__ X1, const T* __restrict__ X2,
                                                  const T* __restrict__ row0, int64_t row0_stride, T* __restrict__ Z,
                                                  int n, int Nt, int first_row, Stencil7<T> sm, Stencil7<T> sa,
                                                  int lshape) {
  const int64_t N = DIM == 2 ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int i = blockIdx.y;
  const int64_t poff = (int64_t)blockIdx.z * Nt * N;  // problem blockIdx.z of the batch
  X1 += poff;
  X2 += poff;
  Z += poff;
  if (row0 != nullptr) row0 += blockIdx.z * row0_stride;
  int ix, iy, iz;
  coords_of<DIM>(p, n, ix, iy, iz);
  const int64_t off = (int64_t)i * N;
  if (DIM == 2 && outside_domain(ix, iy, n, lshape)) {
    Z[off + p] = T(0);
    return;
  }
  T z = mass_of<T, DIM>(load_nbr<T, DIM>(X1 + off, p, ix, iy, iz, n), sm) +
        stiff_of(load_nbr<T, DIM>(X2 + off, p, ix, iy, iz, n), sa);
  if (first_row + i == 0 && row0 != nullptr) z += mass_of<T, DIM>(load_nbr<T, DIM>(row0, p, ix, iy, iz, n), sm);
  Z[off + p] = z;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_apply_A(const T* __restrict__ X, T* __restrict__ Y, int n, Stencil7<T> sa,
                                                 int lshape) {
  const int64_t N = DIM == 2 ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= N) return;
  int ix, iy, iz;
  coords_of<DIM>(p, n, ix, iy, iz);
  const int64_t off = (int64_t)blockIdx.y * N;
  Y[off + p] = (DIM == 2 && outside_domain(ix, iy, n, lshape))
                   ? T(0)
                   : stiff_of(load_nbr<T, DIM>(X + off, p, ix, iy, iz, n), sa);
}

// ---------------------------------------------------------------------------------------
// The same stencils on the square (and the L-shape) with each thread computing QB consecutive
// points of one grid row: the three grid rows it needs are read once for all QB points (16 loads
// per input for 4 points instead of 28), and the grid coordinates come from the block indices.
// Same neighbour sums in the same order as load_nbr.
// ---------------------------------------------------------------------------------------
constexpr int QB = 4;     // points per thread
constexpr int kBT = 128;  // threads per block: 512 columns of one grid row

template <typename T>
struct RowBlock {  // the neighbour sums of the QB points (ix0 .. ix0 + QB - 1, iy)
  Sums<T> v[QB];
};

template <typename T>
__device__ __forceinline__ RowBlock<T> load_rows(const T* __restrict__ u, int ix0, int iy, int n) {
  // rows iy - 1 (columns ix0 - 1 .. ix0 + QB - 1), iy (ix0 - 1 .. ix0 + QB), iy + 1 (ix0 .. ix0 + QB)
  T lo[QB + 1], mid[QB + 2], hi[QB + 1];
  const bool ym = iy > 0, yp = iy < n - 1;
  const T* r0 = u + (int64_t)iy * n;
#pragma unroll
  for (int q = 0; q < QB + 2; ++q) {
    const int c = ix0 - 1 + q;
    const bool cin = c >= 0 && c < n;
    mid[q] = cin ? r0[c] : T(0);
    if (q < QB + 1) lo[q] = (cin && ym) ? r0[c - n] : T(0);
    if (q >= 1) hi[q - 1] = (cin && yp) ? r0[c + n] : T(0);
  }
  RowBlock<T> b;
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    // point ix0 + q: west mid[q], centre mid[q + 1], east mid[q + 2]; south lo[q + 1], north
    // hi[q]; (1,1) hi[q + 1]; (-1,-1) lo[q]
    b.v[q].c = mid[q + 1];
    b.v[q].s1 = mid[q] + mid[q + 2];
    b.v[q].s2 = lo[q + 1] + hi[q];
    b.v[q].s3 = hi[q + 1] + lo[q];
  }
  return b;
}

// Z_i = M X1_i + A X2_i (+ M row0 on row 0), as k_epilogue (DIM 2); grid (columns / 512, n, slices
// of all problems)
template <typename T>
__global__ void __launch_bounds__(kBT) k_epilogue_rows2(const T* __restrict__ X1, const T* __restrict__ X2,
                                                        const T* __restrict__ row0, int64_t row0_stride,
                                                        T* __restrict__ Z, int n, int Nt, Stencil7<T> sm,
                                                        Stencil7<T> sa, int lshape) {
  const int ix0 = QB * (blockIdx.x * kBT + threadIdx.x);
  if (ix0 >= n) return;
  const int iy = blockIdx.y;
  const int slice = blockIdx.z;  // problem slice / Nt, time row slice % Nt
  const int64_t off = (int64_t)slice * n * n;
  const RowBlock<T> a = load_rows(X1 + off, ix0, iy, n);
  const RowBlock<T> c = load_rows(X2 + off, ix0, iy, n);
  T z[QB];
#pragma unroll
  for (int q = 0; q < QB; ++q) z[q] = mass_of<T, 2>(a.v[q], sm) + stiff_of(c.v[q], sa);
  if (slice % Nt == 0 && row0 != nullptr) {
    const RowBlock<T> r = load_rows(row0 + (slice / Nt) * row0_stride, ix0, iy, n);
#pragma unroll
    for (int q = 0; q < QB; ++q) z[q] += mass_of<T, 2>(r.v[q], sm);
  }
  T* zr = Z + off + (int64_t)iy * n;
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    const int ix = ix0 + q;
    if (ix < n) zr[ix] = outside_domain(ix, iy, n, lshape) ? T(0) : z[q];
  }
}

// Y = A_x X on each slice, as k_apply_A (DIM 2)
template <typename T>
__global__ void __launch_bounds__(kBT) k_apply_A_rows2(const T* __restrict__ X, T* __restrict__ Y, int n,
                                                       Stencil7<T> sa, int lshape) {
  const int ix0 = QB * (blockIdx.x * kBT + threadIdx.x);
  if (ix0 >= n) return;
  const int iy = blockIdx.y;
  const int64_t off = (int64_t)blockIdx.z * n * n;
  const RowBlock<T> a = load_rows(X + off, ix0, iy, n);
  T* yr = Y + off + (int64_t)iy * n;
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    const int ix = ix0 + q;
    if (ix < n) yr[ix] = outside_domain(ix, iy, n, lshape) ? T(0) : stiff_of(a.v[q], sa);
  }
}

// ---------------------------------------------------------------------------------------
// three-point wavelet lifting along time, in-place row order (level-j nodes at rows that are
// multiples of 2^(J-j)).  Stage j maps level j (2^j + 1 nodes, coefficients c) plus the
// level-(j+1) wavelet coefficients d (2^j of them) to level j+1, M_j = [P_j | Q_j]:
//   P_j: coarse hat k = fine hat 2k + (fine hats 2k-1, 2k+1) / 2
//   Q_j: psi_k = s (fine hat 2k+1 - aL fine hat 2k - aR fine hat 2k+2), s = 2^((j+1)/2),
//        aL = 1 if 2k = 0 else 1/2, aR = 1 if 2k + 2 = 2^(j+1) else 1/2
// ---------------------------------------------------------------------------------------

// synthesis stage: x = P_j c + Q_j d.  Thread (k, p) writes fine nodes 2k and 2k+1.
template <typename T>
__global__ void k_wsynth(const T* __restrict__ C, const T* __restrict__ D, T* __restrict__ X, int64_t Nx, int j,
                         int J, T s) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= Nx) return;
  const int64_t poff = (int64_t)blockIdx.z * (((int64_t)1 << J) + 1) * Nx;  // problem of the batch
  C += poff;
  D += poff;
  X += poff;
  const int k = blockIdx.y;  // 0 .. 2^j
  const int nw = 1 << j;
  const int sf = 1 << (J - j - 1);  // fine stride in rows
  const T ck = C[(int64_t)(2 * k) * sf * Nx + p];
  const T dk = k < nw ? D[(int64_t)(2 * k + 1) * sf * Nx + p] : T(0);
  const T dkm = k > 0 ? D[(int64_t)(2 * k - 1) * sf * Nx + p] : T(0);
  const T aL = (k == 0) ? T(1) : T(0.5);    // psi_k's weight at fine node 2k
  const T aR = (k == nw) ? T(1) : T(0.5);   // psi_{k-1}'s weight at fine node 2k
  X[(int64_t)(2 * k) * sf * Nx + p] = ck - s * (aR * dkm + aL * dk);
  if (k < nw) {
    const T ck1 = C[(int64_t)(2 * k + 2) * sf * Nx + p];
    X[(int64_t)(2 * k + 1) * sf * Nx + p] = T(0.5) * (ck + ck1) + s * dk;
  }
}

// analysis stage: c = P_j^T x, d = Q_j^T x.  Thread (k, p) writes c_k (and d_k if k < 2^j).
// C and D may be the same buffer (stage 0 writes c_0 and d_0 into w); the rows written are disjoint.
template <typename T>
__global__ void k_wanal(const T* __restrict__ Xf, T* C, T* D, int64_t Nx, int j, int J, T s) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= Nx) return;
  const int64_t poff = (int64_t)blockIdx.z * (((int64_t)1 << J) + 1) * Nx;  // problem of the batch
  Xf += poff;
  C += poff;
  D += poff;
  const int k = blockIdx.y;
  const int nw = 1 << j;
  const int sf = 1 << (J - j - 1);
  const T x0 = Xf[(int64_t)(2 * k) * sf * Nx + p];
  const T xm = k > 0 ? Xf[(int64_t)(2 * k - 1) * sf * Nx + p] : T(0);
  const T xp = k < nw ? Xf[(int64_t)(2 * k + 1) * sf * Nx + p] : T(0);
  C[(int64_t)(2 * k) * sf * Nx + p] = x0 + T(0.5) * (xm + xp);
  if (k < nw) {
    const T x2 = Xf[(int64_t)(2 * k + 2) * sf * Nx + p];
    const T aL = (k == 0) ? T(1) : T(0.5);
    const T aR = (k == nw - 1) ? T(1) : T(0.5);
    D[(int64_t)(2 * k + 1) * sf * Nx + p] = s * (xp - aL * x0 - aR * x2);
  }
}

// A_x and M_x on the finest level of the handle, in element type T (the cube: Kuhn tetrahedra)
template <typename T>
Stencil7<T> fine_A(const st_handle_s* h) {
  const double hx = ldexp(1.0, -h->K);
  if (h->domain == 2) {
    const double m = h->phys.c * hx * hx * hx;
    return Stencil7<T>{(T)(6.0 * hx + 0.4 * m), (T)(-hx + m / 20.0), (T)(m / 30.0), (T)(m / 20.0)};
  }
  const Stencil7<double> a = operator_stencil(h->phys, 1.0, 0.0, hx);
  return Stencil7<T>{(T)a.c0, (T)a.cx, (T)a.cy, (T)a.cd};
}

template <typename T>
Stencil7<T> fine_M(const st_handle_s* h) {
  const double hx = ldexp(1.0, -h->K);
  if (h->domain == 2) {
    const double h3 = hx * hx * hx;
    return Stencil7<T>{(T)(0.4 * h3), (T)(h3 / 20.0), (T)(h3 / 30.0), (T)(h3 / 20.0)};
  }
  const T mh = (T)(hx * hx / 12.0);  // 2D: mass_of uses mh (6 c + (s1 + s2 + s3))
  return Stencil7<T>{T(6) * mh, mh, mh, mh};
}

template <typename T>
TimeConsts<T> time_consts(int J) {
  const double h = ldexp(1.0, -J);
  return TimeConsts<T>{(T)ldexp(1.0, J), (T)(h / 6.0), (T)(h / 3.0), (T)(2.0 * h / 3.0)};
}

}  // namespace

template <typename T>
cudaError_t launch_timemix(const st_handle_s* h, int nb, int mode, const T* U, T* Y) {
  const int n = h->n;
  const int64_t N = h->Nx;
  const int chunk = 32;
  dim3 grid((unsigned)((N + 255) / 256), (int)((h->Nt + chunk - 1) / chunk), nb);
  if (h->domain == 2)
    k_timemix<T, 3><<<grid, 256, 0, h->stream>>>(U, Y, Y + nb * h->Nt * h->Nx, n, (int)h->Nt, 0, (int)h->Nt, 0,
                                                 chunk, fine_M<T>(h),
                                                 fine_A<T>(h), time_consts<T>(h->J), mode, 0);
  else  // (a row-blocked binary32 variant, four points a thread, measured slower: fewer threads,
        // each walking its chunk of time rows)
    k_timemix<T, 2><<<grid, 256, 0, h->stream>>>(U, Y, Y + nb * h->Nt * h->Nx, n, (int)h->Nt, 0, (int)h->Nt, 0,
                                                 chunk, fine_M<T>(h),
                                                 fine_A<T>(h), time_consts<T>(h->J), mode, h->domain);
  count_launch(h);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_epilogue(const st_handle_s* h, int nb, const T* X, const T* row0, int64_t row0_stride, T* Z) {
  const int n = h->n;
  const int64_t N = h->Nx;
  dim3 grid((unsigned)((N + 255) / 256), (int)h->Nt, nb);
  if (h->domain == 2)
    k_epilogue<T, 3><<<grid, 256, 0, h->stream>>>(X, X + nb * h->Nt * h->Nx, row0, row0_stride, Z, n, (int)h->Nt, 0,
                                                  fine_M<T>(h), fine_A<T>(h), 0);
  else if (sizeof(T) == 4)  // binary32: row blocks (binary64 is bound by its arithmetic either way)
    k_epilogue_rows2<T><<<dim3((n + QB * kBT - 1) / (QB * kBT), n, (unsigned)(nb * h->Nt)), kBT, 0, h->stream>>>(
        X, X + nb * h->Nt * h->Nx, row0, row0_stride, Z, n, (int)h->Nt, fine_M<T>(h), fine_A<T>(h), h->domain);
  else
    k_epilogue<T, 2><<<grid, 256, 0, h->stream>>>(X, X + nb * h->Nt * h->Nx, row0, row0_stride, Z, n, (int)h->Nt, 0,
                                                  fine_M<T>(h), fine_A<T>(h), h->domain);
  count_launch(h);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_A(const st_handle_s* h, int nrows, const T* X, T* Y) {
  const int n = h->n;
  const int64_t N = h->Nx;
  dim3 grid((unsigned)((N + 255) / 256), nrows);
  if (h->domain == 2)
    k_apply_A<T, 3><<<grid, 256, 0, h->stream>>>(X, Y, n, fine_A<T>(h), 0);
  else if (sizeof(T) == 4)
    k_apply_A_rows2<T><<<dim3((n + QB * kBT - 1) / (QB * kBT), n, (unsigned)nrows), kBT, 0, h->stream>>>(
        X, Y, n, fine_A<T>(h), h->domain);
  else
    k_apply_A<T, 2><<<grid, 256, 0, h->stream>>>(X, Y, n, fine_A<T>(h), h->domain);
  count_launch(h);
  return cudaGetLastError();
}

// Time-sharded row blocks (one problem): the time mix for output rows row0 .. row0 + nrows - 1
// from U with one neighbour row each side (nrows + 2 rows; the rows outside 0 .. N_t - 1 are not
// read), and the epilogue of those rows (X: X1 block then X2 block of nrows rows each; the Gamma_0
// term only when the block holds row 0).
cudaError_t launch_timemix_rows(const st_handle_s* h, int mode, int row0, int nrows, const double* U, double* Y) {
  const int n = h->n;
  const int64_t N = h->Nx;
  const int chunk = 32;
  dim3 grid((unsigned)((N + 255) / 256), (unsigned)((nrows + chunk - 1) / chunk), 1);
  if (h->domain == 2)
    k_timemix<double, 3><<<grid, 256, 0, h->stream>>>(U, Y, Y + (int64_t)nrows * N, n, (int)h->Nt, row0, nrows, 1,
                                                      chunk, fine_M<double>(h), fine_A<double>(h),
                                                      time_consts<double>(h->J), mode, 0);
  else
    k_timemix<double, 2><<<grid, 256, 0, h->stream>>>(U, Y, Y + (int64_t)nrows * N, n, (int)h->Nt, row0, nrows, 1,
                                                      chunk, fine_M<double>(h), fine_A<double>(h),
                                                      time_consts<double>(h->J), mode, h->domain);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_epilogue_rows(const st_handle_s* h, int row0, int nrows, const double* X, const double* u_row0,
                                 double* Z) {
  const int n = h->n;
  const int64_t N = h->Nx;
  dim3 grid((unsigned)((N + 255) / 256), (unsigned)nrows, 1);
  if (h->domain == 2)
    k_epilogue<double, 3><<<grid, 256, 0, h->stream>>>(X, X + (int64_t)nrows * N, u_row0, 0, Z, n, nrows, row0,
                                                       fine_M<double>(h), fine_A<double>(h), 0);
  else
    k_epilogue<double, 2><<<grid, 256, 0, h->stream>>>(X, X + (int64_t)nrows * N, u_row0, 0, Z, n, nrows, row0,
                                                       fine_M<double>(h), fine_A<double>(h), h->domain);
  count_launch(h);
  return cudaGetLastError();
}

// u = W w.  Stage j reads c_j from the previous stage's output (stage 0: from w) and d_j from
// w, and writes level j+1 into a buffer that differs from the one it reads; the last stage
// writes u.  Scratch buffers V1/V2 alternate.
template <typename T>
cudaError_t wavelet_synth_n(const st_handle_s* h, int nb, int64_t Nx, const T* w, T* u) {
  const int J = h->J;
  const unsigned gx = (unsigned)((Nx + 255) / 256);
  T* V1 = reinterpret_cast<T*>(h->V1);
  T* V2 = reinterpret_cast<T*>(h->V2);
  const T* src = w;
  for (int j = 0; j < J; ++j) {
    T* dst = (j == J - 1) ? u : (((J - 1 - j) & 1) ? V1 : V2);
    dim3 grid(gx, (1u << j) + 1, nb);
    k_wsynth<T><<<grid, 256, 0, h->stream>>>(src, w, dst, Nx, j, J, (T)sqrt(ldexp(1.0, j + 1)));
    count_launch(h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = dst;
  }
  return cudaSuccess;
}

// w = W^T u = diag(W_{J-1}^T, I) M_{J-1}^T u: stage J-1 first.  c goes to alternating
// scratch buffers, d straight to w; stage 0 writes c_0 into rows 0 and 2^J of w.
template <typename T>
cudaError_t wavelet_anal_n(const st_handle_s* h, int nb, int64_t Nx, const T* u, T* w) {
  const int J = h->J;
  const unsigned gx = (unsigned)((Nx + 255) / 256);
  T* V1 = reinterpret_cast<T*>(h->V1);
  T* V2 = reinterpret_cast<T*>(h->V2);
  const T* src = u;
  for (int j = J - 1; j >= 0; --j) {
    T* cdst = (j == 0) ? w : ((j & 1) ? V1 : V2);
    dim3 grid(gx, (1u << j) + 1, nb);
    k_wanal<T><<<grid, 256, 0, h->stream>>>(src, cdst, w, Nx, j, J, (T)sqrt(ldexp(1.0, j + 1)));
    count_launch(h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = cdst;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t wavelet_synth(const st_handle_s* h, int nb, const T* w, T* u) {
  return wavelet_synth_n<T>(h, nb, h->Nx, w, u);
}

template <typename T>
cudaError_t wavelet_anal(const st_handle_s* h, int nb, const T* u, T* w) {
  return wavelet_anal_n<T>(h, nb, h->Nx, u, w);
}

// the transforms of an N_t x ncols block of columns (a time-sharded rank's share after a
// rows-to-columns transpose); ncols <= N_x
cudaError_t wavelet_cols(const st_handle_s* h, int synth, int64_t ncols, const double* in, double* out) {
  return synth ? wavelet_synth_n<double>(h, 1, ncols, in, out) : wavelet_anal_n<double>(h, 1, ncols, in, out);
}

#define ST_INSTANTIATE(T)                                                                           \
  template cudaError_t launch_timemix<T>(const st_handle_s*, int, int, const T*, T*);               \
  template cudaError_t launch_epilogue<T>(const st_handle_s*, int, const T*, const T*, int64_t, T*); \
  template cudaError_t launch_apply_A<T>(const st_handle_s*, int, const T*, T*);                    \
  template cudaError_t wavelet_synth<T>(const st_handle_s*, int, const T*, T*);                     \
  template cudaError_t wavelet_anal<T>(const st_handle_s*, int, const T*, T*);
ST_INSTANTIATE(double)
ST_INSTANTIATE(float)
#undef ST_INSTANTIATE

}  // namespace st
