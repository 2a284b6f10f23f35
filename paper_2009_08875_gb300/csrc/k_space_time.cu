// Kronecker-structured operators of the Schur complement (Lemma 4.2, applied row-wise as in
// Eq. 5.1): P1 mass / stiffness stencils on each time slice fused with the tridiagonal time
// matrices, the S epilogue, and the three-point wavelet transform along time (Eq. 3.1).
#include "st_internal.cuh"

namespace st {

namespace {

// ---------------------------------------------------------------------------------------
// spatial stencils on one slice (interior index p = iy n + ix; outside the grid = 0)
//   M_x: h^2/12 [6 at p; 1 at (+-1,0), (0,+-1), (1,1), (-1,-1)]
//   A_x: [4 at p; -1 at (+-1,0), (0,+-1)]
// ---------------------------------------------------------------------------------------
struct Nbr {
  double c, w, e, s, nn, ne, sw;
};

__device__ __forceinline__ Nbr load_nbr(const double* __restrict__ u, int p, int ix, int iy, int n) {
  Nbr v;
  v.c = u[p];
  v.w = ix > 0 ? u[p - 1] : 0.0;
  v.e = ix < n - 1 ? u[p + 1] : 0.0;
  v.s = iy > 0 ? u[p - n] : 0.0;
  v.nn = iy < n - 1 ? u[p + n] : 0.0;
  v.ne = (ix < n - 1 && iy < n - 1) ? u[p + n + 1] : 0.0;
  v.sw = (ix > 0 && iy > 0) ? u[p - n - 1] : 0.0;
  return v;
}

__device__ __forceinline__ double mass_of(const Nbr& v, double mh) {
  return mh * (6.0 * v.c + (((v.w + v.e) + (v.s + v.nn)) + (v.ne + v.sw)));
}

__device__ __forceinline__ double stiff_of(const Nbr& v) { return 4.0 * v.c - ((v.w + v.e) + (v.s + v.nn)); }

// tridiagonal time matrices on the uniform P1 mesh (h = 2^-J), row i of N_t:
//   A_t = 1/h tridiag(-1, 2, -1), ends 1/h;   M_t = h/6 tridiag(1, 4, 1), ends h/3;
//   L[i,j] = int Phi_j' Phi_i: L[i,i-1] = -1/2, L[i,i+1] = 1/2, L[0,0] = -1/2, L[N-1,N-1] = 1/2.
struct Tri {
  double m, c, p;  // coefficients of rows i-1, i, i+1
};

struct TimeConsts {
  double inv_h, h6, h3, h23;  // 1/h, h/6, h/3, 2h/3
};

__device__ __forceinline__ Tri tri_At(int i, int Nt, const TimeConsts& k) {
  bool end = (i == 0 || i == Nt - 1);
  return Tri{i > 0 ? -k.inv_h : 0.0, end ? k.inv_h : 2.0 * k.inv_h, i < Nt - 1 ? -k.inv_h : 0.0};
}
__device__ __forceinline__ Tri tri_Mt(int i, int Nt, const TimeConsts& k) {
  bool end = (i == 0 || i == Nt - 1);
  return Tri{i > 0 ? k.h6 : 0.0, end ? k.h3 : k.h23, i < Nt - 1 ? k.h6 : 0.0};
}
__device__ __forceinline__ double L_diag(int i, int Nt) { return i == 0 ? -0.5 : (i == Nt - 1 ? 0.5 : 0.0); }
__device__ __forceinline__ Tri tri_L(int i, int Nt) {
  return Tri{i > 0 ? -0.5 : 0.0, L_diag(i, Nt), i < Nt - 1 ? 0.5 : 0.0};
}
__device__ __forceinline__ Tri tri_LT(int i, int Nt) {
  // L^T[i, i-1] = L[i-1, i] = 1/2, L^T[i, i+1] = L[i+1, i] = -1/2
  return Tri{i > 0 ? 0.5 : 0.0, L_diag(i, Nt), i < Nt - 1 ? -0.5 : 0.0};
}

__device__ __forceinline__ double tri_dot(const Tri& t, double a, double b, double c) {
  return t.m * a + t.c * b + t.p * c;
}

// mode 0 (S):  Y1 = A_t (U M) + L^T (U A),  Y2 = L (U M) + M_t (U A)
// mode 1 (rhs): Y1 = L^T (G M),             Y2 = M_t (G M)
// One thread per spatial point walks a chunk of time rows, keeping the stencil results of
// rows i-1, i, i+1 in registers (the chunk edges recompute one halo row).
__global__ void __launch_bounds__(256) k_timemix(const double* __restrict__ U, double* __restrict__ Y1,
                                                 double* __restrict__ Y2, int n, int Nt, int chunk, double mh,
                                                 TimeConsts tk, int mode) {
  const int N = n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int iy = p / n, ix = p - iy * n;
  const int i0 = blockIdx.y * chunk;
  const int i1 = min(Nt, i0 + chunk);
  double um_m = 0.0, ua_m = 0.0, um_c, ua_c, um_p = 0.0, ua_p = 0.0;
  if (i0 > 0) {
    Nbr v = load_nbr(U + (int64_t)(i0 - 1) * N, p, ix, iy, n);
    um_m = mass_of(v, mh);
    ua_m = stiff_of(v);
  }
  {
    Nbr v = load_nbr(U + (int64_t)i0 * N, p, ix, iy, n);
    um_c = mass_of(v, mh);
    ua_c = stiff_of(v);
  }
  for (int i = i0; i < i1; ++i) {
    if (i + 1 < Nt) {
      Nbr v = load_nbr(U + (int64_t)(i + 1) * N, p, ix, iy, n);
      um_p = mass_of(v, mh);
      ua_p = mode == 0 ? stiff_of(v) : 0.0;
    } else {
      um_p = 0.0;
      ua_p = 0.0;
    }
    double y1, y2;
    if (mode == 0) {
      y1 = tri_dot(tri_At(i, Nt, tk), um_m, um_c, um_p) + tri_dot(tri_LT(i, Nt), ua_m, ua_c, ua_p);
      y2 = tri_dot(tri_L(i, Nt), um_m, um_c, um_p) + tri_dot(tri_Mt(i, Nt, tk), ua_m, ua_c, ua_p);
    } else {
      y1 = tri_dot(tri_LT(i, Nt), um_m, um_c, um_p);
      y2 = tri_dot(tri_Mt(i, Nt, tk), um_m, um_c, um_p);
    }
    Y1[(int64_t)i * N + p] = y1;
    Y2[(int64_t)i * N + p] = y2;
    um_m = um_c;
    ua_m = ua_c;
    um_c = um_p;
    ua_c = ua_p;
  }
}

// Z_i = M X1_i + A X2_i (+ M row0 on row 0): the Schur epilogue (K_x already applied)
__global__ void __launch_bounds__(256) k_epilogue(const double* __restrict__ X1, const double* __restrict__ X2,
                                                  const double* __restrict__ row0, double* __restrict__ Z, int n,
                                                  double mh) {
  const int N = n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int i = blockIdx.y;
  const int iy = p / n, ix = p - iy * n;
  const int64_t off = (int64_t)i * N;
  double z = mass_of(load_nbr(X1 + off, p, ix, iy, n), mh) + stiff_of(load_nbr(X2 + off, p, ix, iy, n));
  if (i == 0 && row0 != nullptr) z += mass_of(load_nbr(row0, p, ix, iy, n), mh);
  Z[off + p] = z;
}

__global__ void __launch_bounds__(256) k_apply_A(const double* __restrict__ X, double* __restrict__ Y, int n) {
  const int N = n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int iy = p / n, ix = p - iy * n;
  const int64_t off = (int64_t)blockIdx.y * N;
  Y[off + p] = stiff_of(load_nbr(X + off, p, ix, iy, n));
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
__global__ void k_wsynth(const double* __restrict__ C, const double* __restrict__ D, double* __restrict__ X,
                         int64_t Nx, int j, int J, double s) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= Nx) return;
  const int k = blockIdx.y;  // 0 .. 2^j
  const int nw = 1 << j;
  const int sf = 1 << (J - j - 1);  // fine stride in rows
  const double ck = C[(int64_t)(2 * k) * sf * Nx + p];
  const double dk = k < nw ? D[(int64_t)(2 * k + 1) * sf * Nx + p] : 0.0;
  const double dkm = k > 0 ? D[(int64_t)(2 * k - 1) * sf * Nx + p] : 0.0;
  const double aL = (k == 0) ? 1.0 : 0.5;    // psi_k's weight at fine node 2k
  const double aR = (k == nw) ? 1.0 : 0.5;   // psi_{k-1}'s weight at fine node 2k
  X[(int64_t)(2 * k) * sf * Nx + p] = ck - s * (aR * dkm + aL * dk);
  if (k < nw) {
    const double ck1 = C[(int64_t)(2 * k + 2) * sf * Nx + p];
    X[(int64_t)(2 * k + 1) * sf * Nx + p] = 0.5 * (ck + ck1) + s * dk;
  }
}

// analysis stage: c = P_j^T x, d = Q_j^T x.  Thread (k, p) writes c_k (and d_k if k < 2^j).
// C and D may be the same buffer (stage 0 writes c_0 and d_0 into w); the rows written are disjoint.
__global__ void k_wanal(const double* __restrict__ Xf, double* C, double* D, int64_t Nx,
                        int j, int J, double s) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= Nx) return;
  const int k = blockIdx.y;
  const int nw = 1 << j;
  const int sf = 1 << (J - j - 1);
  const double x0 = Xf[(int64_t)(2 * k) * sf * Nx + p];
  const double xm = k > 0 ? Xf[(int64_t)(2 * k - 1) * sf * Nx + p] : 0.0;
  const double xp = k < nw ? Xf[(int64_t)(2 * k + 1) * sf * Nx + p] : 0.0;
  C[(int64_t)(2 * k) * sf * Nx + p] = x0 + 0.5 * (xm + xp);
  if (k < nw) {
    const double x2 = Xf[(int64_t)(2 * k + 2) * sf * Nx + p];
    const double aL = (k == 0) ? 1.0 : 0.5;
    const double aR = (k == nw - 1) ? 1.0 : 0.5;
    D[(int64_t)(2 * k + 1) * sf * Nx + p] = s * (xp - aL * x0 - aR * x2);
  }
}

TimeConsts time_consts(int J) {
  const double h = ldexp(1.0, -J);
  return TimeConsts{ldexp(1.0, J), h / 6.0, h / 3.0, 2.0 * h / 3.0};
}

}  // namespace

cudaError_t launch_timemix(const st_handle_s* h, int mode, const double* U, double* Y) {
  const int n = h->n;
  const int N = n * n;
  const int chunk = 32;
  dim3 grid((N + 255) / 256, (int)((h->Nt + chunk - 1) / chunk));
  const double hx = ldexp(1.0, -h->K);
  k_timemix<<<grid, 256, 0, h->stream>>>(U, Y, Y + h->Nt * h->Nx, n, (int)h->Nt, chunk, hx * hx / 12.0,
                                         time_consts(h->J), mode);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_epilogue(const st_handle_s* h, const double* X, const double* row0, double* Z) {
  const int n = h->n;
  const int N = n * n;
  dim3 grid((N + 255) / 256, (int)h->Nt);
  const double hx = ldexp(1.0, -h->K);
  k_epilogue<<<grid, 256, 0, h->stream>>>(X, X + h->Nt * h->Nx, row0, Z, n, hx * hx / 12.0);
  count_launch(h);
  return cudaGetLastError();
}

cudaError_t launch_apply_A(const st_handle_s* h, int nrows, const double* X, double* Y) {
  const int n = h->n;
  const int N = n * n;
  dim3 grid((N + 255) / 256, nrows);
  k_apply_A<<<grid, 256, 0, h->stream>>>(X, Y, n);
  count_launch(h);
  return cudaGetLastError();
}

// u = W w.  Stage j reads c_j from the previous stage's output (stage 0: from w) and d_j from
// w, and writes level j+1 into a buffer that differs from the one it reads; the last stage
// writes u.  Scratch buffers V1/V2 alternate.
cudaError_t wavelet_synth(const st_handle_s* h, const double* w, double* u) {
  const int J = h->J;
  const int64_t Nx = h->Nx;
  const unsigned gx = (unsigned)((Nx + 255) / 256);
  const double* src = w;
  for (int j = 0; j < J; ++j) {
    double* dst = (j == J - 1) ? u : (((J - 1 - j) & 1) ? h->V1 : h->V2);
    dim3 grid(gx, (1u << j) + 1);
    k_wsynth<<<grid, 256, 0, h->stream>>>(src, w, dst, Nx, j, J, sqrt(ldexp(1.0, j + 1)));
    count_launch(h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = dst;
  }
  return cudaSuccess;
}

// w = W^T u = diag(W_{J-1}^T, I) M_{J-1}^T u: stage J-1 first.  c goes to alternating
// scratch buffers, d straight to w; stage 0 writes c_0 into rows 0 and 2^J of w.
cudaError_t wavelet_anal(const st_handle_s* h, const double* u, double* w) {
  const int J = h->J;
  const int64_t Nx = h->Nx;
  const unsigned gx = (unsigned)((Nx + 255) / 256);
  const double* src = u;
  for (int j = J - 1; j >= 0; --j) {
    double* cdst = (j == 0) ? w : ((j & 1) ? h->V1 : h->V2);
    dim3 grid(gx, (1u << j) + 1);
    k_wanal<<<grid, 256, 0, h->stream>>>(src, cdst, w, Nx, j, J, sqrt(ldexp(1.0, j + 1)));
    count_launch(h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = cdst;
  }
  return cudaSuccess;
}

}  // namespace st
