// Gauss-Seidel sweeps of the time-slice-batched binary32 multigrid (k_mg.cu) in wide register
// tiles with paired arithmetic: the same three-colour sweeps as k_gs_sweep and k_gs_reg, two
// points of one colour per lane and row updated by one packed binary32 instruction (Blackwell's
// add / fma on float pairs).  The kernels are instantiated in k_gs_wide_*.cu, one translation
// unit per storage type and sweep count, so that they compile in parallel.
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

#include "df64.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

// ---------------------------------------------------------------------------------------
// A block's threads form row groups of NL lanes (whole warps, NL = 32, or half-warps, NL = 16):
// the block holds a region of 6 NL columns x (groups x R) rows of one slice, group w owning the
// region rows w R .. w R + R - 1 and its lane l the columns 6 l .. 6 l + 5 of them ("warp" and
// "lane" below mean the group and the lane in it; shuffles run within the group).  Columns
// 6 l + e and 6 l + e + 3 have the same colour ((i + j) mod 3), so in every row the two points
// of the active colour sit in one register pair x[r][m] = (column 6 l + m, column 6 l + m + 3),
// m = the active element, and every neighbour sum of the update is a pair as well: the update
// x = b' - (a_x/c)(W + E) - (a_y/c)(S + N) - (d/c)(NE + SW) of the Jacobi-scaled system runs as
// packed adds and fmas on both points at once.  Horizontal neighbours come from the lane's own
// pairs or, across a lane boundary, one shuffle per pair; vertical neighbours from the rows above
// and below in registers or, at the edge of a warp's rows, from the neighbouring warp's edge row
// (shared memory, double-buffered by step parity, one barrier per colour step).  The scaled
// right-hand side b' sits in shared memory (read once per point and colour step).
//
// Placement: the region lies inside the grid (n at least its width and height), clamped against the
// grid's edges, so no point of it is outside the grid and no update is masked.  On a side where
// the region ends at the grid's boundary the missing neighbours are the Dirichlet zeros, which
// is exact; on a side inside the grid the region carries a halo of H = 3 NSW points whose
// missing neighbours are taken from wherever is convenient (zeros, or the lane's own values);
// the error this makes travels one point per colour step, so after the 3 NSW steps the points
// at least H from such a side - the block's tile - are exactly what sequential colour-by-colour
// sweeps give.  Every point is updated with the same operations in the same order as in the
// other kernels (fma(-a_x/c, W + E, b'), then fma(-a_y/c, S + N, .), then fma(-d/c, NE + SW, .)),
// and a packed fma rounds each half once, like its scalar counterpart: bitwise the same sweeps.
// ---------------------------------------------------------------------------------------

constexpr int kWW = 192;  // region width: 32 lanes x 6 columns
#ifndef ST_WIDE_PROL_DIRECT
#define ST_WIDE_PROL_DIRECT 1
#endif
constexpr bool kProlDirect = ST_WIDE_PROL_DIRECT;
#ifndef ST_WIDE_ASYNC_B0
#define ST_WIDE_ASYNC_B0 0
#endif

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// The Gauss-Seidel update value of pair m (columns 6 l + m and 6 l + m + 3) of row r of a warp's
// R rows: b' - (a_x/c)(W + E) - (a_y/c)(S + N) [- (d/c)(NE + SW)], with the neighbours of the
// current iterate.  bs: b' of the warp's rows, bs[r * 96 + k * 32 + lane] = the pair k of the
// lane in row r.  below / above: the edge rows of the warps underneath and on top, in the same
// pair layout (zeros past the region).  zl / zr: the lane's west / east neighbour across the
// region's edge is the grid boundary (a zero).  r and m are constants once inlined in an
// unrolled loop.
template <int NL, int R, bool DIAG>
__device__ __forceinline__ float2 pair_update(const float2 (&x)[R][3], int r, int m, const float2* __restrict__ bs,
                                              const float2* __restrict__ below, const float2* __restrict__ above,
                                              int lane, bool zl, bool zr, float2 nax, float2 nay, float2 ndg) {
  constexpr int kR1 = R - 1;
  const int rs = r > 0 ? r - 1 : 0;
  const int rn = r < kR1 ? r + 1 : kR1;
  // west and east pairs (columns 6 l + m -+ 1 and 6 l + m + 3 -+ 1)
  float2 W, E;
  if (m == 0) {
    const float t = __shfl_up_sync(0xffffffffu, x[r][2].y, 1, NL);
    W = make_float2(zl ? 0.f : t, x[r][2].x);
  } else {
    W = x[r][(m + 2) % 3];
  }
  if (m == 2) {
    const float t = __shfl_down_sync(0xffffffffu, x[r][0].x, 1, NL);
    E = make_float2(x[r][0].y, zr ? 0.f : t);
  } else {
    E = x[r][(m + 1) % 3];
  }
  const float2 S = (r > 0) ? x[rs][m] : below[m * NL + lane];
  const float2 N = (r < kR1) ? x[rn][m] : above[m * NL + lane];
  float2 v = fma2(nax, add2(W, E), bs[r * 3 * NL + m * NL + lane]);
  v = fma2(nay, add2(S, N), v);
  if (DIAG) {
    // (1,1) neighbours: the row above shifted east; (-1,-1): the row below shifted west
    float2 NE, SW;
    if (r < kR1) {
      if (m == 2) {
        const float t = __shfl_down_sync(0xffffffffu, x[rn][0].x, 1, NL);
        NE = make_float2(x[rn][0].y, zr ? 0.f : t);
      } else {
        NE = x[rn][(m + 1) % 3];
      }
    } else {
      if (m == 2) {
        const float t = above[lane + 1].x;  // the last lane reads the next pair's slot: unused (zr or halo)
        NE = make_float2(above[lane].y, zr ? 0.f : t);
      } else {
        NE = above[((m + 1) % 3) * NL + lane];
      }
    }
    if (r > 0) {
      if (m == 0) {
        const float t = __shfl_up_sync(0xffffffffu, x[rs][2].y, 1, NL);
        SW = make_float2(zl ? 0.f : t, x[rs][2].x);
      } else {
        SW = x[rs][(m + 2) % 3];
      }
    } else {
      if (m == 0) {
        const float t = below[2 * NL + lane - 1].y;  // lane 0 reads the previous pair's slot: unused (zl or halo)
        SW = make_float2(zl ? 0.f : t, below[2 * NL + lane].x);
      } else {
        SW = below[((m + 2) % 3) * NL + lane];
      }
    }
    v = fma2(ndg, add2(NE, SW), v);
  }
  return v;
}

// One colour step on a warp's R rows.  P is the active element of the warp's first row (row r:
// m(r) = (P - r) mod 3); the step overwrites the active pair of every row with its update value.
template <int NL, int R, bool DIAG, int P>
__device__ __forceinline__ void wide_step(float2 (&x)[R][3], const float2* __restrict__ bs,
                                          const float2* __restrict__ below, const float2* __restrict__ above,
                                          int lane, bool zl, bool zr, float2 nax, float2 nay, float2 ndg) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int m = ((P - (r % 3)) + 3) % 3;  // a constant once the loop is unrolled
    x[r][m] = pair_update<NL, R, DIAG>(x, r, m, bs, below, above, lane, zl, zr, nax, nay, ndg);
  }
}

// The scaled residual r' = b' - C' x (C' = D^-1 C: the update value minus the point's own value)
// of every point of a warp's rows, written over b' in shared memory (pair layout; b' of a row is
// read only for that row's residual, and before its slot is overwritten).  (The points of the
// last colour step have residual exactly 0, but skipping them in these unrolled rows measured
// slower than forming them.)
template <int NL, int R, bool DIAG>
__device__ __forceinline__ void wide_residual(const float2 (&x)[R][3], float2* __restrict__ bs,
                                              const float2* __restrict__ below, const float2* __restrict__ above,
                                              int lane, bool zl, bool zr, float2 nax, float2 nay, float2 ndg) {
  const float2 mone = make_float2(-1.f, -1.f);
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 v = pair_update<NL, R, DIAG>(x, r, k, bs, below, above, lane, zl, zr, nax, nay, ndg);
      bs[r * 3 * NL + k * NL + lane] = fma2(x[r][k], mone, v);  // v - x, rounded once
    }
  }
}

// The restriction of the scaled residual to the coarse points whose fine centre lies in the
// block's tile: D_c^-1 P^T D r' = rho r'(centre) + (rho / 2) ((r'_W + r'_E) + (r'_S + r'_N) +
// (r'_NE + r'_SW)), rho = c / c_coarse (nested P1: the six fine neighbours along the coarse
// edges carry weight 1/2).  A warp takes the centres in its own rows: rows r = PY, PY + 2, ...
// (odd grid rows), and in a lane's columns the elements PA, PA + 2, PA + 4 (odd grid columns), so
// every shared-memory offset is a constant.  rs: the residuals of the region in pair layout
// (float index 2 ((e mod 3) 32 + lane) + e / 3 of element e of a lane in a row of 192 floats).
template <typename G, int NL, int R, int RH, int PA, int PY>
__device__ __forceinline__ void wide_restrict(const float* __restrict__ rs, G* __restrict__ bcs, int nc, int warp,
                                              int lane, int gyw, int gx_lane, int tx0, int tx1, int ty0, int ty1,
                                              float rho, float hrho) {
  auto at = [&](int row, int e) -> float {  // residual at row `row` of the region, element e of this lane
    row = row < 0 ? 0 : (row >= RH ? RH - 1 : row);  // clamped: only for centres outside the tile
    const int ln = e < 0 ? lane - 1 : (e > 5 ? lane + 1 : lane);
    const int ee = e < 0 ? 5 : (e > 5 ? 0 : e);
    return rs[row * 6 * NL + 2 * ((ee % 3) * NL + ln) + ee / 3];
  };
  const int ry0 = warp * R;
#pragma unroll
  for (int r = PY; r < R; r += 2) {
    const int gy = gyw + r;
    if (gy < ty0 || gy >= ty1) continue;  // uniform in the row group
    const int cy = (gy - 1) >> 1;
#pragma unroll
    for (int e = PA; e < 6; e += 2) {
      const int gx = gx_lane + e;
      const int row = ry0 + r;
      const float c = at(row, e);
      const float sum = ((at(row, e - 1) + at(row, e + 1)) + (at(row - 1, e) + at(row + 1, e))) +
                        (at(row + 1, e + 1) + at(row - 1, e - 1));
      if (gx >= tx0 && gx < tx1) bcs[(int64_t)cy * nc + ((gx - 1) >> 1)] = G(__fmaf_rn(rho, c, hrho * sum));
    }
  }
}

// x += P xc on a warp's R rows (the coarse-grid correction of the V-cycle; nested P1: the average
// of the coarse values at the two ends of the coarse edge whose midpoint the fine node is, the
// same node twice at even-even nodes).  cw: the coarse values staged row by row (CW a row) from
// the coarse node under the lane's element 0 of the warp's first row.  With PA = (x0 + 1) mod 2
// and PY = (y0 + 1) mod 2 the coarse offsets of every element are constants: element e of row r
// reads coarse rows (r + PY) / 2 and that + (r + PY) mod 2, columns (PA + e) / 2 and that +
// (PA + e) mod 2.  At the points of the first colour step's colour the sum is formed but never
// read (that step overwrites them reading only the other colours).
template <int R, int CW, int PA, int PY>
__device__ __forceinline__ void wide_add_prol(float2 (&x)[R][3], const float* __restrict__ cw) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int j0 = (r + PY) >> 1, j1 = j0 + ((r + PY) & 1);
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int i0 = (PA + e) >> 1, i1 = i0 + ((PA + e) & 1);
      const float c = 0.5f * (cw[j0 * CW + i0] + cw[j1 * CW + i1]);
      if (e < 3)
        x[r][e].x += c;
      else
        x[r][e - 3].y += c;
    }
    // keep the shared loads of later rows from being hoisted here (registers: x already holds the
    // whole region)
    asm volatile("" ::: "memory");
  }
}

// The same with the coarse values read straight from global memory into registers: the lane's
// columns need the coarse columns I0 .. I0 + 3 (1-based, I0 = the coarse node under its element 0)
// and the warp's rows the coarse rows J0 .. J0 + R / 2 (zero outside 1 .. nc); the loads go out
// with the fine loads, and no barrier or staging is needed.
template <typename G, int R, int PA, int PY>
__device__ __forceinline__ void wide_add_prol_direct(float2 (&x)[R][3], const G* __restrict__ xcs, int nc, int I0,
                                                     int J0) {
  constexpr int JR = R / 2 + 1;
  float cv[JR][4];
#pragma unroll
  for (int jr = 0; jr < JR; ++jr) {
    const int Jc = J0 + jr;
    const bool rowok = Jc >= 1 && Jc <= nc;
    const int64_t rowbase = (int64_t)(Jc - 1) * nc - 1;  // + I: the 1-based coarse node (Jc, I)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int I = I0 + c;
      cv[jr][c] = (rowok && I >= 1 && I <= nc) ? float(xcs[rowbase + I]) : 0.f;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int j0 = (r + PY) >> 1, j1 = j0 + ((r + PY) & 1);
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int i0 = (PA + e) >> 1, i1 = i0 + ((PA + e) & 1);
      const float c = 0.5f * (cv[j0][i0] + cv[j1][i1]);
      if (e < 3)
        x[r][e].x += c;
      else
        x[r][e - 3].y += c;
    }
  }
}

// The first colour step of a sweep from x = 0: every neighbour is zero, so x = b'.
template <int NL, int R, int P>
__device__ __forceinline__ void wide_step_first(float2 (&x)[R][3], const float2* __restrict__ bs, int lane) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int m = ((P - (r % 3)) + 3) % 3;
    x[r][m] = bs[r * 3 * NL + m * NL + lane];
  }
}

// Tiles along one axis of n grid points (n >= W): regions of W points, tiles of W - 2 M points
// inside the grid, but the first and the last tile W - M wide (a region that ends at the grid's
// boundary needs no margin there; the last one ends at n and is at most W - M wide).  Tile b is
// [t, e), its region starts at o = clamp(t - M, 0, n - W): the tile lies at least M inside every
// side of its region that is not the grid's boundary.
__host__ __device__ inline int wide_ntiles(int n, int W, int M) {
  const int w0 = W - M, ti = W - 2 * M;
  const int rest = n - 2 * w0;
  return 2 + (rest > 0 ? (rest + ti - 1) / ti : 0);
}
__device__ __forceinline__ void wide_tile(int b, int nb, int n, int W, int M, int& t, int& e, int& o) {
  const int w0 = W - M, ti = W - 2 * M;
  t = b == 0 ? 0 : w0 + (b - 1) * ti;
  e = b == nb - 1 ? n : w0 + b * ti;
  o = min(max(t - M, 0), n - W);
}

// dynamic shared memory of one block of NWARP warps in row groups of NL lanes (NVW = 32 NWARP /
// NL groups of R rows, RH = NVW R region rows): b' (RH rows x 3 NL pairs), the edge rows (2
// parities x NVW groups x 2 rows x 3 NL pairs; also the coarse values of the prolongation before
// the first step), and a zero row of 3 NL pairs
template <int NL, int R, int NWARP>
constexpr size_t wide_smem() {
  constexpr int NVW = 32 * NWARP / NL;
  return sizeof(float2) * (size_t)(NVW * R * 3 * NL + 2 * NVW * 2 * 3 * NL + 3 * NL);
}

// The kernel body for one parity class of block regions: PA = (x0 + 1) mod 2, PY = (y0 + 1) mod 2
// fix the coarse offsets of the prolongation (PROL); every class is its own code path, so the
// registers of one do not add to another's.
template <typename G, int NL, int NSW, int R, int NWARP, bool ASYNCB, bool PDIR, bool DIAG, bool PROL, bool RESTR,
          bool SCALE, int PA, int PY>
__device__ __forceinline__ void wide_body(G* __restrict__ x_out, const G* __restrict__ x_in, const G* __restrict__ b,
                                          const G* __restrict__ xc, G* __restrict__ bc,
                                          const float* __restrict__ braw, G* __restrict__ bsc, int n,
                                          const Coef<float>* __restrict__ coef, int coef_class, int J, int K,
                                          int level, int reverse, int zero_init) {
  constexpr int H = 3 * NSW;
  // row groups of NL lanes (a warp, or half a warp): NVW groups of R rows; regions of W columns
  constexpr int NVW = 32 * NWARP / NL, RH = NVW * R, W = 6 * NL, P3 = 3 * NL;
  static_assert(NL == 32 || R % 3 == 0, "half-warp groups must share their colour-step branch: R % 3 == 0");
  // binary32 storage: b' may come by asynchronous copies, which frees the registers the direct
  // prolongation needs; bfloat16 storage stages the coarse values in shared memory
  constexpr bool kF32 = std::is_same<G, float>::value;
  // tile margin: H, and 2 more when the launch also restricts the residual (the residual at the
  // fine neighbours of the tile's coarse centres needs the iterate one point further out)
  constexpr int M = H + (RESTR ? 2 : 0);
  constexpr int CW = W / 2 + 2, CH = RH / 2 + 2;  // coarse values under the region (PROL)
  static_assert(CW * CH <= 2 * NVW * 2 * P3 * 2, "coarse values fit in the edge-row space");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* bsh = reinterpret_cast<float2*>(smem_raw);  // [RH][3][NL]
  float2* edge = bsh + RH * P3;                        // [2][NVW][2][3][NL]
  float2* zrow = edge + 2 * NVW * 2 * P3;              // [3][NL]
  float* ct = reinterpret_cast<float*>(edge);          // [CH][CW] before the first step

  // lane within the row group, and the group ("warp" below)
  const int lane = threadIdx.x % NL, warp = threadIdx.x / NL;
  const int slice = blockIdx.z;
  const int64_t off = (int64_t)slice * n * n;
  // the block's tile and its region, clamped into the grid
  int tx0, tx1, x0, ty0, ty1, y0;
  wide_tile(blockIdx.x, gridDim.x, n, W, M, tx0, tx1, x0);
  wide_tile(blockIdx.y, gridDim.y, n, RH, M, ty0, ty1, y0);
  const int ry0 = warp * R;
  const int gyw = y0 + ry0;       // grid row of the warp's first row
  const int cb = x0 + 6 * lane;   // grid column of the lane's element 0
  const bool zl = lane == 0 && x0 == 0;
  const bool zr = lane == NL - 1 && x0 + W == n;
  const Coef<float> cf = slice_coef(coef, coef_class, slice, J, K, level);
  const float2 nax = make_float2(-cf.axs, -cf.axs), nay = make_float2(-cf.ays, -cf.ays);
  const float2 ndg = make_float2(-cf.dgs, -cf.dgs);
  for (int i = threadIdx.x; i < P3; i += blockDim.x) zrow[i] = make_float2(0.f, 0.f);

  // load: x into registers (0 from x = 0) and b' into shared memory, in the pair layout
  float2 x[R][3];
  {
    const G* xw = x_in + off + (int64_t)gyw * n + cb;
    const G* bg = b + off + (int64_t)gyw * n + cb;
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float2* d = &bsh[(ry0 + r) * P3 + k * NL + lane];
        if constexpr ((ASYNCB || (PROL && PDIR)) && kF32) {
          // binary32: asynchronous 4-byte copies straight into the pair slots (no registers held)
          const unsigned dx = (unsigned)__cvta_generic_to_shared(&d->x);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dx), "l"(bg + (int64_t)r * n + k));
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dx + 4u), "l"(bg + (int64_t)r * n + k + 3));
        } else if constexpr (SCALE) {
          // the finest level's b' = b / c formed here (what k_scale_rhs writes); the tile's part
          // is written out after the colour steps
          const float* br = braw + off + (int64_t)(gyw + r) * n + cb;
          *d = make_float2(float(G(br[k] * cf.inv_c)), float(G(br[k + 3] * cf.inv_c)));
        } else {
          *d = make_float2(float(bg[(int64_t)r * n + k]), float(bg[(int64_t)r * n + k + 3]));
        }
        x[r][k] = zero_init ? make_float2(0.f, 0.f)
                            : make_float2(float(xw[(int64_t)r * n + k]), float(xw[(int64_t)r * n + k + 3]));
      }
    }
    // each thread's copies are complete here; the first step's barrier publishes them to the block
    if constexpr ((ASYNCB || (PROL && PDIR)) && kF32) asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  if (PROL && PDIR && kF32) {
    const int nc = (n - 1) / 2;
    wide_add_prol_direct<G, R, PA, PY>(x, xc + (int64_t)slice * nc * nc, nc, ((x0 + 1) >> 1) + 3 * lane,
                                       ((y0 + 1) >> 1) + (ry0 >> 1));
  } else if (PROL) {
    // the coarse values under the region, coarse row by coarse row (coarse interior indices
    // Ib .. Ib + CW - 1 by Jb .. Jb + CH - 1, zero outside 1 .. nc), then x += P xc
    const int nc = (n - 1) / 2;
    const int Ib = (x0 + 1) >> 1, Jb = (y0 + 1) >> 1;
    const G* xcs = xc + (int64_t)slice * nc * nc;
    for (int jj = warp; jj < CH; jj += NVW) {
      const int Jc = Jb + jj;
      const bool rowok = Jc >= 1 && Jc <= nc;
      const G* src = xcs + (int64_t)(Jc - 1) * nc - 1;  // indexed by the 1-based I
      for (int ii = lane; ii < CW; ii += NL) {
        const int I = Ib + ii;
        ct[jj * CW + ii] = (rowok && I >= 1 && I <= nc) ? float(src[I]) : 0.f;
      }
    }
    __syncthreads();
    wide_add_prol<R, CW, PA, PY>(x, ct + (ry0 >> 1) * CW + 3 * lane);
    __syncthreads();  // ct (the edge-row space) is read before the first step writes it
  }

  const float2* bw = bsh + ry0 * P3;
#pragma unroll 1
  for (int t = 0; t < 3 * NSW; ++t) {
    const int colour = reverse ? 2 - t % 3 : t % 3;
    float2* ed = edge + ((t & 1) * NVW + warp) * 2 * P3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ed[k * NL + lane] = x[0][k];
      ed[P3 + k * NL + lane] = x[R - 1][k];
    }
    __syncthreads();
    const float2* below = warp > 0 ? edge + ((t & 1) * NVW + warp - 1) * 2 * P3 + P3 : zrow;
    const float2* above = warp < NVW - 1 ? edge + ((t & 1) * NVW + warp + 1) * 2 * P3 : zrow;
    int P = (colour - 2 - gyw - x0) % 3;  // active element in the warp's first row
    P += (P < 0) ? 3 : 0;
    if (!PROL && zero_init && t == 0) {
      if (P == 0)
        wide_step_first<NL, R, 0>(x, bw, lane);
      else if (P == 1)
        wide_step_first<NL, R, 1>(x, bw, lane);
      else
        wide_step_first<NL, R, 2>(x, bw, lane);
    } else if (P == 0) {
      wide_step<NL, R, DIAG, 0>(x, bw, below, above, lane, zl, zr, nax, nay, ndg);
    } else if (P == 1) {
      wide_step<NL, R, DIAG, 1>(x, bw, below, above, lane, zl, zr, nax, nay, ndg);
    } else {
      wide_step<NL, R, DIAG, 2>(x, bw, below, above, lane, zl, zr, nax, nay, ndg);
    }
  }

  if (SCALE) {
    // b' of the tile's points for the launches that follow, one group row at a time with lane l
    // at the columns l + NL j (coalesced), read from the pair layout in shared memory before the
    // residual overwrites it
    const float* bf = reinterpret_cast<const float*>(bsh) + ry0 * 2 * P3;
    // column c = lane + NL j of a row is element e = c mod 6 of lane c / 6: its float index in
    // the pair layout, a lane constant
    int sp[6];
    bool in[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int c = lane + NL * j, e = c % 6;
      sp[j] = 2 * ((e % 3) * NL + c / 6) + e / 3;
      in[j] = x0 + c >= tx0 && x0 + c < tx1;
    }
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      const int gy = gyw + r;
      if (gy < ty0 || gy >= ty1) continue;  // uniform in the row group
      G* row = bsc + off + (int64_t)gy * n + x0 + lane;
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if (in[j]) row[NL * j] = G(bf[r * 2 * P3 + sp[j]]);
    }
  }
  if (RESTR) {
    // the residual of the smoothed iterate over the region (exact on the tile widened by one
    // point), then its restriction to the coarse points of the tile: the coarse level's scaled
    // right-hand side, with no pass of its own over x and b'
    // the residual is that of the iterate as stored: round it to the storage type first (a
    // no-op for binary32; bfloat16 storage keeps 8 bits)
    if constexpr (!kF32) {
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) x[r][k] = make_float2(float(G(x[r][k].x)), float(G(x[r][k].y)));
    }
    constexpr int t = 3 * NSW;  // the next step parity's edge buffer
    float2* ed = edge + ((t & 1) * NVW + warp) * 2 * P3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ed[k * NL + lane] = x[0][k];
      ed[P3 + k * NL + lane] = x[R - 1][k];
    }
    __syncthreads();
    const float2* below = warp > 0 ? edge + ((t & 1) * NVW + warp - 1) * 2 * P3 + P3 : zrow;
    const float2* above = warp < NVW - 1 ? edge + ((t & 1) * NVW + warp + 1) * 2 * P3 : zrow;
    wide_residual<NL, R, DIAG>(x, bsh + ry0 * P3, below, above, lane, zl, zr, nax, nay, ndg);
    __syncthreads();
    const int nc = (n - 1) / 2;
    wide_restrict<G, NL, R, RH, PA, PY>(reinterpret_cast<const float*>(bsh), bc + (int64_t)slice * nc * nc, nc,
                                        warp, lane, gyw, cb, tx0, tx1, ty0, ty1, cf.rho, 0.5f * cf.rho);
  }

  // store the tile (inside the grid)
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gy = gyw + r;
    if (gy < ty0 || gy >= ty1) continue;
    const int64_t rbase = off + (int64_t)gy * n + cb;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int gx = cb + e;
      const float v = e < 3 ? x[r][e].x : x[r][e - 3].y;
      if (gx >= tx0 && gx < tx1) x_out[rbase + e] = G(v);
    }
  }
}

template <typename G, int NL, int NSW, int R, int NWARP, int MINB, bool ASYNCB, bool PDIR, bool DIAG, bool PROL,
          bool RESTR, bool SCALE>
__global__ void __launch_bounds__(32 * NWARP, MINB) k_gs_wide(G* __restrict__ x_out, const G* __restrict__ x_in,
                                                            const G* __restrict__ b, const G* __restrict__ xc,
                                                            G* __restrict__ bc, const float* __restrict__ braw,
                                                            G* __restrict__ bsc, int n,
                                                            const Coef<float>* __restrict__ coef, int coef_class,
                                                            int J, int K, int level, int reverse, int zero_init) {
  static_assert(!(PROL && RESTR), "the prolongation starts post-smoothing, the restriction ends pre-smoothing");
  static_assert(!SCALE || RESTR, "the scaling is fused into the one pre-smoothing launch, which also restricts");
#define ST_WIDE_BODY(PA, PY)                                                                                    \
  wide_body<G, NL, NSW, R, NWARP, ASYNCB, PDIR, DIAG, PROL, RESTR, SCALE, PA, PY>(x_out, x_in, b, xc, bc, braw, bsc, \
                                                                                  n,                               \
                                                                              coef, coef_class,                   \
                                                                       J, K, level, reverse, zero_init)
  if (!PROL && !RESTR) {
    ST_WIDE_BODY(0, 0);
    return;
  }
  // the region origin as in wide_body: block-uniform parities, one code path per class
  constexpr int M = 3 * NSW + (RESTR ? 2 : 0);
  int t, e, x0, y0;
  wide_tile(blockIdx.x, gridDim.x, n, 6 * NL, M, t, e, x0);
  wide_tile(blockIdx.y, gridDim.y, n, (32 * NWARP / NL) * R, M, t, e, y0);
  const int pa = (x0 + 1) & 1, py = (y0 + 1) & 1;
  if (pa == 0 && py == 0)
    ST_WIDE_BODY(0, 0);
  else if (pa == 0)
    ST_WIDE_BODY(0, 1);
  else if (py == 0)
    ST_WIDE_BODY(1, 0);
  else
    ST_WIDE_BODY(1, 1);
#undef ST_WIDE_BODY
}

// Block shapes (lanes per row group, rows per group, warps, minimum resident blocks per SM): 0 the
// 192 x 96 regions of whole warps (levels with n >= 192), 1 the 96 x 96 regions of half-warps
// (96 <= n < 192; 6 rows a group, a multiple of 3, so both halves of a warp take the same
// colour-step branch)
template <int SHAPE>
struct WideShape;
template <>
struct WideShape<0> {
  static constexpr int NL = 32, R = 12, NWARP = 8, MINB = 2;
  static constexpr bool ASYNCB = ST_WIDE_ASYNC_B0;  // b' through registers
  static constexpr bool PDIRECT = kProlDirect;      // coarse values straight into registers
};
template <>
struct WideShape<1> {
  static constexpr int NL = 16, R = 6, NWARP = 8, MINB = 3;
  static constexpr bool ASYNCB = ST_WIDE_ASYNC_B0;
  static constexpr bool PDIRECT = kProlDirect;
};
// the shape for level k (n = 2^k - 1 >= 96; wide_fits)
inline int wide_shape_for(int k) { return ((1 << k) - 1) >= 192 ? 0 : 1; }

template <typename G, int NSW, int SHAPE, bool DIAG, bool PROL, bool RESTR, bool SCALE = false>
cudaError_t wide_launch_shape(const st_handle_s* h, int k, int nslices, int cls, G* x_out, const G* x_in,
                              const G* b, const G* xc, G* bc, bool reverse, bool zero_init,
                              const float* braw = nullptr, G* bsc = nullptr) {
  using S = WideShape<SHAPE>;
  constexpr int M = 3 * NSW + (RESTR ? 2 : 0), RH = (32 * S::NWARP / S::NL) * S::R;
  const int n = (1 << k) - 1;
  dim3 grid(wide_ntiles(n, 6 * S::NL, M), wide_ntiles(n, RH, M), nslices);
  constexpr size_t smem = wide_smem<S::NL, S::R, S::NWARP>();
  const bool prof = (k == h->K) && prof_start(h);
  k_gs_wide<G, S::NL, NSW, S::R, S::NWARP, S::MINB, S::ASYNCB, S::PDIRECT, DIAG, PROL, RESTR, SCALE>
      <<<grid, 32 * S::NWARP, smem, h->stream>>>(x_out, x_in, b, xc, bc, braw, bsc, n, coef_table<float>(h), cls, h->J,
                                                 h->K, k, reverse ? 1 : 0, zero_init ? 1 : 0);
  count_launch(h);
  if (prof) {
    // bytes: read x (not from x = 0) and b' (with SCALE: b, and write b'), write x; the coarse
    // iterate read by the prolongation, or the coarse right-hand side written by the restriction
    const double pts = (double)n * n * nslices;
    const double nc = (double)((n - 1) / 2);
    prof_stop(h, (DIAG ? 1 : 0) + 2, pts * NSW * (DIAG ? 6.0 : 4.0),
              sizeof(G) * (pts * ((zero_init ? 2.0 : 3.0) + (SCALE ? 1.0 : 0.0)) +
                           ((PROL || RESTR) ? nc * nc * nslices : 0.0)));
  }
  return cudaGetLastError();
}

// dynamic shared-memory limits of the kernels of one storage type, sweep count and block shape
template <typename G, int NSW, int SHAPE>
cudaError_t wide_attr_shape() {
  using S = WideShape<SHAPE>;
  const int smem = (int)wide_smem<S::NL, S::R, S::NWARP>();
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
#define ST_WIDE_ATTR(DIAG, PROL, RESTR, SCALE)                                                                 \
  if (e == cudaSuccess)                                                                                        \
    e = cudaFuncSetAttribute(                                                                                  \
        k_gs_wide<G, S::NL, NSW, S::R, S::NWARP, S::MINB, S::ASYNCB, S::PDIRECT, DIAG, PROL, RESTR, SCALE>, attr, \
        smem);
  ST_WIDE_ATTR(false, false, false, false)
  ST_WIDE_ATTR(false, true, false, false)
  ST_WIDE_ATTR(false, false, true, false)
  ST_WIDE_ATTR(true, false, false, false)
  ST_WIDE_ATTR(true, true, false, false)
  ST_WIDE_ATTR(true, false, true, false)
  if constexpr (std::is_same<G, float>::value && NSW == 3) {
    ST_WIDE_ATTR(false, false, true, true)
    ST_WIDE_ATTR(true, false, true, true)
  }
#undef ST_WIDE_ATTR
  return e;
}

template <typename G, int NSW>
cudaError_t wide_attr() {
  cudaError_t e = wide_attr_shape<G, NSW, 0>();
  if (e == cudaSuccess) e = wide_attr_shape<G, NSW, 1>();
  return e;
}

}  // namespace

template <typename G, int NSW, bool DIAG, bool PROL>
cudaError_t wide_launch(const st_handle_s* h, int /*shape*/, int k, int nslices, int cls, G* x_out, const G* x_in,
                        const G* b, const G* xc, bool reverse, bool zero_init) {
  if (wide_shape_for(k) == 1)
    return wide_launch_shape<G, NSW, 1, DIAG, PROL, false>(h, k, nslices, cls, x_out, x_in, b, xc, nullptr, reverse,
                                                           zero_init);
  return wide_launch_shape<G, NSW, 0, DIAG, PROL, false>(h, k, nslices, cls, x_out, x_in, b, xc, nullptr, reverse,
                                                         zero_init);
}

template <typename G, int NSW, bool DIAG>
cudaError_t wide_launch_restrict(const st_handle_s* h, int /*shape*/, int k, int nslices, int cls, G* x_out,
                                 const G* x_in, const G* b, G* bc, bool zero_init) {
  if (wide_shape_for(k) == 1)
    return wide_launch_shape<G, NSW, 1, DIAG, false, true>(h, k, nslices, cls, x_out, x_in, b, nullptr, bc, false,
                                                           zero_init);
  return wide_launch_shape<G, NSW, 0, DIAG, false, true>(h, k, nslices, cls, x_out, x_in, b, nullptr, bc, false,
                                                         zero_init);
}

// the finest level's only pre-smoothing launch of the first V-cycle (x = 0): b' = b / c formed from
// the input b and written to bsc, three sweeps, and the residual restricted to bc (binary32
// storage, three fused sweeps)
template <bool DIAG>
cudaError_t wide_launch_scale_restrict(const st_handle_s* h, int k, int nslices, int cls, float* x_out,
                                       const float* braw, float* bsc, float* bc) {
  if (wide_shape_for(k) == 1)
    return wide_launch_shape<float, 3, 1, DIAG, false, true, true>(h, k, nslices, cls, x_out, nullptr, bsc, nullptr,
                                                                   bc, false, true, braw, bsc);
  return wide_launch_shape<float, 3, 0, DIAG, false, true, true>(h, k, nslices, cls, x_out, nullptr, bsc, nullptr, bc,
                                                                 false, true, braw, bsc);
}

// the launchers of one storage type G and sweep count NSW, and that pair's attribute setter
#define ST_WIDE_INSTANTIATE(G, NSW, SETTER)                                                                   \
  template cudaError_t wide_launch<G, NSW, false, false>(const st_handle_s*, int, int, int, int, G*, const G*, \
                                                         const G*, const G*, bool, bool);                      \
  template cudaError_t wide_launch<G, NSW, false, true>(const st_handle_s*, int, int, int, int, G*, const G*,  \
                                                        const G*, const G*, bool, bool);                       \
  template cudaError_t wide_launch<G, NSW, true, false>(const st_handle_s*, int, int, int, int, G*, const G*,  \
                                                        const G*, const G*, bool, bool);                       \
  template cudaError_t wide_launch<G, NSW, true, true>(const st_handle_s*, int, int, int, int, G*, const G*,   \
                                                       const G*, const G*, bool, bool);                        \
  template cudaError_t wide_launch_restrict<G, NSW, false>(const st_handle_s*, int, int, int, int, G*,         \
                                                           const G*, const G*, G*, bool);                      \
  template cudaError_t wide_launch_restrict<G, NSW, true>(const st_handle_s*, int, int, int, int, G*,          \
                                                          const G*, const G*, G*, bool);                       \
  cudaError_t SETTER() { return wide_attr<G, NSW>(); }

// attribute setters of the four translation units
cudaError_t wide_attr_f32_nsw1();
cudaError_t wide_attr_f32_nsw3();
cudaError_t wide_attr_bf16_nsw1();
cudaError_t wide_attr_bf16_nsw3();

}  // namespace st
