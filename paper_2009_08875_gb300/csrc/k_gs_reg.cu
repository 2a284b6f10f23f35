// Gauss-Seidel sweeps of the time-slice-batched multigrid (k_mg.cu) in register tiles: the same
// three-colour sweeps as k_gs_sweep, with the region held in registers instead of shared memory.
#include <cuda_bf16.h>

#include <type_traits>

#include "df64.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

// ---------------------------------------------------------------------------------------
// Gauss-Seidel in register tiles.  A block of NWARP warps holds a region of 96 columns x
// NWARP * R rows of one slice in registers: warp w owns the region rows w R .. w R + R - 1 and
// lane l the columns 3 l .. 3 l + 2 of them, so that in every row exactly one of a lane's three
// points has the active colour (the colour steps below never branch per lane).  A colour step
// takes its horizontal neighbours from the lane's own registers or, across a lane boundary, by a
// shuffle; its vertical neighbours from the rows above and below in registers or, at the edge of
// a warp's rows, from the neighbouring warp's edge row, exchanged through shared memory once per
// step.  A colour step reads only points of the other two colours, which the step does not
// change, so the edge rows copied at its start are current.  As in k_gs_sweep the region
// carries a halo of H = 3 NSW points: points next to the region's edge are updated with missing
// neighbours taken as 0 (columns) or skipped (rows outside the shrinking window), and the error
// this makes travels one point per colour step, so after the 3 NSW steps the interior (the tile)
// is exactly what sequential colour-by-colour sweeps give, with the same update expression as
// k_gs_sweep: bitwise the same results.  With PROL the coarse values under the region are staged
// in shared memory once and the prolongated correction x + P xc is formed from there.
// ---------------------------------------------------------------------------------------

// floor(v / 2) for any sign
__device__ __forceinline__ int floor_half(int v) { return v >= 0 ? (v >> 1) : -((-v + 1) >> 1); }

// One colour step on a warp's R rows.  P is the lane element of the active colour in the warp's
// first row (element m(r) = (P - r) mod 3 in row r).  below / above: the edge rows of the warps
// underneath and on top (96 values each, zeros past the region).  Only the rows whose bit is set
// in `rows` are updated (the shrinking window, inside the grid), and in them the points whose
// column is in the grid (ok_lo[m]) or, on the L-shape in rows at y >= 1/2 (bit set in `qrows`),
// also left of x = 1/2 (ok_hi[m]).
template <typename T, int R, bool DIAG, bool LSH, int P>
__device__ __forceinline__ void reg_step(T (&x)[R][3], const T (&bb)[R][3], const T* __restrict__ below,
                                         const T* __restrict__ above, int lane, unsigned rows, unsigned qrows, T axs,
                                         T ays, T dgs, const bool (&ok_lo)[3], const bool (&ok_hi)[3]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    constexpr int kR1 = R - 1;
    const int m = ((P - (r % 3)) + 3) % 3;  // a constant once the loop is unrolled
    const int rs = r > 0 ? r - 1 : 0;      // row below inside the warp (valid when r > 0)
    const int rn = r < kR1 ? r + 1 : kR1;  // row above inside the warp (valid when r < R - 1)
    if (!(rows & (1u << r))) continue;     // warp-uniform
    const int cidx = 3 * lane + m;         // region column of the active point
    // the shuffles run on every lane (the branches are uniform: m is a constant)
    const T west = (m == 0) ? shfl_up(x[r][2], 1) : x[r][(m + 2) % 3];
    const T east = (m == 2) ? shfl_down(x[r][0], 1) : x[r][(m + 1) % 3];
    const T south = (r > 0) ? x[rs][m] : below[cidx];
    const T north = (r < kR1) ? x[rn][m] : above[cidx];
    T v = bb[r][m] - axs * (west + east);
    v -= ays * (south + north);
    if (DIAG) {
      // (1,1) and (-1,-1) neighbours
      const T ne = (r < kR1) ? ((m == 2) ? shfl_down(x[rn][0], 1) : x[rn][(m + 1) % 3])
                             : above[cidx < 95 ? cidx + 1 : 95];
      const T sw = (r > 0) ? ((m == 0) ? shfl_up(x[rs][2], 1) : x[rs][(m + 2) % 3]) : below[cidx > 0 ? cidx - 1 : 0];
      v -= dgs * (ne + sw);
    }
    const bool ok = LSH ? ((qrows & (1u << r)) ? ok_hi[m] : ok_lo[m]) : ok_lo[m];
    if (ok) x[r][m] = v;
  }
}

// The first colour step of a sweep from x = 0: every neighbour is zero, so x = b'.
template <typename T, int R, bool LSH, int P>
__device__ __forceinline__ void reg_step_first(T (&x)[R][3], const T (&bb)[R][3], unsigned rows, unsigned qrows,
                                               const bool (&ok_lo)[3], const bool (&ok_hi)[3]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int m = ((P - (r % 3)) + 3) % 3;
    if (!(rows & (1u << r))) continue;
    const bool ok = LSH ? ((qrows & (1u << r)) ? ok_hi[m] : ok_lo[m]) : ok_lo[m];
    if (ok) x[r][m] = bb[r][m];
  }
}

// bits lo .. hi - 1 of a 32-bit mask (empty when hi <= lo)
__device__ __forceinline__ unsigned bit_range(int lo, int hi) {
  lo = lo < 0 ? 0 : lo;
  hi = hi > 31 ? 31 : hi;
  return hi <= lo ? 0u : (((1u << hi) - 1u) & ~((1u << lo) - 1u));
}


template <typename T, typename G, int NSW, int R, int NWARP, bool DIAG, bool PROL, bool LSH>
__global__ void __launch_bounds__(32 * NWARP, 2) k_gs_reg(G* __restrict__ x_out, const G* __restrict__ x_in,
                                                       const G* __restrict__ b, const G* __restrict__ xc, int n,
                                                       const Coef<T>* __restrict__ coef, int coef_class, int J,
                                                       int K, int level, int reverse, int zero_init) {
  constexpr int H = 3 * NSW;
  constexpr int RH = NWARP * R;  // region rows
  constexpr int TX = kWR - 2 * H, TY = RH - 2 * H;
  constexpr int CW = kWR / 2 + 2, CH = RH / 2 + 2;  // coarse values under the region (PROL)
  static_assert(R < 32, "row masks hold 31 rows");
  __shared__ T edge[2][NWARP][2][kWR];               // [step parity][warp][bottom row, top row]
  __shared__ T zrow[kWR];                            // zeros past the region's first and last rows
  __shared__ T ct[PROL ? CH * CW : 1];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slice = blockIdx.z;
  const int64_t off = (int64_t)slice * n * n;
  const int gx0 = blockIdx.x * TX - H, gy0 = blockIdx.y * TY - H;
  const int ry0 = warp * R;       // first region row of the warp
  const int gyw = gy0 + ry0;      // its grid row
  const int cb = gx0 + 3 * lane;  // grid column of the lane's element 0
  const int q = (n - 1) >> 1;     // L-shape: index of x = 1/2
  const Coef<T> cf = slice_coef(coef, coef_class, slice, J, K, level);
  // ok_lo: column in the grid; ok_hi: also left of x = 1/2 (L-shape rows at y >= 1/2)
  bool ok_lo[3], ok_hi[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    ok_lo[e] = cb + e >= 0 && cb + e < n;
    ok_hi[e] = ok_lo[e] && !(LSH && cb + e >= q);
  }
  // the warp's rows in the grid, and (L-shape) those at y >= 1/2
  const unsigned grid_rows = bit_range(-gyw, n - gyw);
  const unsigned qrows = LSH ? bit_range(q - gyw, R) : 0u;
  for (int i = threadIdx.x; i < kWR; i += blockDim.x) zrow[i] = T(0);

  const int nc = (n - 1) / 2;
  const int Ib = floor_half(gx0 + 1), Jb = floor_half(gy0 + 1);  // coarse indices at ct[0]
  if (PROL) {
    const G* xcs = xc + (int64_t)slice * nc * nc;
    for (int idx = threadIdx.x; idx < CH * CW; idx += blockDim.x) {
      const int jj = idx / CW, ii = idx - jj * CW;
      const int I = Ib + ii, Jc = Jb + jj;
      ct[idx] = (I >= 1 && I <= nc && Jc >= 1 && Jc <= nc) ? T(xcs[(int64_t)(Jc - 1) * nc + (I - 1)]) : T(0);
    }
    __syncthreads();
  }

  // load the warp's rows: b, and x (0 from x = 0; + P xc with PROL, whose points of the first
  // colour step's colour are overwritten unread, so they are not formed)
  T x[R][3], bb[R][3];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gy = gyw + r;
    const bool hi = LSH && (qrows & (1u << r));
    const bool rowok = (grid_rows >> r) & 1u;
    const int64_t rbase = off + (int64_t)gy * n + cb;
    int eskip = ((reverse ? 2 : 0) - 2 - gy - gx0) % 3;
    eskip += (eskip < 0) ? 3 : 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const bool in = rowok && (hi ? ok_hi[e] : ok_lo[e]);
      bb[r][e] = in ? T(b[rbase + e]) : T(0);
      T v = T(0);
      if (!PROL) {
        if (in && !zero_init) v = T(x_in[rbase + e]);
      } else if (e != eskip) {
        if (in && !zero_init) v = T(x_in[rbase + e]);
        if (in) {
          const int i = cb + e + 1, j = gy + 1;  // 1-based grid indices
          const int I0 = i >> 1, J0 = j >> 1;
          const int I1 = I0 + (i & 1), J1 = J0 + (j & 1);
          v += T(0.5) * (ct[(J0 - Jb) * CW + (I0 - Ib)] + ct[(J1 - Jb) * CW + (I1 - Ib)]);
        }
      }
      x[r][e] = v;
    }
  }

#pragma unroll 1
  for (int t = 0; t < 3 * NSW; ++t) {
    const int colour = reverse ? 2 - t % 3 : t % 3;
    // publish this warp's first and last rows for the neighbouring warps (double-buffered by step
    // parity: a warp writing step t + 1's rows has passed step t's barrier, so every warp has
    // finished reading step t - 1's)
    T* ed = &edge[t & 1][warp][0][0];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      ed[3 * lane + e] = x[0][e];
      ed[kWR + 3 * lane + e] = x[R - 1][e];
    }
    __syncthreads();
    const T* below = warp > 0 ? &edge[t & 1][warp - 1][1][0] : zrow;
    const T* above = warp < NWARP - 1 ? &edge[t & 1][warp + 1][0][0] : zrow;
    // rows of the shrinking window (region rows t + 1 .. RH - t - 2) that lie in the grid
    const unsigned rows = grid_rows & bit_range(t + 1 - ry0, RH - t - 1 - ry0);
    int P = (colour - 2 - gyw - gx0) % 3;  // active element in the warp's first row
    P += (P < 0) ? 3 : 0;
    if (!PROL && zero_init && t == 0) {
      if (P == 0)
        reg_step_first<T, R, LSH, 0>(x, bb, rows, qrows, ok_lo, ok_hi);
      else if (P == 1)
        reg_step_first<T, R, LSH, 1>(x, bb, rows, qrows, ok_lo, ok_hi);
      else
        reg_step_first<T, R, LSH, 2>(x, bb, rows, qrows, ok_lo, ok_hi);
    } else if (P == 0) {
      reg_step<T, R, DIAG, LSH, 0>(x, bb, below, above, lane, rows, qrows, cf.axs, cf.ays, cf.dgs, ok_lo, ok_hi);
    } else if (P == 1) {
      reg_step<T, R, DIAG, LSH, 1>(x, bb, below, above, lane, rows, qrows, cf.axs, cf.ays, cf.dgs, ok_lo, ok_hi);
    } else {
      reg_step<T, R, DIAG, LSH, 2>(x, bb, below, above, lane, rows, qrows, cf.axs, cf.ays, cf.dgs, ok_lo, ok_hi);
    }
  }

  // store the tile: region rows H .. RH - H - 1, columns H .. 95 - H
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int ry = ry0 + r, gy = gyw + r;
    if (ry < H || ry >= RH - H || gy >= n) continue;
    const int64_t rbase = off + (int64_t)gy * n + cb;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int rx = 3 * lane + e;
      if (rx >= H && rx < kWR - H && cb + e < n) x_out[rbase + e] = G(x[r][e]);
    }
  }
}

}  // namespace

// Block shapes (rows per warp, warps): binary32 picks among three (autotuned), binary64 and
// double-float keep one.
template <typename T, int SHAPE>
struct RegShape;
template <int S>
struct RegShape<double, S> {
  static constexpr int R = 6, NWARP = 8;
};
template <int S>
struct RegShape<df64, S> {  // 8-byte values like binary64
  static constexpr int R = 6, NWARP = 8;
};
template <>
struct RegShape<float, 0> {
  static constexpr int R = 12, NWARP = 8;
};
template <>
struct RegShape<float, 1> {
  static constexpr int R = 8, NWARP = 12;
};
template <>
struct RegShape<float, 2> {
  static constexpr int R = 6, NWARP = 16;
};

template <typename T, typename G, int NSW, int SHAPE, bool DIAG, bool PROL>
cudaError_t reg_launch_shape(const st_handle_s* h, int k, int nslices, int cls, G* x_out, const G* x_in, const G* b,
                             const G* xc, bool reverse, bool zero_init) {
  constexpr int R = RegShape<T, SHAPE>::R, NW = RegShape<T, SHAPE>::NWARP;
  constexpr int H = 3 * NSW;
  const int n = (1 << k) - 1;
  const int TX = kWR - 2 * H, TY = NW * R - 2 * H;
  dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, nslices);
  const bool prof = (k == h->K) && prof_start(h);
  if (h->domain == 1)
    k_gs_reg<T, G, NSW, R, NW, DIAG, PROL, true><<<grid, 32 * NW, 0, h->stream>>>(
        x_out, x_in, b, xc, n, coef_table<T>(h), cls, h->J, h->K, k, reverse ? 1 : 0, zero_init ? 1 : 0);
  else
    k_gs_reg<T, G, NSW, R, NW, DIAG, PROL, false><<<grid, 32 * NW, 0, h->stream>>>(
        x_out, x_in, b, xc, n, coef_table<T>(h), cls, h->J, h->K, k, reverse ? 1 : 0, zero_init ? 1 : 0);
  count_launch(h);
  if (prof) {
    const double pts = (double)n * n * nslices;
    const double nc = (double)((n - 1) / 2);
    prof_stop(h, (DIAG ? 1 : 0) + (sizeof(T) == 4 ? 2 : 0), pts * NSW * (DIAG ? 6.0 : 4.0),
              sizeof(G) * (pts * (zero_init ? 2.0 : 3.0) + (PROL ? nc * nc * nslices : 0.0)));
  }
  return cudaGetLastError();
}

template <typename T, typename G, int NSW, bool DIAG, bool PROL>
cudaError_t reg_launch(const st_handle_s* h, int shape, int k, int nslices, int cls, G* x_out, const G* x_in,
                       const G* b, const G* xc, bool reverse, bool zero_init) {
  // shape 3: binary32 wide regions with paired arithmetic (k_gs_wide.cuh) on the levels whose
  // grid holds a region; shape 0 elsewhere
  if constexpr (std::is_same<T, float>::value) {
    if (shape == 3) {
      if (wide_fits(h, 0, k))
        return wide_launch<G, NSW, DIAG, PROL>(h, 0, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
      shape = 0;
    }
  }
  if (sizeof(T) == 4 && shape == 1)
    return reg_launch_shape<T, G, NSW, 1, DIAG, PROL>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
  if (sizeof(T) == 4 && shape == 2)
    return reg_launch_shape<T, G, NSW, 2, DIAG, PROL>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
  return reg_launch_shape<T, G, NSW, 0, DIAG, PROL>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
}

#define ST_REG(T, G, NSW)                                                                                     \
  template cudaError_t reg_launch<T, G, NSW, false, false>(const st_handle_s*, int, int, int, int, G*, const G*, \
                                                           const G*, const G*, bool, bool);                    \
  template cudaError_t reg_launch<T, G, NSW, false, true>(const st_handle_s*, int, int, int, int, G*, const G*,  \
                                                          const G*, const G*, bool, bool);                     \
  template cudaError_t reg_launch<T, G, NSW, true, false>(const st_handle_s*, int, int, int, int, G*, const G*,  \
                                                          const G*, const G*, bool, bool);                     \
  template cudaError_t reg_launch<T, G, NSW, true, true>(const st_handle_s*, int, int, int, int, G*, const G*,   \
                                                         const G*, const G*, bool, bool);
ST_REG(double, double, 1)
ST_REG(df64, df64, 1)
ST_REG(float, float, 1)
ST_REG(float, float, 3)
ST_REG(float, __nv_bfloat16, 1)
ST_REG(float, __nv_bfloat16, 3)
#undef ST_REG

}  // namespace st
