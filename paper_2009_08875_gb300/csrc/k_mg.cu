// Time-slice-batched symmetric multigrid for C = a A_x + s M_x (K_x, K_l of Sec. 3.1 and
// Thm. 3.1; "2 V-cycles with 3 Gauss-Seidel steps per grid", Sec. 5.1).
//
// One launch processes every slice of a batch.  Level k has n = 2^k - 1 interior points
// per side, slices are contiguous n*n blocks.  Readings (the paper leaves them open):
// nested P1 prolongation, restriction = its transpose, rediscretised coarse operators,
// Gauss-Seidel in three colours c = (i + j) mod 3 of the grid indices (i, j) = (ix+1, iy+1),
// pre-sweeps in colour order 0,1,2 and post-sweeps 2,1,0 (a symmetric V-cycle), exact
// solve on level 1 (one unknown), every application starting from x = 0.
#include <cuda_bf16.h>

#include <type_traits>

#include "df64.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

// ---------------------------------------------------------------------------------------
// coefficient table: class 0 -> (a, s) = (1, 0); class 1 + l -> (alpha, 2^l), l = 0..J, of
// C = a A_x + s M_x with A_x = <D grad, grad> + c M_x (Sec. 4)
// ---------------------------------------------------------------------------------------
// In 3D (the unit cube, Kuhn tetrahedra, heat equation plus c): A_x = h [6; -1 at the axis
// neighbours] and M_x = h^3 [2/5; 1/20 at the axis and body-diagonal, 1/30 at the face-diagonal
// neighbours]; ax, ay, dg then hold the axis, face-diagonal and body-diagonal coefficients.
template <typename T>
__global__ void k_make_coef(Coef<T>* coef, int K, int J, double alpha, Phys ph, int dim) {
  int nclass = J + 2;
  for (int e = threadIdx.x; e < nclass * (K + 1); e += blockDim.x) {
    int cls = e / (K + 1), k = e % (K + 1);
    double a = cls == 0 ? 1.0 : alpha;
    double s = cls == 0 ? 0.0 : ldexp(1.0, cls - 1);
    if (dim == 3) {
      const double h = ldexp(1.0, -k), hc = ldexp(1.0, -(k - 1));
      const double ms = (a * ph.c + s) * h * h * h, msc = (a * ph.c + s) * hc * hc * hc;
      const double cc = 6.0 * a * h + 0.4 * ms, cc_coarse = 6.0 * a * hc + 0.4 * msc;
      const double ax = -a * h + ms / 20.0, face = ms / 30.0, body = ms / 20.0;
      Coef<T> c;
      c.c = (T)cc;
      c.ax = (T)ax;
      c.ay = (T)face;
      c.dg = (T)body;
      c.inv_c = (T)(1.0 / cc);
      c.axs = (T)(ax / cc);
      c.ays = (T)(face / cc);
      c.dgs = (T)(body / cc);
      c.rho = (T)(cc / cc_coarse);
      c.pad = T(0);
      coef[e] = c;
      continue;
    }
    const double m = (a * ph.c + s) * ldexp(1.0, -2 * k) / 12.0;            // level k
    const double mc = (a * ph.c + s) * ldexp(1.0, -2 * (k - 1)) / 12.0;      // level k - 1
    const double stiff_c = a * 2.0 * (ph.d11 + ph.d22 - ph.d12);
    const double cc = stiff_c + 6.0 * m;
    const double ax = a * (ph.d12 - ph.d11) + m, ay = a * (ph.d12 - ph.d22) + m, dg = -a * ph.d12 + m;
    const double cc_coarse = stiff_c + 6.0 * mc;
    Coef<T> c;
    c.c = (T)cc;
    c.ax = (T)ax;
    c.ay = (T)ay;
    c.dg = (T)dg;
    c.inv_c = (T)(1.0 / cc);
    c.axs = (T)(ax / cc);
    c.ays = (T)(ay / cc);
    c.dgs = (T)(dg / cc);
    c.rho = (T)(cc / cc_coarse);
    c.pad = T(0);
    coef[e] = c;
  }
}


// Nested P1 prolongation: prolong_value (st_internal.cuh).

// ---------------------------------------------------------------------------------------
// Gauss-Seidel: NSW full 3-colour sweeps of one slice tile, staged in shared memory.
// The block owns an interior tile of TX x TY points and loads a halo of H = 3 NSW points:
// colour step t (0-based) updates every point within H - 1 - t of the tile, so after the
// last step the interior is exactly what sequential colour-by-colour sweeps over the whole
// slice produce.  Each lane owns three consecutive columns, of which exactly one has the
// active colour in any row, so every lane does one update per row and step.
// ---------------------------------------------------------------------------------------

// Exact solve on level 2 (3 x 3 grid, the coarsest level of the L-shape): one thread per slice
// assembles C = a A + s M on the level's nodes (rows of nodes outside the domain become the
// identity with zero right-hand side) and solves C x = D b' by Gaussian elimination (C is SPD on
// the domain nodes, so no pivoting is needed).
template <typename T, typename G>
__global__ void k_coarse_dense3(G* __restrict__ x, const G* __restrict__ b, int nslices,
                                const Coef<T>* __restrict__ coef, int coef_class, int J, int K, int lshape) {
  const int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslices) return;
  const Coef<T> cf = slice_coef(coef, coef_class, sl, J, K, 2);
  using C = typename std::conditional<std::is_same<T, df64>::value, double, T>::type;  // elimination type
  C A[9][10];
  for (int p = 0; p < 9; ++p) {
    for (int q = 0; q < 10; ++q) A[p][q] = C(0);
    const int ix = p % 3, iy = p / 3;
    if (outside_domain(ix, iy, 3, lshape)) {
      A[p][p] = C(1);
      continue;
    }
    A[p][p] = C(cf.c);
    A[p][9] = C(cf.c) * C(b[(int64_t)sl * 9 + p]);
    const int nb[6][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}, {1, 1}, {-1, -1}};
    for (int t = 0; t < 6; ++t) {
      const int jx = ix + nb[t][0], jy = iy + nb[t][1];
      if (jx < 0 || jx > 2 || jy < 0 || jy > 2 || outside_domain(jx, jy, 3, lshape)) continue;
      A[p][jy * 3 + jx] = C(t < 2 ? cf.ax : (t < 4 ? cf.ay : cf.dg));
    }
  }
  for (int c = 0; c < 9; ++c) {
    for (int r = c + 1; r < 9; ++r) {
      const C f = A[r][c] / A[c][c];
      for (int q = c; q < 10; ++q) A[r][q] -= f * A[c][q];
    }
  }
  for (int r = 8; r >= 0; --r) {
    C v = A[r][9];
    for (int q = r + 1; q < 9; ++q) v -= A[r][q] * A[q][9];
    A[r][9] = v / A[r][r];
  }
  for (int p = 0; p < 9; ++p) x[(int64_t)sl * 9 + p] = G(A[p][9]);
}

// The sweep is out of place (x_in -> x_out): a block's halo overlaps its neighbours' interiors,
// so reading and writing one buffer in the same launch would race.
// With PROL the launch first adds the prolongated coarse correction P xc to the iterate it loads
// (the coarse-grid correction of the V-cycle, fused into the first post-smoothing launch).
template <typename T, typename G, int NSW, int HR, bool DIAG, bool PROL>
__global__ void __launch_bounds__(256) k_gs_sweep(G* __restrict__ x_out, const G* __restrict__ x_in,
                                                  const G* __restrict__ b, const G* __restrict__ xc, int n,
                                                  const Coef<T>* __restrict__ coef, int coef_class, int J,
                                                  int K, int level, int reverse, int zero_init, int lshape) {
  constexpr int H = 3 * NSW;
  constexpr int TX = kWR - 2 * H;
  constexpr int TY = HR - 2 * H;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  T* bs = xs + HR * kWR;

  const int slice = blockIdx.z;
  const int64_t off = (int64_t)slice * n * n;
  G* xsl = x_out + off;
  const G* xin = x_in + off;
  const G* bsl = b + off;
  const int nc = (n - 1) / 2;
  const G* xcs = PROL ? xc + (int64_t)slice * nc * nc : nullptr;
  const int gx0 = blockIdx.x * TX - H;
  const int gy0 = blockIdx.y * TY - H;
  const Coef<T> cf = slice_coef(coef, coef_class, slice, J, K, level);

  // stage the region: warp w takes rows w, w + 8, ..., lane l the columns l, l + 32, l + 64
  constexpr int kWarps = 8;  // launched with 256 threads
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int ry = warp; ry < HR; ry += kWarps) {
    const int gy = gy0 + ry;
    const bool row_in = gy >= 0 && gy < n;
    const int64_t grow = (int64_t)gy * n;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int rx = lane + 32 * e, idx = ry * kWR + rx;
      const int gx = gx0 + rx;
      const bool in = row_in && gx >= 0 && gx < n && !outside_domain(gx, gy, n, lshape);
      const int64_t gi = grow + gx;
      if (!PROL) xs[idx] = (in && !zero_init) ? T(xin[gi]) : T(0);
      bs[idx] = in ? T(bsl[gi]) : T(0);
    }
    if (PROL) {
      // x + P xc, lane l taking the columns 3 l .. 3 l + 2, where the colour of element e is the
      // same in every lane.  The points of the first colour step's colour c0 are overwritten by
      // that step, which reads only other colours, and no earlier read touches them, so their
      // old values and corrections are not formed (a warp-uniform branch; they hold 0).
      // colour (gx + gy + 2) mod 3 == c0  <=>  e == c0 - 2 - gy - gx0 (mod 3)
      int eskip = ((reverse ? 2 : 0) - 2 - gy - gx0) % 3;
      eskip += (eskip < 0) ? 3 : 0;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int rx = 3 * lane + e, idx = ry * kWR + rx;
        const int gx = gx0 + rx;
        T v = T(0);
        if (e != eskip) {
          const bool in = row_in && gx >= 0 && gx < n && !outside_domain(gx, gy, n, lshape);
          if (in && !zero_init) v = T(xin[grow + gx]);
          if (in) v += prolong_value<T>(xcs, nc, gx + 1, gy + 1);
        }
        xs[idx] = v;
      }
    }
  }
  __syncthreads();

#pragma unroll 1
  for (int t = 0; t < 3 * NSW; ++t) {
    const int tc = t % 3;
    const int colour = reverse ? 2 - tc : tc;
    const int lo = t + 1;
    const int ry_lo = max(lo, -gy0), ry_hi = min(HR - lo, n - gy0);
    const int rx_lo = max(lo, -gx0), rx_hi = min(kWR - lo, n - gx0);
    // each warp updates R rows per pass: all operands are gathered before any result is
    // stored, so R independent FP64 chains are in flight (points of one colour never couple)
    constexpr int R = 2;
    // colour (gx + gy + 2) mod 3 == colour  <=>  rx == colour - 2 - gy - gx0 (mod 3): the lane's
    // active column in row ry is 3 lane + m(ry), and m(ry + 8) = m(ry) + 1, m(ry + 16) = m(ry) - 1
    // (mod 3), so m is stepped instead of recomputed
    int m0 = (colour - 2 - gy0 - (ry_lo + warp) - gx0) % 3;
    m0 += (m0 < 0) ? 3 : 0;
    // one pass over RR rows ry0, ry0 + 8, ...; every row of it lies below ry_hi
    auto pass = [&](auto rr, int ry0, int m_first) {
      constexpr int RR = decltype(rr)::value;
      T sx[RR], sy[RR], sd[RR], bv[RR];
      int at[RR];
#pragma unroll
      for (int q = 0; q < RR; ++q) {
        const int ry = ry0 + q * kWarps;
        const int gy = gy0 + ry;
        const int mq = q == 0 ? m_first : (m_first == 2 ? 0 : m_first + 1);
        const int rx = 3 * lane + mq;
        const bool ok = rx >= rx_lo && rx < rx_hi && !outside_domain(gx0 + rx, gy, n, lshape);
        const int i = ok ? ry * kWR + rx : kWR + 1;  // a harmless interior address when idle
        at[q] = ok ? i : -1;
        sx[q] = xs[i - 1] + xs[i + 1];
        sy[q] = xs[i - kWR] + xs[i + kWR];
        sd[q] = DIAG ? (xs[i + kWR + 1] + xs[i - kWR - 1]) : T(0);
        bv[q] = bs[i];
      }
#pragma unroll
      for (int q = 0; q < RR; ++q) {
        // scaled system: x = b' - (ax/c) sx - (ay/c) sy - (dg/c) sd with b' = b / c
        T v = bv[q] - cf.axs * sx[q];
        v -= cf.ays * sy[q];
        if (DIAG) v -= cf.dgs * sd[q];
        if (at[q] >= 0) xs[at[q]] = v;
      }
    };
    if (!PROL && zero_init && t == 0) {
      // the first colour of a sweep from x = 0 sees only zero neighbours: x = b'
      for (int ry = ry_lo + warp; ry < ry_hi; ry += kWarps, m0 = (m0 == 2) ? 0 : m0 + 1) {
        const int rx = 3 * lane + m0;
        if (rx >= rx_lo && rx < rx_hi && !outside_domain(gx0 + rx, gy0 + ry, n, lshape))
          xs[ry * kWR + rx] = bs[ry * kWR + rx];
      }
      __syncthreads();
      continue;
    }
    for (int ry0 = ry_lo + warp; ry0 < ry_hi; ry0 += R * kWarps) {
      // the second row is skipped by the whole warp (a uniform branch) when it lies past ry_hi
      if (ry0 + kWarps < ry_hi)
        pass(std::integral_constant<int, 2>(), ry0, m0);
      else
        pass(std::integral_constant<int, 1>(), ry0, m0);
      m0 = (m0 == 0) ? 2 : m0 - 1;
    }
    __syncthreads();
  }

  // write the tile interior
  for (int ty = warp; ty < TY; ty += kWarps) {
    const int gy = gy0 + H + ty;
    if (gy >= n) break;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int tx = lane + 32 * e;
      const int gx = gx0 + H + tx;
      if (tx < TX && gx < n) xsl[(int64_t)gy * n + gx] = G(xs[(ty + H) * kWR + tx + H]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Gauss-Seidel as a register wavefront.  One warp owns a strip of 96 columns (3 per lane) of one
// slice and walks its rows from bottom to top.  The S = 3 * NSW colour steps of NSW sweeps form
// a pipeline along the rows: at time tau, step s (colour c_s) updates row tau - s, for
// s = 0, 1, ..., S - 1 in that order.  Row j then sees row j + 1 after step s - 1 (done earlier
// in the same time step) and row j - 1 after step s, which differs from "after step s - 1" only
// at colour c_s, and same-colour points of adjacent rows are not coupled (the 7-point pattern
// couples (i, j) with (i, j - 1) and (i - 1, j - 1), whose colours differ).  So the result is
// that of sequential colour-by-colour sweeps.  The rows tau - S .. tau + 1 of x (and tau - S + 1
// .. tau of b) live in registers, horizontal neighbours come from the adjacent lane by shuffles,
// and only the strip's horizontal halo (S columns each side) is recomputed; row tau - S + 1 is
// complete at time tau and is stored.  For parallelism a strip is also cut into segments of SEG
// rows, each walked by its own warp over SEG + 2 S rows: errors from the segment's missing
// neighbours travel one row per colour step, so after S steps the middle SEG rows are exact.
// ---------------------------------------------------------------------------------------
template <typename T, typename G, int S, bool DIAG, bool PROL>
__global__ void __launch_bounds__(128) k_gs_wave(G* __restrict__ x_out, const G* __restrict__ x_in,
                                                 const G* __restrict__ b, const G* __restrict__ xc, int n,
                                                 const Coef<T>* __restrict__ coef, int coef_class, int J, int K,
                                                 int level, int reverse, int zero_init, int lshape, int nstrips,
                                                 int nseg, int seg, int nslices) {
  constexpr int W = S + 2;          // ring of x rows: row ybase + r lives in slot r mod W
  constexpr int TXW = kWR - 2 * S;  // output columns of a strip
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (gw >= nstrips * nseg * nslices) return;  // whole warps only
  const int slice = gw / (nstrips * nseg);
  const int rest = gw - slice * nstrips * nseg;
  const int sg = rest / nstrips, strip = rest - sg * nstrips;
  const int r0 = sg * seg;        // first output row of the segment
  const int ybase = r0 - S;       // row of time step 0
  const int gx0 = strip * TXW - S;      // global column of the strip's column 0
  const int64_t off = (int64_t)slice * n * n;
  const G* xin = x_in + off;
  const G* bsl = b + off;
  G* xo = x_out + off;
  const int nc = (n - 1) / 2;
  const G* xcs = PROL ? xc + (int64_t)slice * nc * nc : nullptr;
  const Coef<T> cf = slice_coef(coef, coef_class, slice, J, K, level);
  const int cbase = gx0 + 3 * lane;  // global column of this lane's element 0

  T xw[W][3], bw[W][3];
#pragma unroll
  for (int r = 0; r < W; ++r)
#pragma unroll
    for (int e = 0; e < 3; ++e) xw[r][e] = bw[r][e] = T(0);

  // Row r into registers.  The points of step 0's colour c0 are overwritten by step 0, which
  // reads only other colours, before any read of them that matters (a row past the walked rows
  // is never updated and counts among the missing neighbours above), so their old values and
  // corrections are not loaded: element e has colour c0 in every lane for one e per row.
  auto load_row = [&](int r, T (&xr)[3], T (&br)[3]) {
    int eskip = ((reverse ? 2 : 0) - 2 - r - gx0) % 3;  // colour (gx + r + 2) mod 3 == c0
    eskip += (eskip < 0) ? 3 : 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int gx = cbase + e;
      const bool in = r >= 0 && r < n && gx >= 0 && gx < n && !outside_domain(gx, r, n, lshape);
      const int64_t gi = (int64_t)r * n + gx;
      T v = T(0);
      if (e != eskip) {
        if (in && !zero_init) v = T(xin[gi]);
        if (PROL && in) v += prolong_value<T>(xcs, nc, gx + 1, r + 1);
      }
      xr[e] = v;
      br[e] = in ? T(bsl[gi]) : T(0);
    }
  };

  // one colour step on row j: xc = row j, xn = row j + 1, xs = row j - 1, bc = b of row j
  // m: the lane's element of the step's colour in row j
  auto update_row = [&](T (&xcr)[3], const T (&xn)[3], const T (&xs)[3], const T (&bc)[3], int j, int s, int m) {
    const int cl = 3 * lane + m;
    const int gx = cbase + m;
    const bool ok = cl >= s + 1 && cl < kWR - s - 1 && gx >= 0 && gx < n && !outside_domain(gx, j, n, lshape);
    // neighbours west, east, south, north, north-east, south-west (uniform branch on m)
    const T up_c2 = shfl_up(xcr[2], 1);
    const T dn_c0 = shfl_down(xcr[0], 1);
    T up_s2 = T(0), dn_n0 = T(0);
    if (DIAG) {
      up_s2 = shfl_up(xs[2], 1);
      dn_n0 = shfl_down(xn[0], 1);
    }
    if (!PROL && zero_init && s == 0) {
      // the first colour step of a sweep from x = 0 sees only zero neighbours: x = b'
      // (m is warp-uniform; constant indices keep the rows in registers)
      if (ok) {
        if (m == 0)
          xcr[0] = bc[0];
        else if (m == 1)
          xcr[1] = bc[1];
        else
          xcr[2] = bc[2];
      }
      return;
    }
    if (m == 0) {
      T v = bc[0] - cf.axs * (up_c2 + xcr[1]);
      v -= cf.ays * (xs[0] + xn[0]);
      if (DIAG) v -= cf.dgs * (xn[1] + up_s2);
      if (ok) xcr[0] = v;
    } else if (m == 1) {
      T v = bc[1] - cf.axs * (xcr[0] + xcr[2]);
      v -= cf.ays * (xs[1] + xn[1]);
      if (DIAG) v -= cf.dgs * (xn[2] + xs[0]);
      if (ok) xcr[1] = v;
    } else {
      T v = bc[2] - cf.axs * (xcr[1] + dn_c0);
      v -= cf.ays * (xs[2] + xn[2]);
      if (DIAG) v -= cf.dgs * (dn_n0 + xs[1]);
      if (ok) xcr[2] = v;
    }
  };

  load_row(ybase, xw[0], bw[0]);
  const int L = seg + 2 * S;      // rows walked
  const int tau_end = L + S - 1;  // the last row completes at tau = L + S - 2
  const int r1 = min(r0 + seg, n);
  // Step s at time tau updates row j = ybase + tau - s in colour c_s (s mod 3, or 2 - s mod 3 in
  // reverse); the lane's element of that colour is m = (c_s - 2 - j - gx0) mod 3
  // = (z - tau + c_s + s) mod 3 with z = (-2 - ybase - gx0) mod 3, and c_s + s = 2 s (forward) or
  // 2 (reverse) mod 3.  With tz = (z - tau0) mod 3 kept per block of W steps, m is tz plus a
  // constant of (s, u) reduced once.
  int tz = (-2 - ybase - gx0) % 3;
  tz += (tz < 0) ? 3 : 0;
  constexpr int kStepW = (3 - W % 3) % 3;  // (-W) mod 3: the change of tz per block
  for (int tau0 = 0; tau0 < tau_end; tau0 += W, tz = (tz + kStepW >= 3) ? tz + kStepW - 3 : tz + kStepW) {
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const int tau = tau0 + u;
      if (tau < tau_end) {
        load_row(ybase + tau + 1, xw[(u + 1) % W], bw[(u + 1) % W]);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const int j = ybase + tau - s;
          if (tau - s >= 0 && tau - s < L && j >= 0 && j < n) {
            const int cf_ = ((2 * s - u) % 3 + 3) % 3, cr_ = ((2 - u) % 3 + 3) % 3;  // folded at compile time
            int m = tz + (reverse ? cr_ : cf_);
            m -= (m >= 3) ? 3 : 0;
            update_row(xw[(u - s + 4 * W) % W], xw[(u - s + 1 + 4 * W) % W], xw[(u - s - 1 + 4 * W) % W],
                       bw[(u - s + 4 * W) % W], j, s, m);
          }
        }
        const int ro = ybase + tau - S + 1;
        if (ro >= r0 && ro < r1) {
          const T(&xr)[3] = xw[(u - S + 1 + 4 * W) % W];
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const int cl = 3 * lane + e;
            const int gx = cbase + e;
            if (cl >= S && cl < kWR - S && gx < n) xo[(int64_t)ro * n + gx] = G(xr[e]);
          }
        }
      }
    }
  }
}

// b' = b / c on the finest level (the multigrid's scaled right-hand side)
template <typename T, typename G, typename Tin = T>
__global__ void k_scale_rhs(G* __restrict__ bs, const Tin* __restrict__ b, int n, const Coef<T>* __restrict__ coef,
                            int coef_class, int J, int K) {
  const int N = n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int slice = blockIdx.y;
  const Coef<T> cf = slice_coef(coef, coef_class, slice, J, K, K);
  const int64_t i = (int64_t)slice * N + p;
  bs[i] = G(T(b[i]) * cf.inv_c);
}

// x += P xc (used when there is no post-smoothing to fuse the correction into)
template <typename T, typename G>
__global__ void k_prolong_add(G* __restrict__ x, const G* __restrict__ xc, int nf, int lshape) {
  const int N = nf * nf;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int nc = (nf - 1) / 2;
  const int slice = blockIdx.y;
  const int iy = p / nf, ix = p - iy * nf;
  if (outside_domain(ix, iy, nf, lshape)) return;
  const int64_t i = (int64_t)slice * N + p;
  x[i] = G(T(x[i]) + prolong_value<T>(xc + (int64_t)slice * nc * nc, nc, ix + 1, iy + 1));
}

// ---------------------------------------------------------------------------------------
// Residual and restriction in one pass: the coarse scaled right-hand side D_c^-1 P^T (b - C x)
// on a tile of CTX x CTY coarse points.  Coarse point (cx, cy) is fine interior point (2cx+1, 2cy+1); its restriction reads
// the fine residual there and at the midpoints of its six coarse edges, so the block forms the
// residual on the (2 CTX + 1) x (2 CTY + 1) fine points it covers (neighbouring tiles share one
// fine row/column) from x staged with a one-point halo.
// ---------------------------------------------------------------------------------------
constexpr int kRCX = 32, kRCY = 16;
constexpr int kRFX = 2 * kRCX + 1, kRFY = 2 * kRCY + 1;  // residual points
constexpr int kRXX = kRFX + 2, kRXY = kRFY + 2;          // x points (one-point halo)
constexpr int kRZ = (kRFX + 2) / 3;                      // groups of three columns of a residual row

// a b + c: one fused multiply-add in binary32 and binary64, the two double-float operations in
// double-float
__device__ __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ df64 mad(df64 a, df64 b, df64 c) { return a * b + c; }

template <typename T, typename G, bool DIAG>
__global__ void __launch_bounds__(256) k_residual_restrict(G* __restrict__ bc, const G* __restrict__ x,
                                                           const G* __restrict__ b, int n,
                                                           const Coef<T>* __restrict__ coef, int coef_class, int J,
                                                           int K, int level, int lshape, int zc) {
  __shared__ T xs[kRXY * kRXX];
  __shared__ T rs[kRFY * kRFX];
  const int nc = (n - 1) / 2;
  const int slice = blockIdx.z;
  const int64_t off = (int64_t)slice * n * n;
  const G* xsl = x + off;
  const G* bsl = b + off;
  const int cx0 = blockIdx.x * kRCX, cy0 = blockIdx.y * kRCY;
  const int fx0 = 2 * cx0, fy0 = 2 * cy0;  // first residual point (fine interior index)
  const Coef<T> cf = slice_coef(coef, coef_class, slice, J, K, level);
  // scaled residual r' = D^-1 (b - C x) = b' - x - (ax/c) sx - (ay/c) sy - (dg/c) sd at fine point
  // (fx0 + rx, gy), 0 outside the grid or the domain
  auto residual_at = [&](int rx, int ry, int gy) -> T {
    const int gx = fx0 + rx;
    if (gx >= n || gy >= n || outside_domain(gx, gy, n, lshape)) return T(0);
    const int i = (ry + 1) * kRXX + (rx + 1);
    T v = T(bsl[(int64_t)gy * n + gx]) - cf.axs * (xs[i - 1] + xs[i + 1]);
    v -= cf.ays * (xs[i - kRXX] + xs[i + kRXX]);
    if (DIAG) v -= cf.dgs * (xs[i + kRXX + 1] + xs[i - kRXX - 1]);
    return v - xs[i];
  };
  if constexpr (sizeof(T) == 4) {
    // binary32 is bound by instruction issue: rows by warp and columns by lane, no division
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = 8;  // launched with 256 threads
    for (int ry = warp; ry < kRXY; ry += kWarps) {
      const int gy = fy0 - 1 + ry;
      const bool row_in = gy >= 0 && gy < n;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int rx = lane + 32 * e;
        if (rx >= kRXX) break;
        const int gx = fx0 - 1 + rx;
        const bool in = row_in && gx >= 0 && gx < n && !outside_domain(gx, gy, n, lshape);
        xs[ry * kRXX + rx] = in ? T(xsl[(int64_t)gy * n + gx]) : T(0);
      }
    }
    __syncthreads();
    for (int ry = warp; ry < kRFY; ry += kWarps) {
      const int gy = fy0 + ry;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int rx = lane + 32 * e;
        if (rx >= kRFX) break;
        rs[ry * kRFX + rx] = residual_at(rx, ry, gy);
      }
    }
  } else {
    // binary64 is bound by the FP64 pipe: flat loops keep every lane busy
    for (int idx = threadIdx.x; idx < kRXY * kRXX; idx += blockDim.x) {
      const int ry = idx / kRXX, rx = idx - ry * kRXX;
      const int gx = fx0 - 1 + rx, gy = fy0 - 1 + ry;
      const bool in = gx >= 0 && gx < n && gy >= 0 && gy < n && !outside_domain(gx, gy, n, lshape);
      xs[idx] = in ? T(xsl[(int64_t)gy * n + gx]) : T(0);
    }
    __syncthreads();
    if (zc >= 0) {
      // the residual of colour zc is exactly 0: the binary64 pipe forms only the other two
      for (int idx = threadIdx.x; idx < kRFY * 2 * kRZ; idx += blockDim.x) {
        const int ry = idx / (2 * kRZ), q = idx - ry * (2 * kRZ);
        int ph = (zc - fx0 - (fy0 + ry) - 2) % 3;
        ph += (ph < 0) ? 3 : 0;
        const int rx = 3 * (q >> 1) + (ph + 1 + (q & 1)) % 3;
        if (rx < kRFX) rs[ry * kRFX + rx] = residual_at(rx, ry, fy0 + ry);
      }
      for (int idx = threadIdx.x; idx < kRFY * kRZ; idx += blockDim.x) {
        const int ry = idx / kRZ, j = idx - ry * kRZ;
        int ph = (zc - fx0 - (fy0 + ry) - 2) % 3;
        ph += (ph < 0) ? 3 : 0;
        if (3 * j + ph < kRFX) rs[ry * kRFX + 3 * j + ph] = T(0);
      }
    } else {
      for (int idx = threadIdx.x; idx < kRFY * kRFX; idx += blockDim.x) {
        const int ry = idx / kRFX, rx = idx - ry * kRFX;
        rs[idx] = residual_at(rx, ry, fy0 + ry);
      }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kRCX * kRCY; idx += blockDim.x) {
    const int ty = idx / kRCX, tx = idx - ty * kRCX;
    const int cx = cx0 + tx, cy = cy0 + ty;
    if (cx >= nc || cy >= nc) continue;
    if (outside_domain(cx, cy, nc, lshape)) {
      bc[(int64_t)slice * nc * nc + (int64_t)cy * nc + cx] = G(0.0f);
      continue;
    }
    const int i = (2 * ty + 1) * kRFX + (2 * tx + 1);
    T e = (rs[i - 1] + rs[i + 1]) + (rs[i - kRFX] + rs[i + kRFX]) + (rs[i + kRFX + 1] + rs[i - kRFX - 1]);
    // coarse scaled rhs: D_c^-1 P^T D r' = (c / c_coarse) P^T r', as one fma onto the rounded
    // edge term (the order the fused restriction of the wide Gauss-Seidel kernel uses)
    bc[(int64_t)slice * nc * nc + (int64_t)cy * nc + cx] = G(mad(cf.rho, rs[i], (T(0.5) * cf.rho) * e));
  }
}

// exact solve on level 1 (one unknown per slice)
template <typename G>
__global__ void k_coarse1(G* __restrict__ x, const G* __restrict__ b, int nslices) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  // one unknown: the scaled right-hand side is the solution
  x[s] = b[s];
}



// Tile shapes (chosen by measurement on GB300): binary64 is bound by the FP64 pipe, so one sweep
// per launch keeps the halo recomputation small (3-point halo, 90 x 26 interior; 49 KB of shared
// memory, 4 blocks per SM to hide shared-memory latency); binary32 is bound by memory, so the
// pre- or post-smoothing sweeps are fused three to a launch (9-point halo, 78 x 46 interior,
// 4 blocks per SM), reading x and b once and writing x once per three sweeps.
template <typename T>
struct SweepShape;
#ifndef ST_GS_HR64
#define ST_GS_HR64 34
#endif
#ifndef ST_GS_HR32
#define ST_GS_HR32 64
#endif
#ifndef ST_GS_SEG
#define ST_GS_SEG 64
#endif
#ifndef ST_GS_NSW32
#define ST_GS_NSW32 3
#endif
template <>
struct SweepShape<double> {
  static constexpr int kFusedNSW = 1, kFusedHR = ST_GS_HR64, kSingleHR = ST_GS_HR64;
};
template <>
struct SweepShape<df64> {  // 8-byte values like binary64; one sweep per launch
  static constexpr int kFusedNSW = 1, kFusedHR = ST_GS_HR64, kSingleHR = ST_GS_HR64;
};
template <>
struct SweepShape<float> {
  static constexpr int kFusedNSW = ST_GS_NSW32, kFusedHR = ST_GS_HR32, kSingleHR = 64;
};

// the autotuner's element-type index: 0 binary64, 1 binary32, 2 double-float
template <typename T>
constexpr int type_slot() {
  return std::is_same<T, df64>::value ? 2 : (sizeof(T) == 4 ? 1 : 0);
}

template <typename T, typename G, int NSW, int HR, bool DIAG, bool PROL>
cudaError_t gs_launch(const st_handle_s* h, int k, int nslices, int cls, G* x_out, const G* x_in, const G* b,
                      const G* xc, bool reverse, bool zero_init) {
  constexpr int H = 3 * NSW;
  const int n = (1 << k) - 1;
  const int TX = kWR - 2 * H, TY = HR - 2 * H;
  dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, nslices);
  const size_t smem = 2 * sizeof(T) * HR * kWR;
  // profiled: the finest level, which carries three quarters of the sweep work
  const bool prof = (k == h->K) && prof_start(h);
  k_gs_sweep<T, G, NSW, HR, DIAG, PROL><<<grid, 256, smem, h->stream>>>(x_out, x_in, b, xc, n, coef_table<T>(h),
                                                                         cls, h->J, h->K, k, reverse ? 1 : 0,
                                                                         zero_init ? 1 : 0, h->domain);
  count_launch(h);
  if (prof) {
    // per point and sweep: 3 adds + 1 fma (+ 1 add + 1 fma with diagonal couplings);
    // bytes: read x and b, write x (x is not read when the launch starts from x = 0), and the
    // coarse iterate when the launch adds the prolongated correction
    const double pts = (double)n * n * nslices;
    const double nc = (double)((n - 1) / 2);
    prof_stop(h, (DIAG ? 1 : 0) + (sizeof(T) == 4 ? 2 : 0), pts * NSW * (DIAG ? 6.0 : 4.0),
              sizeof(G) * (pts * (zero_init ? 2.0 : 3.0) + (PROL ? nc * nc * nslices : 0.0)));
  }
  return cudaGetLastError();
}

template <typename T, typename G, int NSW, bool DIAG, bool PROL>
cudaError_t wave_launch(const st_handle_s* h, int k, int nslices, int cls, G* x_out, const G* x_in, const G* b,
                        const G* xc, bool reverse, bool zero_init) {
  constexpr int S = 3 * NSW;
  const int n = (1 << k) - 1;
  const int TXW = kWR - 2 * S;
  const int nstrips = (n + TXW - 1) / TXW;
  // rows per segment: the autotuned or forced choice, else the compiled default; at most n
  const int chosen = h->gs_seg[type_slot<T>()][DIAG ? 1 : 0][k];
  const int seg = min(chosen > 0 ? chosen : ST_GS_SEG, n);
  const int nseg = (n + seg - 1) / seg;
  const int64_t warps = (int64_t)nstrips * nseg * nslices;
  const unsigned blocks = (unsigned)((warps * 32 + 127) / 128);
  const bool prof = (k == h->K) && prof_start(h);
  k_gs_wave<T, G, S, DIAG, PROL><<<blocks, 128, 0, h->stream>>>(x_out, x_in, b, xc, n, coef_table<T>(h), cls,
                                                                 h->J, h->K, k, reverse ? 1 : 0, zero_init ? 1 : 0,
                                                                 h->domain, nstrips, nseg, seg, nslices);
  count_launch(h);
  if (prof) {
    const double pts = (double)n * n * nslices;
    const double nc = (double)((n - 1) / 2);
    prof_stop(h, (DIAG ? 1 : 0) + (sizeof(T) == 4 ? 2 : 0), pts * NSW * (DIAG ? 6.0 : 4.0),
              sizeof(G) * (pts * (zero_init ? 2.0 : 3.0) + (PROL ? nc * nc * nslices : 0.0)));
  }
  return cudaGetLastError();
}

// nsw consecutive sweeps of one colour order from x_in (+ P xc if xc != nullptr) into x_out
// (x_in == x_out is not allowed)
// Which Gauss-Seidel kernel a launch uses: the handle's autotuned choice per element type,
// coupling pattern and level (0: shared-memory tiles, the default; 1: register wavefront;
// 2 + s: register tiles of block shape s).
template <typename T>
int gs_kind(const st_handle_s* h, bool diag, int k) {
  return h->gs_kind[type_slot<T>()][diag ? 1 : 0][k];
}

// Whether pre-smoothing on level k runs the wide binary32 kernel, whose last launch can also form
// and restrict the residual (wide_launch_restrict)
template <typename T>
bool wide_restricts(const st_handle_s* h, bool diag, int k) {
  if (!std::is_same<T, float>::value) return false;
  const int kind = gs_kind<T>(h, diag, k);
  return kind == 5 && wide_fits(h, 0, k);
}

// bc != nullptr (only where wide_restricts): the launch also writes the coarse right-hand side
template <typename T, typename G, bool DIAG>
cudaError_t gs_sweeps(const st_handle_s* h, int k, int nslices, int cls, G* x_out, const G* x_in, const G* b,
                      const G* xc, bool reverse, bool zero_init, int nsw, G* bc = nullptr) {
  constexpr int F = SweepShape<T>::kFusedNSW;
  if constexpr (std::is_same<T, float>::value) {
    if (bc) {
      return (F > 1 && nsw == F)
                 ? wide_launch_restrict<G, F, DIAG>(h, 0, k, nslices, cls, x_out, x_in, b, bc, zero_init)
                 : wide_launch_restrict<G, 1, DIAG>(h, 0, k, nslices, cls, x_out, x_in, b, bc, zero_init);
    }
  }
  {
    const int kind = gs_kind<T>(h, DIAG, k);
    if (kind >= 2) {  // register tiles, block shape kind - 2
      const int sh = kind - 2;
      if (F > 1 && nsw == F)
        return xc ? reg_launch<T, G, F, DIAG, true>(h, sh, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init)
                  : reg_launch<T, G, F, DIAG, false>(h, sh, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
      return xc ? reg_launch<T, G, 1, DIAG, true>(h, sh, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init)
                : reg_launch<T, G, 1, DIAG, false>(h, sh, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
    }
  }
  if (gs_kind<T>(h, DIAG, k) == 1) {
    if (F > 1 && nsw == F)
      return xc ? wave_launch<T, G, F, DIAG, true>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init)
                : wave_launch<T, G, F, DIAG, false>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
    return xc ? wave_launch<T, G, 1, DIAG, true>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init)
              : wave_launch<T, G, 1, DIAG, false>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
  }
  constexpr int FHR = SweepShape<T>::kFusedHR, HR1 = SweepShape<T>::kSingleHR;
  if (F > 1 && nsw == F) {
    return xc ? gs_launch<T, G, F, FHR, DIAG, true>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init)
              : gs_launch<T, G, F, FHR, DIAG, false>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
  }
  return xc ? gs_launch<T, G, 1, HR1, DIAG, true>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init)
            : gs_launch<T, G, 1, HR1, DIAG, false>(h, k, nslices, cls, x_out, x_in, b, xc, reverse, zero_init);
}

// One V-cycle on level k.  xb[0], xb[1] are the level's two iterate buffers and *cur the one
// holding the iterate; every sweep moves it to the other buffer.  braw != nullptr (binary32, the
// finest level's first V-cycle, one pre-smoothing launch that also restricts): b' = b / c is not
// there yet; that launch forms it from braw and writes it to bsc (= b).
template <typename T, typename G, bool DIAG>
cudaError_t vcycle(const st_handle_s* h, int k, int nslices, int cls, G* const xb[2], int* cur, const G* b,
                   bool x_is_zero, const T* braw = nullptr, G* bsc = nullptr) {
  const st::MGLevels& L = h->mg;
  const int n = (1 << k) - 1;
  const int N = n * n;
  cudaError_t e;
  if (k == L.kmin) {
    if (k == 1)
      k_coarse1<G><<<(nslices + 255) / 256, 256, 0, h->stream>>>(xb[*cur], b, nslices);
    else
      k_coarse_dense3<T, G><<<(nslices + 127) / 128, 128, 0, h->stream>>>(xb[*cur], b, nslices, coef_table<T>(h),
                                                                           cls, h->J, h->K, h->domain);
    count_launch(h);
    return cudaGetLastError();
  }
  G* bc = reinterpret_cast<G*>(L.bc[k - 1]);
  // the wide binary32 kernel forms and restricts the residual in its last pre-smoothing launch
  const bool fused = h->cfg.n_pre > 0 && wide_restricts<T>(h, DIAG, k);
  for (int s = 0; s < h->cfg.n_pre;) {
    const int nsw = (h->cfg.n_pre - s >= SweepShape<T>::kFusedNSW) ? SweepShape<T>::kFusedNSW : 1;
    if constexpr (std::is_same<T, float>::value && std::is_same<G, float>::value) {
      if (braw) {  // the caller checked: one launch of all n_pre sweeps, fused restriction
        if ((e = wide_launch_scale_restrict<DIAG>(h, k, nslices, cls, xb[*cur ^ 1], braw, bsc, bc)) != cudaSuccess)
          return e;
        *cur ^= 1;
        s += nsw;
        continue;
      }
    }
    G* bco = (fused && s + nsw == h->cfg.n_pre) ? bc : nullptr;
    if ((e = gs_sweeps<T, G, DIAG>(h, k, nslices, cls, xb[*cur ^ 1], xb[*cur], b, nullptr, false,
                                x_is_zero && s == 0, nsw, bco)) != cudaSuccess)
      return e;
    *cur ^= 1;
    s += nsw;
  }
  if (h->cfg.n_pre == 0 && x_is_zero) {
    // nothing smoothed yet: the iterate must hold zeros before the residual is formed
    if ((e = cudaMemsetAsync(xb[*cur], 0, sizeof(G) * (size_t)N * nslices, h->stream)) != cudaSuccess) return e;
  }
  G* x = xb[*cur];
  if (!fused) {
    const int nc = (1 << (k - 1)) - 1;
    dim3 gr((nc + kRCX - 1) / kRCX, (nc + kRCY - 1) / kRCY, nslices);
    // pre-smoothing ends with a colour-2 step, which set those points from the same operations
    // the residual uses, on neighbours that have not changed since: their residual is exactly 0
    // (not so after no pre-smoothing, or for an iterate stored narrower than it is computed).
    // Only binary64 and double-float, bound by their arithmetic, gain from not forming them
    // (measured: binary32 issue-bound lanes lose more to the uneven enumeration than they save).
    const int zc = (h->cfg.n_pre > 0 && std::is_same<T, G>::value && sizeof(T) != 4) ? 2 : -1;
    k_residual_restrict<T, G, DIAG><<<gr, 256, 0, h->stream>>>(bc, x, b, n, coef_table<T>(h), cls, h->J, h->K, k,
                                                               h->domain, zc);
    count_launch(h);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  G* const xcb[2] = {reinterpret_cast<G*>(L.xc[k - 1]), reinterpret_cast<G*>(L.xc2[k - 1])};
  int ccur = 0;
  if ((e = vcycle<T, G, DIAG>(h, k - 1, nslices, cls, xcb, &ccur, bc, true)) != cudaSuccess) return e;
  if (h->cfg.n_post == 0) {
    dim3 g1((N + 255) / 256, nslices);
    k_prolong_add<T, G><<<g1, 256, 0, h->stream>>>(x, xcb[ccur], n, h->domain);
    count_launch(h);
    return cudaGetLastError();
  }
  for (int s = 0; s < h->cfg.n_post;) {
    const int nsw = (h->cfg.n_post - s >= SweepShape<T>::kFusedNSW) ? SweepShape<T>::kFusedNSW : 1;
    // the first post-smoothing launch also applies the coarse-grid correction x += P xc
    if ((e = gs_sweeps<T, G, DIAG>(h, k, nslices, cls, xb[*cur ^ 1], xb[*cur], b, s == 0 ? xcb[ccur] : nullptr, true,
                                false, nsw)) != cudaSuccess)
      return e;
    *cur ^= 1;
    s += nsw;
  }
  return cudaSuccess;
}

// x = the iterate, widened from the storage type (bfloat16 storage of binary32 work; double-float
// work into binary64)
template <typename T, typename G>
__global__ void k_widen(T* __restrict__ x, const G* __restrict__ g, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = T(g[i]);
}

// the same in place: element i of a buffer of 8-byte double-float values becomes a double
__global__ void k_widen_df_inplace(void* buf, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const df64 v = reinterpret_cast<const df64*>(buf)[i];
    reinterpret_cast<double*>(buf)[i] = double(v);
  }
}

}  // namespace

cudaError_t launch_make_coef(Coef<double>* coef, int K, int J, double alpha, Phys ph, int dim, cudaStream_t s) {
  k_make_coef<double><<<1, 256, 0, s>>>(coef, K, J, alpha, ph, dim);
  return cudaGetLastError();
}

cudaError_t launch_make_coef_df(Coef<df64>* coef, int K, int J, double alpha, Phys ph, int dim, cudaStream_t s) {
  k_make_coef<df64><<<1, 256, 0, s>>>(coef, K, J, alpha, ph, dim);
  return cudaGetLastError();
}

cudaError_t launch_make_coef32(Coef<float>* coef, int K, int J, double alpha, Phys ph, int dim, cudaStream_t s) {
  k_make_coef<float><<<1, 256, 0, s>>>(coef, K, J, alpha, ph, dim);
  return cudaGetLastError();
}

template <typename T, typename G, int NSW, int HR>
cudaError_t set_smem_attr() {
  const int smem = 2 * sizeof(T) * HR * kWR;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_gs_sweep<T, G, NSW, HR, true, true>, attr, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gs_sweep<T, G, NSW, HR, true, false>, attr, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gs_sweep<T, G, NSW, HR, false, true>, attr, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gs_sweep<T, G, NSW, HR, false, false>, attr, smem);
  return e;
}

cudaError_t mg_set_attributes() {
  using SD = SweepShape<double>;
  using SF = SweepShape<float>;
  cudaError_t e = set_smem_attr<double, double, SD::kFusedNSW, SD::kFusedHR>();
  if (e == cudaSuccess) e = set_smem_attr<double, double, 1, SD::kSingleHR>();
  if (e == cudaSuccess) e = set_smem_attr<float, float, SF::kFusedNSW, SF::kFusedHR>();
  if (e == cudaSuccess) e = set_smem_attr<float, float, 1, SF::kSingleHR>();
  if (e == cudaSuccess) e = set_smem_attr<float, __nv_bfloat16, SF::kFusedNSW, SF::kFusedHR>();
  if (e == cudaSuccess) e = set_smem_attr<float, __nv_bfloat16, 1, SF::kSingleHR>();
  if (e == cudaSuccess) e = set_smem_attr<df64, df64, 1, SweepShape<df64>::kSingleHR>();
  if (e == cudaSuccess) e = wide_set_attributes();
  return e;
}

// x = K b on nslices slices: n_vcycles V-cycles from x = 0.  The multigrid keeps its vectors in
// the storage type G (T, or binary16 bfloat16 for binary32 work) and computes in T.
template <typename T, typename G>
cudaError_t mg_run(const st_handle_s* h, int nslices, int coef_class, const T* b, T* x) {
  // class 0 (K_x: s = 0) has no diagonal couplings unless D has d12 != 0 or c != 0; the K_l
  // classes always do
  const bool diag = coef_class != 0 || h->diag0;
  constexpr bool same = std::is_same<T, G>::value;
  const size_t npts = (size_t)h->Nx * nslices;
  // iterate buffers: the output and the alternate buffer, or (narrower storage) two halves of
  // the alternate buffer, which holds 2 B N_t N_x doubles
  G* const xb[2] = {same ? reinterpret_cast<G*>(x) : reinterpret_cast<G*>(h->Xalt),
                    same ? reinterpret_cast<G*>(h->Xalt) : reinterpret_cast<G*>(h->Xalt) + npts};
  int cur = 0;
  G* bs = reinterpret_cast<G*>(h->Bs);
  const int n = h->n;
  // binary32 on the wide regions with one pre-smoothing launch: the scaling b' = b / c is formed
  // by that launch of the first V-cycle
  const bool fuse_scale = std::is_same<T, float>::value && std::is_same<G, float>::value && h->cfg.n_vcycles > 0 &&
                          h->cfg.n_pre == SweepShape<T>::kFusedNSW && wide_restricts<T>(h, diag, h->K);
  cudaError_t e = cudaSuccess;
  if (!fuse_scale) {
    dim3 gs((n * n + 255) / 256, nslices);
    k_scale_rhs<T, G><<<gs, 256, 0, h->stream>>>(bs, b, n, coef_table<T>(h), coef_class, h->J, h->K);
    count_launch(h);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (int c = 0; c < h->cfg.n_vcycles; ++c) {
    const T* braw = (fuse_scale && c == 0) ? b : nullptr;
    e = diag ? vcycle<T, G, true>(h, h->K, nslices, coef_class, xb, &cur, bs, c == 0, braw, bs)
             : vcycle<T, G, false>(h, h->K, nslices, coef_class, xb, &cur, bs, c == 0, braw, bs);
    if (e != cudaSuccess) return e;
  }
  if (h->cfg.n_vcycles == 0) return cudaMemsetAsync(x, 0, sizeof(T) * npts, h->stream);
  if (!same) {
    k_widen<T, G><<<(unsigned)((npts + 255) / 256), 256, 0, h->stream>>>(x, xb[cur], (int64_t)npts);
    count_launch(h);
    return cudaGetLastError();
  }
  // an odd total number of sweeps leaves the iterate in the alternate buffer
  if (cur == 1) return cudaMemcpyAsync(x, xb[1], sizeof(T) * npts, cudaMemcpyDeviceToDevice, h->stream);
  return cudaSuccess;
}

// binary64 in and out, the multigrid in double-float: the iterate lives in x's memory (8 bytes a
// value either way) and the alternate buffer, and is widened to binary64 at the end
cudaError_t mg_apply_df(const st_handle_s* h, int nslices, int coef_class, const double* b, double* x) {
  using D = df64;
  const bool diag = coef_class != 0 || h->diag0;
  const size_t npts = (size_t)h->Nx * nslices;
  D* const xb[2] = {reinterpret_cast<D*>(x), reinterpret_cast<D*>(h->Xalt)};
  int cur = 0;
  D* bs = reinterpret_cast<D*>(h->Bs);
  const int n = h->n;
  k_scale_rhs<D, D, double><<<dim3((n * n + 255) / 256, nslices), 256, 0, h->stream>>>(bs, b, n, coef_table<D>(h),
                                                                                      coef_class, h->J, h->K);
  count_launch(h);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int c = 0; c < h->cfg.n_vcycles; ++c) {
    e = diag ? vcycle<D, D, true>(h, h->K, nslices, coef_class, xb, &cur, bs, c == 0)
             : vcycle<D, D, false>(h, h->K, nslices, coef_class, xb, &cur, bs, c == 0);
    if (e != cudaSuccess) return e;
  }
  if (h->cfg.n_vcycles == 0) return cudaMemsetAsync(x, 0, sizeof(double) * npts, h->stream);
  const unsigned blocks = (unsigned)((npts + 255) / 256);
  if (cur == 1)
    k_widen<double, D><<<blocks, 256, 0, h->stream>>>(x, xb[1], (int64_t)npts);
  else
    k_widen_df_inplace<<<blocks, 256, 0, h->stream>>>(x, (int64_t)npts);
  count_launch(h);
  return cudaGetLastError();
}

template <typename T>
cudaError_t mg_apply(const st_handle_s* h, int nslices, int coef_class, const T* b, T* x) {
  if constexpr (std::is_same<T, double>::value) {
    if (h->mg_df) return h->domain == 2 ? mg_apply3_df(h, nslices, coef_class, b, x)
                                        : mg_apply_df(h, nslices, coef_class, b, x);
  }
  if (h->domain == 2) return mg_apply3<T>(h, nslices, coef_class, b, x);
  return mg_run<T, T>(h, nslices, coef_class, b, x);
}

cudaError_t mg_apply_bf16(const st_handle_s* h, int nslices, int coef_class, const float* b, float* x) {
  return mg_run<float, __nv_bfloat16>(h, nslices, coef_class, b, x);
}

// Times the Gauss-Seidel kernels on every level of the handle's shapes (the pre-smoothing launch
// of a V-cycle: K_x on 2 B N_t slices, K_l on B N_t slices) and keeps the fastest per element
// type, coupling pattern and level.  The wavefront is timed at several segment lengths,
// ceil(n / q) rows for q = 1 .. 12 segments per strip: fewer segments recompute fewer overlap
// rows (2 S per segment), more segments fill the GPU's last wave of warps better.  Uses the
// workspace as scratch.  ms[0..2]: shared-memory tiles, wavefront (best length), register tiles
// (best block shape).
template <typename T, bool DIAG>
cudaError_t autotune_one(st_handle_s* h, int k, float* ms) {
  const int nslices = (int)((DIAG ? 1 : 2) * h->B * h->Nt);
  const int cls = DIAG ? -1 : 0;
  const int n = (1 << k) - 1;
  T* xo = reinterpret_cast<T*>(h->X);
  const T* xi = reinterpret_cast<const T*>(h->Xalt);
  const T* b = reinterpret_cast<const T*>(h->Bs);
  const int nsw = SweepShape<T>::kFusedNSW;
  unsigned char& kind_sel = h->gs_kind[type_slot<T>()][DIAG ? 1 : 0][k];
  unsigned short& seg_sel = h->gs_seg[type_slot<T>()][DIAG ? 1 : 0][k];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = cudaSuccess;
  auto time_it = [&](float* out) {
    float t = 1e30f;
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
      cudaEventRecord(e0, h->stream);
      err = gs_sweeps<T, T, DIAG>(h, k, nslices, cls, xo, xi, b, nullptr, false, false, nsw);
      cudaEventRecord(e1, h->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float t1 = 0.f;
      if (err == cudaSuccess) cudaEventElapsedTime(&t1, e0, e1);
      if (rep > 0) t = t1 < t ? t1 : t;  // the first run warms up
    }
    *out = t;
  };
  float t_tile = 1e30f, t_wave = 1e30f, t_reg = 1e30f;
  int best_seg = 0, last_seg = -1, best_reg = 2;
  kind_sel = 0;
  time_it(&t_tile);
  {
    // register tiles: every block shape (binary64 and double-float have one)
    for (int sh = 0; sh < (sizeof(T) == 4 ? kRegShapes : 1) && err == cudaSuccess; ++sh) {
      kind_sel = (unsigned char)(2 + sh);
      float t;
      time_it(&t);
      if (t < t_reg) {
        t_reg = t;
        best_reg = 2 + sh;
      }
    }
  }
  kind_sel = 1;
  for (int q = 1; q <= 12 && err == cudaSuccess; ++q) {
    const int seg = (n + q - 1) / q;
    if (seg == last_seg) continue;
    last_seg = seg;
    seg_sel = (unsigned short)seg;
    float t;
    time_it(&t);
    if (t < t_wave) {
      t_wave = t;
      best_seg = seg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  kind_sel = (t_wave < t_tile && t_wave < t_reg) ? 1 : (t_reg < t_tile ? best_reg : 0);
  seg_sel = (unsigned short)best_seg;
  ms[0] = t_tile;
  ms[1] = t_wave;
  ms[2] = t_reg;
  return err;
}

cudaError_t mg_autotune(st_handle_s* h, float* table) {
  if (h->domain == 2) return cudaSuccess;  // the cube has one Gauss-Seidel kernel
  const size_t bytes = sizeof(double) * 2 * (size_t)h->B * h->Nt * h->Nx;
  cudaError_t e = cudaMemsetAsync(h->Xalt, 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Bs, 0, bytes, h->stream);
  const bool saved = h->prof_on;
  h->prof_on = false;
  for (int k = h->mg.kmin + 1; k <= h->K && e == cudaSuccess; ++k) {
    float* row = table + 12 * k;
    if (e == cudaSuccess) e = autotune_one<double, false>(h, k, row + 0);
    if (e == cudaSuccess) e = autotune_one<double, true>(h, k, row + 3);
    if (e == cudaSuccess) e = autotune_one<float, false>(h, k, row + 6);
    if (e == cudaSuccess) e = autotune_one<float, true>(h, k, row + 9);
    if (e == cudaSuccess && h->mg_df) {  // double-float kernels, recorded in their own slot only
      float t[3];
      e = autotune_one<df64, false>(h, k, t);
      if (e == cudaSuccess) e = autotune_one<df64, true>(h, k, t);
    }
  }
  h->prof_on = saved;
  return e;
}

template cudaError_t mg_apply<double>(const st_handle_s*, int, int, const double*, double*);
template cudaError_t mg_apply<float>(const st_handle_s*, int, int, const float*, float*);

}  // namespace st
