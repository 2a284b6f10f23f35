// Internal declarations of libst: handle layout, kernel launchers, shared helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/st.h"
#include "df64.cuh"

namespace st {

// ---------------------------------------------------------------------------------------
// Multigrid operator coefficients.  On mesh level k (h = 2^-k) the P1 matrix
// C = a A_x + s M_x has a 7-point stencil (x neighbours, y neighbours, (1,1)/(-1,-1)
// diagonal neighbours); for the heat equation (A_x: 5-point Laplacian; M_x: h^2/12 [6; 1 x 6]
// on the (i,j)-(i+1,j+1) triangulation) it is centre 4a + s h^2/2, axis neighbours
// -a + s h^2/12, diagonal s h^2/12.  Phys below gives the general reaction-diffusion one.
// One entry per (coefficient class, level).  Class 0 is K_x (a = 1, s = 0); class 1 + l is
// K_l (a = alpha, s = 2^l), l = 0..J.
// The multigrid works with the Jacobi-scaled system D^-1 C x = D^-1 b (D = the centre
// coefficient of the level): Gauss-Seidel is invariant under that row scaling, and it saves the
// division of every update.  The right-hand side of every level is stored scaled.
// ---------------------------------------------------------------------------------------
template <typename T>
struct Coef {
  T inv_c;  // 1 / centre
  T c;      // centre
  T ax;     // coefficient of the x neighbours (+-1, 0)
  T ay;     // coefficient of the y neighbours (0, +-1)
  T dg;     // coefficient of the (1,1) / (-1,-1) diagonal neighbours
  T axs;    // ax / c
  T ays;    // ay / c
  T dgs;    // dg / c
  T rho;    // c of this level / c of the next coarser level (rescales restricted residuals)
  T pad;
};

// Constant coefficients of the reaction-diffusion form of Sec. 4, a(eta, zeta) =
// <D grad eta, grad zeta> + c <eta, zeta> with D = [[d11, d12], [d12, d22]] (D = Id, c = 0: the
// heat equation).  On the mesh (squares cut along their (1,1) diagonal) the P1 stiffness of D is
// the 7-point stencil centre 2(d11 + d22 - d12), x neighbours d12 - d11, y neighbours d12 - d22,
// (1,1)/(-1,-1) neighbours -d12; c adds c times the mass stencil h^2/12 [6; 1 at the six].
struct Phys {
  double d11, d12, d22, c;
};

// A 7-point stencil [centre; x, y, (1,1)/(-1,-1) neighbours] in element type T.
template <typename T>
struct Stencil7 {
  T c0, cx, cy, cd;
};

// The stencil of a A_x + s M_x on mesh width h (A_x = <D grad, grad> + c M_x).
inline Stencil7<double> operator_stencil(const Phys& ph, double a, double s, double h) {
  const double m = (a * ph.c + s) * h * h / 12.0;
  return Stencil7<double>{a * 2.0 * (ph.d11 + ph.d22 - ph.d12) + 6.0 * m, a * (ph.d12 - ph.d11) + m,
                          a * (ph.d12 - ph.d22) + m, -a * ph.d12 + m};
}

// Nested P1 prolongation: the value at fine grid node (i, j) (1-based grid indices, coarse grid of
// nc x nc interior nodes stored in cs) of the coarse P1 function: the coarse value at even-even
// nodes, the average of the two coarse end points at the midpoints of horizontal, vertical and
// (1,1)-diagonal coarse edges; coarse boundary values are 0.  Branch-free: with (I, J) = (i >> 1,
// j >> 1) it is the average of the coarse values at (I, J) and (I + i mod 2, J + j mod 2); at
// even-even nodes both are the same node and the average is exact.  G is the storage type.
template <typename T, typename G>
__device__ __forceinline__ T prolong_value(const G* __restrict__ cs, int nc, int i, int j) {
  const int I0 = i >> 1, J0 = j >> 1, I1 = I0 + (i & 1), J1 = J0 + (j & 1);
  const T a = (I0 >= 1 && I0 <= nc && J0 >= 1 && J0 <= nc) ? T(cs[(J0 - 1) * nc + (I0 - 1)]) : T(0);
  const T b = (I1 >= 1 && I1 <= nc && J1 >= 1 && J1 <= nc) ? T(cs[(J1 - 1) * nc + (I1 - 1)]) : T(0);
  return T(0.5) * (a + b);
}

// The same on the unit cube's Kuhn mesh (nc^3 coarse interior nodes): the fine node (i, j, k)
// (1-based) takes the average of the coarse values at (i >> 1, j >> 1, k >> 1) and
// (i >> 1 + i mod 2, ...), the end points of the coarse edge (axis, face diagonal or body
// diagonal) whose midpoint it is; the same node at even-even-even nodes.
template <typename T>
__device__ __forceinline__ T prolong_value3(const T* __restrict__ cs, int nc, int i, int j, int k) {
  const int I0 = i >> 1, J0 = j >> 1, L0 = k >> 1;
  const int I1 = I0 + (i & 1), J1 = J0 + (j & 1), L1 = L0 + (k & 1);
  const int64_t nn = (int64_t)nc * nc;
  const T a = (I0 >= 1 && I0 <= nc && J0 >= 1 && J0 <= nc && L0 >= 1 && L0 <= nc)
                  ? cs[(L0 - 1) * nn + (int64_t)(J0 - 1) * nc + (I0 - 1)]
                  : T(0);
  const T c = (I1 >= 1 && I1 <= nc && J1 >= 1 && J1 <= nc && L1 >= 1 && L1 <= nc)
                  ? cs[(L1 - 1) * nn + (int64_t)(J1 - 1) * nc + (I1 - 1)]
                  : T(0);
  return T(0.5) * (a + c);
}

// Coefficient class of multigrid slice `slice` for a coef_class argument: a class >= 0 applies to
// every slice (0: K_x, 1 + l: K_l); a negative value -1 - r0 selects, per slice, K_l for the level
// l of wavelet row (r0 + slice) mod N_t (slices are the wavelet rows of B problems stored back to
// back, or rows r0, r0 + 1, ... of one problem for a rank that owns those rows).
__host__ __device__ inline int wavelet_row_level(int i, int J);
__host__ __device__ inline int slice_class(int coef_class, int slice, int J) {
  if (coef_class >= 0) return coef_class;
  return 1 + wavelet_row_level((slice + (-1 - coef_class)) % ((1 << J) + 1), J);
}

// Level |lambda| of in-place wavelet row i (rows 0 and 2^J: level 0; else J - ctz(i)).
__host__ __device__ inline int wavelet_row_level(int i, int J) {
  if (i == 0 || i == (1 << J)) return 0;
#ifdef __CUDA_ARCH__
  return J - (__ffs(i) - 1);
#else
  return J - __builtin_ctz((unsigned)i);
#endif
}

// Domain mask.  On the L-shape (0,1)^2 minus [1/2,1)^2 the grid nodes with x >= 1/2 and y >= 1/2
// are outside the domain or on its boundary; the library stores the full (2^k - 1)^2 grid and
// keeps those nodes at zero.  With q = (n - 1) / 2 (the node x = 1/2 has interior index q) a
// node (ix, iy) of a level with n points per side is outside iff ix >= q and iy >= q.
__host__ __device__ inline bool outside_domain(int ix, int iy, int n, int lshape) {
  const int q = (n - 1) >> 1;
  return lshape && ix >= q && iy >= q;
}

// Per-problem state of a device-driven PCG loop (device arrays of B entries, plus counters):
// ctr[0] the PCG or outer refinement step, ctr[1] whether an inner refinement solve made
// progress, ctr[2] the inner step; iterations, refinement steps, status, K_X-norm rho_0 and
// relative residual per problem; oact (refinement: still in the outer loop) and its (inner
// iterations of the current outer step).
struct DevState {
  int* ctr;
  int* iters;
  int* outer;
  int* status;
  int* oact;
  int* its;
  double* relres;
  double* rho0;
};
enum { LOOP_INIT = 0, LOOP_ITER = 1 };

// the coefficients of multigrid slice `slice` on level `level` (slice_class)
template <typename T>
__device__ __forceinline__ Coef<T> slice_coef(const Coef<T>* coef, int coef_class, int slice, int J, int K,
                                              int level) {
  return coef[slice_class(coef_class, slice, J) * (K + 1) + level];
}

constexpr int kWR = 96;  // Gauss-Seidel region width = 32 lanes x 3 columns

struct MGLevels {
  int K;                 // finest level
  int kmin;              // coarsest level (exact solve)
  int max_slices;        // capacity of the per-level buffers
  // per level k (index k), kmin <= k < K: the two iterate buffers, right-hand side
  double* xc[16];
  double* xc2[16];
  double* bc[16];
};

}  // namespace st

struct st_handle_s {
  int domain, K, J;
  int64_t Nt, Nx;
  int n;  // 2^K - 1
  st_config cfg;
  st::Phys phys;     // D and c of the reaction-diffusion form (from cfg)
  bool diag0;        // K_x's operator couples the (1,1) diagonal (d12 != 0 or c != 0)
  bool mg_df;        // ST_FP64_DF: the binary64 multigrid applications run in double-float
  cudaStream_t stream;
  int device;

  st::MGLevels mg;
  st::Coef<double>* coef;   // device, (J + 2) x (K + 1)
  st::Coef<float>* coef32;  // the same table rounded to binary32 (mixed precision)
  st::Coef<st::df64>* coefdf;  // the same table in double-float (ST_FP64_DF)

  // workspace, each N_t x N_x doubles unless noted
  double* U;       // single-scale state
  double* Y;       // 2 N_t slices: Y1 then Y2
  double* X;       // 2 N_t slices: K_x Y
  double* Xalt;    // 2 N_t slices: second iterate buffer of the finest multigrid level
  double* Bs;      // 2 N_t slices: the finest level's scaled right-hand side D^-1 b
  double* Z;       // single-scale S u
  double* V1;      // wavelet ping-pong scratch
  double* V2;
  double* r;       // PCG residual
  double* p;       // search direction
  double* z;       // preconditioned residual
  double* q;       // S_hat p
  double* g;       // device copy of g (st_solve_host)
  double* fhat;    // right-hand side (st_solve_host)
  double* w;       // solution (st_solve_host)
  double* u0;      // N_x doubles (st_solve_host)
  float* xi;         // ST_MIXED_FP32 inner solve: correction, residual, direction,
  float* ri;         //   preconditioned residual, S_hat direction (binary32, N_t x N_x)
  float* pi;
  float* zi;
  float* qi;
  int last_iters, last_outer;
  double last_relres;
  int B;             // problems in the batch (vectors are B x N_t x N_x)
  // PCG starts from the content of w (r = f_hat - S_hat w) instead of w = 0 (nested iteration)
  bool use_guess;
  // handles of the coarser meshes (K - m, J - m), m = 1.., of st_nested_solve (created on first use)
  st_handle_s* nest[16];
  // Gauss-Seidel kernel per [element type: 0 binary64, 1 binary32, 2 double-float][mass
  // couplings][level]: 0 shared-memory tiles (default), 1 register wavefront, 2 register tiles
  // (st_autotune, st_set_smoother)
  unsigned char gs_kind[3][2][16];
  // rows per segment of the register wavefront, same indices (0: the compiled default)
  unsigned short gs_seg[3][2][16];
  // CUDA graphs of the PCG iteration bodies (0: binary64 PCG, 1: binary32 inner PCG,
  // 2: binary64 PCG with binary32 preconditioner), re-captured when `graph_key` changes
  cudaGraphExec_t graph_exec[3];
  int64_t graph_launches[3];
  const void* graph_key[3];
  // the whole PCG solve as one CUDA graph whose WHILE nodes repeat the iteration body while the
  // device-side stop tests keep them going (cfg.use_graphs = 2), re-instantiated when the key
  // (right-hand side, solution vector, initial-guess mode) changes
  cudaGraphExec_t loop_exec;
  const void* loop_key[3];
  st::DevState ds;
  void* ds_mem;      // device allocation behind ds
  int* act;          // device: 1 while problem b iterates (B ints)
  int* act_host;     // page-locked mirror
  int* info_iters;   // host, per problem: iterations, refinement steps, status
  int* info_outer;
  int* info_status;
  double* info_relres;
  double* partials;  // dot-product partial sums (B x kDotBlocks)
  double* scal;      // PCG scalars (device)
  double* scal_host; // page-locked mirror

  // profiling (st_profile_begin / st_profile_end): kernel launch count, and CUDA events around
  // every finest-level Gauss-Seidel sweep with that launch's algorithmic FP64 ops and bytes
  mutable int64_t launches;
  mutable bool prof_on;
  mutable int prof_cap, prof_n;
  mutable cudaEvent_t* prof_ev;
  // per event pair: 0 / 1 sweep of 8-byte values (binary64, double-float) without / with mass
  // couplings, 2 / 3 the same for binary32 arithmetic (binary32 or bfloat16 storage)
  mutable unsigned char* prof_cat;
  mutable double prof_ops[4], prof_bytes[4];
};

namespace st {

// the handle's multigrid coefficient table in compute type T
template <typename T>
inline const Coef<T>* coef_table(const st_handle_s* h);
template <>
inline const Coef<double>* coef_table<double>(const st_handle_s* h) {
  return h->coef;
}
template <>
inline const Coef<float>* coef_table<float>(const st_handle_s* h) {
  return h->coef32;
}
template <>
inline const Coef<df64>* coef_table<df64>(const st_handle_s* h) {
  return h->coefdf;
}

// Gauss-Seidel sweeps in register tiles (k_gs_reg.cu): nsw = NSW consecutive sweeps of one colour
// order from x_in (+ P xc if xc != nullptr) into x_out, block shape `shape` (0: 12 rows x 8 warps
// in binary32, 6 rows x 8 warps in binary64 and double-float; binary32 only: 1: 8 rows x 12
// warps; 2: 6 rows x 16 warps; 3: the wide regions of k_gs_wide.cuh, 12 rows x 8 warps, on the
// levels where they fit, else shape 0; binary64 and double-float have shape 0 only)
template <typename T, typename G, int NSW, bool DIAG, bool PROL>
cudaError_t reg_launch(const st_handle_s* h, int shape, int k, int nslices, int cls, G* x_out, const G* x_in,
                       const G* b, const G* xc, bool reverse, bool zero_init);
constexpr int kRegShapes = 4;
// Binary32 Gauss-Seidel sweeps in wide register regions (k_gs_wide.cuh): 192 columns x 96 rows
// of whole warps where n = 2^k - 1 >= 192, else 96 x 96 of half-warps, two points of one colour
// per lane and row in packed binary32 arithmetic, regions clamped into the grid.  wide_fits: the
// unit square and a level with n >= 96 (`shape` is 0; the region shape follows from the level).
bool wide_fits(const st_handle_s* h, int shape, int k);
template <typename G, int NSW, bool DIAG, bool PROL>
cudaError_t wide_launch(const st_handle_s* h, int shape, int k, int nslices, int cls, G* x_out, const G* x_in,
                        const G* b, const G* xc, bool reverse, bool zero_init);
// the same for the last pre-smoothing launch of a V-cycle, which also forms the residual of the
// smoothed iterate and restricts it: bc receives the next coarser level's scaled right-hand side
// (what k_residual_restrict would write)
template <typename G, int NSW, bool DIAG>
cudaError_t wide_launch_restrict(const st_handle_s* h, int shape, int k, int nslices, int cls, G* x_out,
                                 const G* x_in, const G* b, G* bc, bool zero_init);
// the finest level's first pre-smoothing launch when it is also the last one (three sweeps from
// x = 0, binary32 storage): forms b' = b / c from the input b (written to bsc, what k_scale_rhs
// would write), smooths, and restricts the residual to bc
template <bool DIAG>
cudaError_t wide_launch_scale_restrict(const st_handle_s* h, int k, int nslices, int cls, float* x_out,
                                       const float* braw, float* bsc, float* bc);
// dynamic shared-memory limits of the wide kernels (once per device)
cudaError_t wide_set_attributes();

// launch accounting: every kernel launch site calls count_launch
inline void count_launch(const st_handle_s* h, int n = 1) { h->launches += n; }
// event pair around one profiled launch (no-op unless profiling); returns false if out of events
bool prof_start(const st_handle_s* h);
void prof_stop(const st_handle_s* h, int cat, double ops, double bytes);

// error helpers (thread-local message)
void set_error(const std::string& msg);
st_status cuda_fail(const char* where, cudaError_t e);

// ---------------------------------------------------------------------------------------
// launchers (all enqueue on `s`; return cudaGetLastError())
// ---------------------------------------------------------------------------------------
cudaError_t launch_make_coef(Coef<double>* coef, int K, int J, double alpha, Phys ph, int dim, cudaStream_t s);
cudaError_t launch_make_coef32(Coef<float>* coef, int K, int J, double alpha, Phys ph, int dim, cudaStream_t s);
cudaError_t launch_make_coef_df(Coef<df64>* coef, int K, int J, double alpha, Phys ph, int dim, cudaStream_t s);

// The operator launchers below are instantiated for T = double and T = float; the float
// versions reuse the handle's double workspace (half of each buffer).

// x = K b on nslices slices of the finest level: n_vcycles V-cycles from zero.
// coef_class < 0: per-slice class 1 + level(slice) (K_X); else a fixed class.
template <typename T>
cudaError_t mg_apply(const st_handle_s* h, int nslices, int coef_class, const T* b, T* x);
// the unit cube's multigrid (domain 2), and the same in double-float with binary64 in and out
template <typename T>
cudaError_t mg_apply3(const st_handle_s* h, int nslices, int coef_class, const T* b, T* x);
cudaError_t mg_apply3_df(const st_handle_s* h, int nslices, int coef_class, const double* b, double* x);
// the same in binary32 arithmetic with the multigrid's vectors stored as bfloat16
cudaError_t mg_apply_bf16(const st_handle_s* h, int nslices, int coef_class, const float* b, float* x);
// times the Gauss-Seidel kernels per level and records the fastest in h->gs_kind; table[12 k + i]
// receives the times (ms) of (binary64 K_x: shared-memory tiles, wavefront, register tiles;
// binary64 K_l: the same three; binary32 K_x; binary32 K_l)
cudaError_t mg_autotune(st_handle_s* h, float* table);

// The time-coupled launchers act on nb problems stored back to back (N_t x N_x each).
// wavelet transforms over N_t x N_x
template <typename T>
cudaError_t wavelet_synth(const st_handle_s* h, int nb, const T* w, T* u);
template <typename T>
cudaError_t wavelet_anal(const st_handle_s* h, int nb, const T* u, T* w);

// Y1, Y2 (Y = [Y1 of all nb problems; Y2 of all nb problems]) from U:
// mode 0 (S): Y1 = A_t U M + L^T U A, Y2 = L U M + M_t U A;
// mode 1 (right-hand side): Y1 = L^T G M, Y2 = M_t G M.
template <typename T>
cudaError_t launch_timemix(const st_handle_s* h, int nb, int mode, const T* U, T* Y);
// Z = M X1 + A X2 + e_0 (x) M row0 per problem (row0 of problem b at row0 + b row0_stride,
// N_x values added to its row 0)
template <typename T>
cudaError_t launch_epilogue(const st_handle_s* h, int nb, const T* X, const T* row0, int64_t row0_stride, T* Z);
// Y = A_x X on nrows slices
template <typename T>
cudaError_t launch_apply_A(const st_handle_s* h, int nrows, const T* X, T* Y);

// vector kernels (dot products accumulate in binary64).  launch_dot, launch_update_wr and
// launch_update_p act on problems b0 .. b0 + nb - 1 (the vectors passed start at problem b0)
// of n elements each, with per-problem scalars h->scal[b * SC_COUNT + slot] and the
// per-problem active flags h->act[b].
template <typename Ta, typename Tb>
cudaError_t launch_dot(const st_handle_s* h, int b0, int nb, const Ta* a, const Tb* b, int64_t n, int slot, int op);
template <typename T>
cudaError_t launch_update_wr(const st_handle_s* h, int b0, int nb, T* w, T* r, const T* p, const T* q, int64_t n);
template <typename T>
cudaError_t launch_update_p(const st_handle_s* h, int b0, int nb, T* p, const T* z, int64_t n);
template <typename Td, typename Ts>
cudaError_t launch_copy(const st_handle_s* h, Td* dst, const Ts* src, int64_t n);
template <typename T>
cudaError_t launch_zero(const st_handle_s* h, T* dst, int64_t n);
cudaError_t launch_add_correction(const st_handle_s* h, double* w, const float* d, int64_t n);
// y = alpha x + beta y
cudaError_t launch_axpby(const st_handle_s* h, double* y, const double* x, double alpha, double beta, int64_t n);
// time-sharded row blocks and column blocks (k_space_time.cu)
cudaError_t launch_timemix_rows(const st_handle_s* h, int mode, int row0, int nrows, const double* U, double* Y);
cudaError_t launch_epilogue_rows(const st_handle_s* h, int row0, int nrows, const double* X, const double* u_row0,
                                 double* Z);
cudaError_t wavelet_cols(const st_handle_s* h, int synth, int64_t ncols, const double* in, double* out);
// r = f - q, and rs = (float) r unless rs is null
cudaError_t launch_residual_split(const st_handle_s* h, double* r, float* rs, const double* f, const double* q,
                                  int64_t n);
// device-side stop tests of the graph-driven PCG loops (k_vec.cu); each sets the condition hc
cudaError_t launch_loop_test(const st_handle_s* h, int mode, int slot, bool check_pq, bool refine,
                             cudaGraphConditionalHandle hc);
cudaError_t launch_inner_test(const st_handle_s* h, int mode, cudaGraphConditionalHandle hc);
cudaError_t launch_refine_count(const st_handle_s* h);

// whole-handle pipelines (api.cu): right-hand side of nb problems, and the PCG solve of all
// problems of the handle in its configured precision
st_status rhs_impl(st_handle_s* h, int nb, const double* g, const double* u0, double* fhat);
st_status pcg_impl(st_handle_s* h, const double* fhat, double* w, int* iters, double* relres);
// the device-driven solve of a handle captured into graph G after the nodes `deps` (pre: work
// enqueued on the handle's stream before the PCG, post: after it; either may be null); `leaves`
// receives the last nodes.  After the graph has run, solve_collect reads the per-problem results.
st_status capture_solve(st_handle_s* h, cudaGraph_t G, const std::vector<cudaGraphNode_t>& deps,
                        const double* fhat, double* w, st_status (*pre)(st_handle_s*, void*),
                        st_status (*post)(st_handle_s*, void*), void* arg, std::vector<cudaGraphNode_t>* leaves);
st_status solve_collect_enqueue(st_handle_s* h, cudaStream_t s);
st_status solve_collect_finish(st_handle_s* h);
// continuous batching on a handle's slots (ST_FP64 or ST_MIXED_PRECOND): see api.cu
st_status slot_start(st_handle_s* h, int b);
st_status step_enqueue(st_handle_s* h, int nb);
st_status slot_result(st_handle_s* h, int b, double* u_host);
st_status push_active(st_handle_s* h);

// PCG scalar slots in h->scal
enum {
  SC_RHO = 0,
  SC_PQ = 1,
  SC_ALPHA = 2,
  SC_RHO_NEW = 3,
  SC_BETA = 4,
  SC_RHO0 = 5,
  SC_OUTER = 6,
  SC_RZOLD = 7,
  SC_COUNT = 8
};
// dot "op" after reduction into `slot`
enum { DOT_STORE = 0, DOT_ALPHA = 1, DOT_BETA = 2, DOT_INIT = 3, DOT_BETA_FLEX = 4 };

constexpr int kDotBlocks = 1216;  // 8 blocks x 152 SMs; fixed for deterministic reductions
constexpr int kThreads = 256;

}  // namespace st
