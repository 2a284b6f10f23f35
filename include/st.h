/*
 * libst: space-time Schur-complement PCG for the heat equation on one GB300 (sm_103a).
 *
 * Method: R. van Venetie and J. Westerdiep, "A parallel algorithm for solving linear
 * parabolic evolution equations", arXiv 2009.08875.  The library computes the paper's
 * hot path: PCG on  S_hat w = f_hat  (Sec. 3.4), S_hat = W^T S W, with S in the form of
 * Lemma 4.2 and the wavelet-in-time, multigrid-in-space preconditioner K_X (Thm. 3.1),
 * for u' - Laplace(u) = g (Sec. 5), or u' - div(D grad u) + c u = g (Sec. 4), on uniformly
 * refined P1 meshes of the unit square, an L-shape and the unit cube, P1 in time, three-point
 * wavelets in time; with reduced-precision variants, nested iteration, batches of problems, a
 * solve server and the building blocks of a solve whose time axis is split over processes.
 *
 * ---------------------------------------------------------------------------------------
 * Conventions shared by every entry point
 * ---------------------------------------------------------------------------------------
 * Sizes.  Space level K >= 1: N_x = (2^K - 1)^2 interior nodes (Sec. 5.1; (2^K - 1)^3 on the
 *   cube).  Time level J >= 1: N_t = 2^J + 1 time nodes.
 * Domains.  0: the unit square (Sec. 5.1).  1: the L-shape (0,1)^2 minus [1/2,1)^2 (not in the
 *   paper), K >= 2; it is stored on the same (2^K - 1)^2 grid, and the grid nodes with
 *   x >= 1/2 and y >= 1/2 (ix >= 2^(K-1) - 1 and iy >= 2^(K-1) - 1) are outside it: inputs must
 *   hold zeros there and outputs hold zeros there.  2: the unit cube (Sec. 5.2), see st_setup.
 * Layout.  A space-time vector is a dense row-major array of N_t x N_x doubles (time
 *   slowest).  Column p = iy * (2^K - 1) + ix is interior grid node (ix + 1, iy + 1) at
 *   (x, y) = ((ix+1) h, (iy+1) h), h = 2^-K.
 *   - single-scale vectors (u, g, f): row i is time node t_i = i 2^-J;
 *   - wavelet vectors (w, f_hat, r, z, q): "in-place" lifting order: rows 0 and 2^J hold
 *     the level-0 coefficients c_0, row i = (2k + 1) 2^(J-j-1) holds d_j[k] (level j + 1).
 *     The paper lists the same coefficients as (c_0, d_0, ..., d_{J-1}) (Sec. 3.3).
 * Batches.  A handle made by st_setup_batch holds B problems of the same domain, K and J; every
 *   vector then holds B problems back to back (B x N_t x N_x, u0: B x N_x), every operator acts
 *   on all of them, and each problem has its own PCG scalars and stop test.  A problem gives the
 *   same bits alone and inside a batch.  st_setup is st_setup_batch with B = 1.
 * Memory.  Unless a name ends in _host, every vector pointer is a CUDA device pointer to
 *   caller-owned memory, 8-byte aligned, not aliased with any other argument of the
 *   same call.  The handle owns its internal workspace (allocated by st_setup).
 * Streams.  All work is enqueued on the stream given to st_setup, in order, and is
 *   asynchronous unless stated otherwise.
 * Errors.  Every function returns an st_status; nothing is thrown across the ABI.  On
 *   failure st_last_error() returns a message for the calling thread.  Argument errors
 *   are detected before any work is enqueued.
 */
#ifndef ST_H
#define ST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct st_handle_s* st_handle;

typedef enum {
  ST_OK = 0,
  ST_ERR_ARG = 1,        /* invalid argument (null handle/pointer, size out of range)   */
  ST_ERR_NOMEM = 2,      /* device workspace allocation failed                          */
  ST_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed                 */
  ST_ERR_BREAKDOWN = 4,  /* PCG breakdown: p^T S_hat p <= 0 or a non-finite scalar      */
  ST_ERR_MAXIT = 5,      /* PCG stopped at maxit before reaching the tolerance          */
  ST_ERR_TIMEOUT = 6,    /* a served request passed its deadline before it finished      */
  ST_ERR_CANCELLED = 7   /* a served request was cancelled (st_server_cancel)            */
} st_status;

typedef enum {
  ST_FP64 = 0,           /* every operation in IEEE binary64                              */
  ST_MIXED_FP32 = 1,     /* binary64 iterative refinement around a binary32 inner PCG:
                            the outer residual f_hat - S_hat w uses the binary64 S (with
                            its binary64 K_x), corrections and sums are binary64; the inner
                            solve runs S_hat and K_X in binary32 with binary64 inner products */
  ST_MIXED_PRECOND = 2,  /* one binary64 PCG (binary64 S_hat, recurrences and inner products)
                            preconditioned by K_X in binary32, with the flexible (Polak-Ribiere)
                            beta = r^T (z - z_old) / rho_old */
  ST_MIXED_BF16 = 3,     /* as ST_MIXED_FP32, but the inner PCG's preconditioner K_X keeps its
                            multigrid vectors (iterates, right-hand sides, coarse levels) in
                            bfloat16 storage with binary32 arithmetic, and the inner PCG uses
                            the flexible beta; the inner S_hat and the outer stopping test
                            stay binary32 / binary64 as in ST_MIXED_FP32 */
  ST_FP64_DF = 4         /* as ST_FP64, but every multigrid application (K_x in S and in the
                            right-hand side, K_l in K_X) computes in double-float: pairs of
                            binary32 values with error-free transformations, about 48
                            significant bits (binary64: 53); inputs and outputs stay binary64. */
} st_precision;

typedef struct {
  double alpha;     /* scaling of A_x inside K_j = (alpha A_x + 2^j M_x)^-1, Sec. 5.1: 0.3 */
  int n_vcycles;    /* V-cycles per multigrid application, from x = 0; Sec. 5.1: 2          */
  int n_pre;        /* 3-colour Gauss-Seidel pre-sweeps per level; Sec. 5.1: 3              */
  int n_post;       /* post-sweeps per level (reverse colour order); Sec. 5.1: 3            */
  double tol;       /* PCG tolerance                                                        */
  int tol_mode;     /* 0: stop when sqrt(r^T K_X r / r_0^T K_X r_0) <= tol;
                       1: stop when sqrt(r^T K_X r) <= tol (Eq. 3.3, the paper's rule)      */
  int maxit;        /* PCG iteration limit                                                  */
  int precision;    /* st_precision                                                         */
  double inner_tol; /* ST_MIXED_FP32 / _BF16: relative K_X-norm reduction of each inner solve */
  int inner_maxit;  /* ST_MIXED_FP32 / _BF16: iteration limit of each inner solve            */
  int use_graphs;   /* 2 (default): the whole PCG solve is one CUDA graph whose WHILE node
                       repeats the iteration body while device-side stop tests (the same
                       decisions as the host's, bitwise the same results) keep it going, so
                       a solve makes no host round trip per iteration; st_batch_run runs all
                       shape groups as branches of one such graph.  1: the host tests after
                       every iteration, each iteration body captured once as a CUDA graph and
                       replayed.  0: plain launches.  Graphs are used only on a stream other
                       than the legacy/per-thread default streams and outside
                       st_profile_begin/end (plain launches there).                        */
  double diffusion[3]; /* D = [[d11, d12], [d12, d22]] as (d11, d12, d22) and             */
  double reaction;     /* c of the reaction-diffusion form of Sec. 4,
                          a(eta, zeta) = <D grad eta, grad zeta> + c <eta, zeta>, which
                          defines A_x (Lemma 4.1) in S, f and every K.  D must be symmetric
                          positive definite and c >= 0 (else ST_ERR_ARG); D = Id, c = 0 is
                          the heat equation.  st_apply_Kx_static always uses the heat
                          equation's A_x.                                                 */
  int initial_guess;   /* 1: st_pcg_solve starts from the content of w (r = f_hat - S_hat w);
                          0 (default): from w = 0 as in Sec. 3.4                          */
} st_config;

/* Fills *cfg with the paper's settings (alpha 0.3, 2 V-cycles, 3+3 sweeps, Sec. 5.1),
 * tol 1e-10 relative, maxit 200, FP64; inner_tol 1e-5, inner_maxit 60, use_graphs 2;
 * D = Id, c = 0 (the heat equation of Sec. 5); initial_guess 0. */
void st_default_config(st_config* cfg);

/* Creates a handle for `domain` at space level K and time level J (1..14), binds it to
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream) and allocates its device
 * workspace (about 26 vectors of N_t x N_x doubles) on the current device.  Domains:
 *   0  unit square, K in 1..12, N_x = (2^K - 1)^2 (Sec. 5.1);
 *   1  L-shape (0,1)^2 minus [1/2,1)^2 stored on the square's grid with zeros outside,
 *      K in 2..12;
 *   2  unit cube, K in 1..8, N_x = (2^K - 1)^3, P1 on the six Kuhn tetrahedra of every grid
 *      cube (the 3D problem of Sec. 5.2); D = Id only, c >= 0; not ST_MIXED_BF16;
 *      the column index is (iz (2^K - 1) + iy) (2^K - 1) + ix.
 * The multigrid's coarsest level is 1 (one unknown) on the square and the cube and 2 (five
 * unknowns, dense solve) on the L-shape.  cfg may be NULL (defaults).  Synchronous. */
st_status st_setup(st_handle* out, int domain, int space_level, int time_level,
                   const st_config* cfg, void* cuda_stream);

/* As st_setup for a batch of B independent problems (B >= 1, 2 B N_t <= 65535). */
st_status st_setup_batch(st_handle* out, int domain, int space_level, int time_level, int batch,
                         const st_config* cfg, void* cuda_stream);

/* Reports the batch size B of the handle. */
st_status st_batch_size(st_handle h, int* B);

/* Frees the workspace (after synchronising the bound stream).  NULL is accepted. */
st_status st_destroy(st_handle h);

/* Reports N_t and N_x of the handle. */
st_status st_dims(st_handle h, int64_t* Nt, int64_t* Nx);

/* x[s] = K_x b[s] for slices s < nslices (nslices <= 2 B N_t), each of N_x doubles:
 * K_x ~ A_x^-1 is n_vcycles symmetric V-cycles from zero on A_x (Sec. 3.1, Sec. 5.1).
 * b and x must not overlap. */
st_status st_apply_Kx(st_handle h, int nslices, const double* b, double* x);

/* y = S u in single-scale coordinates, S by Lemma 4.2:
 * S = A_t (x) M K_x M + M_t (x) A K_x A + L^T (x) M K_x A + L (x) A K_x M + Gamma_0 (x) M. */
st_status st_apply_S_nodal(st_handle h, const double* u, double* y);

/* u = W w: the wavelet synthesis W = W_t (x) Id, W_t by Eq. (3.1).  w in wavelet order. */
st_status st_synthesize(st_handle h, const double* w, double* u);

/* w = W^T u: the transposed (analysis) transform.  w in wavelet order. */
st_status st_analyze(st_handle h, const double* u, double* w);

/* q = S_hat w = W^T S W w (Sec. 3.4).  w and q in wavelet order. */
st_status st_apply_S(st_handle h, const double* w, double* q);

/* z = K_X r = blockdiag[K_|l| A_x K_|l|] r (Thm. 3.1), K_l ~ (alpha A_x + 2^l M_x)^-1 by
 * multigrid, |l| the level of each wavelet row.  r and z in wavelet order. */
st_status st_apply_KX(st_handle h, const double* r, double* z);

/* f_hat = W^T f with f = B^T K_Y g + u_0 (Lemma 4.1), g interpolated in P1 (x) P1 at the
 * space-time nodes (g_nodal: N_t x N_x single-scale) and u_0 in P1 (u0_nodal: N_x). */
st_status st_rhs(st_handle h, const double* g_nodal, const double* u0_nodal, double* fhat);

/* PCG on S_hat w = f_hat with preconditioner K_X (Sec. 3.4), starting from w = 0 (the
 * input content of w is ignored and overwritten) or, with cfg.initial_guess = 1, from the
 * content of w.  Stops by cfg.tol / cfg.tol_mode.
 * Synchronises the bound stream once at the end with cfg.use_graphs = 2, else once per
 * iteration (8 scalars per problem read back).
 * *iters receives the iteration count; *relres sqrt(r^T K_X r / r_0^T K_X r_0).
 * With cfg.precision = ST_MIXED_FP32 (or ST_MIXED_BF16) the solve is iterative refinement: each outer step
 * solves S_hat d = r with binary32 PCG to cfg.inner_tol, adds d to w in binary64 and
 * recomputes r = f_hat - S_hat w in binary64; it stops when the binary64 residual meets
 * cfg.tol in the K_X norm (K_X applied in binary32).  *iters is then the total number of
 * inner PCG iterations (outer steps: st_solve_info).
 * Returns ST_ERR_MAXIT (w holds the last iterate) or ST_ERR_BREAKDOWN on failure. */
st_status st_pcg_solve(st_handle h, const double* fhat, double* w, int* iters, double* relres);

/* Statistics of the last st_pcg_solve / st_solve_host on the handle (maxima over the batch). */
typedef struct {
  int iterations;        /* PCG iterations (binary32 inner iterations for ST_MIXED_FP32) */
  int outer_iterations;  /* refinement steps (binary64 S_hat applications); 0 otherwise   */
  double relres;         /* final sqrt(r^T K_X r / r_0^T K_X r_0)                        */
} st_solve_info;
st_status st_solve_info_get(st_handle h, st_solve_info* out);

/* The same for problem b of the batch; *status (may be NULL) receives its st_status. */
st_status st_problem_info(st_handle h, int b, st_solve_info* out, int* status);

/* The binary32 operators of the ST_MIXED_FP32 inner solve (same definitions as st_apply_S and
 * st_apply_KX; float device vectors of N_t x N_x in wavelet order).  Valid on any handle. */
st_status st_apply_S_f32(st_handle h, const float* w, float* q);
st_status st_apply_KX_f32(st_handle h, const float* r, float* z);

/* K_X of the ST_MIXED_BF16 inner solve: binary32 arithmetic with every multigrid vector stored
 * as bfloat16 (r and z are float device vectors of N_t x N_x in wavelet order).  Not in the
 * paper.  Valid on any handle. */
st_status st_apply_KX_bf16(st_handle h, const float* r, float* z);

/* End-to-end solve from host memory: copies g_nodal_host (B x N_t x N_x) and u0_host (B x N_x)
 * to the device, forms f_hat, runs PCG, synthesises u = W w and copies u to u_host
 * (B x N_t x N_x).  Host buffers should be page-locked for full copy bandwidth.
 * Synchronous.  Returns like st_pcg_solve. */
st_status st_solve_host(st_handle h, const double* g_nodal_host, const double* u0_host,
                        double* u_host, int* iters, double* relres);

/* Allocation-free variant of st_apply_Kx (the paper has no counterpart; it exists for callers
 * that cannot allocate device memory: processes whose device memory budget is owned by another
 * allocator, such as a framework's caching allocator or a serving runtime's arena, where a raw
 * cudaMalloc can fail or fragment that pool, and latency-critical loops that forbid allocation
 * after start-up because cudaMalloc/cudaFree may synchronise the device).
 * Computes x[s] = K_x b[s] for s < nslices at space level K, bitwise the same as st_apply_Kx
 * with the default multigrid settings (2 V-cycles, 3 + 3 sweeps), enqueued on cuda_stream.
 * Needs no handle and allocates nothing: its scratch is one static device array of 32 MiB,
 * held by every device that loads the library until the process exits.  Sizes whose scratch
 * (about nslices * N_x * 3 doubles) exceeds 32 MiB, and nslices above 65535 (a launch grid
 * dimension), are rejected with ST_ERR_ARG before any work is enqueued; for example K = 9
 * allows 5 slices, K = 7 allows 87.
 * The first call on each device looks up the array's device address and sets kernel
 * attributes; make that first call before any stream capture on that device.  The address is
 * kept for the life of the process: calls after cudaDeviceReset on that device are not
 * supported (the reset reloads the module, and the kept address would be stale).
 * Every call on a device shares the one array, which keeps the last call's contents (nothing
 * in it needs to start at zero), so calls whose work overlaps on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  b and x are device pointers to
 * caller-owned memory of nslices * N_x doubles and must not overlap. */
st_status st_apply_Kx_static(int space_level, int nslices, const double* b, double* x, void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Batches of problems of any shape (not in the paper: a throughput interface for many
 * independent solves).  Problems registered with st_batch_add are grouped by (domain, K, J);
 * each group is solved as one batched handle on a stream of its own, and the groups run
 * concurrently.  Every problem's result is bitwise what st_setup + st_solve_host would give
 * for it alone with the same st_config.  Host buffers belong to the caller and must stay
 * valid until st_batch_run returns; page-locked buffers copy fastest.
 * --------------------------------------------------------------------------------------- */
typedef struct st_batch_s* st_batch;

/* Creates an empty batch solved with *cfg (NULL: defaults) on the current device. */
st_status st_batch_create(st_batch* out, const st_config* cfg);

/* Registers one problem (domain 0, 1 or 2 with the levels st_setup accepts): g_host (N_t x N_x),
 * u0_host (N_x), result u_host (N_t x N_x) in the layout of st_solve_host.  *id (may be NULL)
 * receives its index (0, 1, ...). */
st_status st_batch_add(st_batch b, int domain, int space_level, int time_level, const double* g_host,
                       const double* u0_host, double* u_host, int* id);

/* Solves every registered problem (synchronous).  Workspace is allocated per group for the
 * duration of the call.  Returns the first failing problem's status (ST_ERR_MAXIT or
 * ST_ERR_BREAKDOWN) after solving all of them, or ST_OK. */
st_status st_batch_run(st_batch b);

/* Statistics and status of problem id after st_batch_run. */
st_status st_batch_problem_info(st_batch b, int id, st_solve_info* out, int* status);

/* Number of groups (batched handles) the last st_batch_run used. */
st_status st_batch_buckets(st_batch b, int* n);

st_status st_batch_destroy(st_batch b);

/* ---------------------------------------------------------------------------------------
 * Continuous-batching server (not in the paper).  One worker thread serves queued solves:
 * problems of one shape share a group (a batched handle with a fixed number of slots, its CG
 * state resident on the GPU); each round it admits queued requests into free slots (creating
 * a group when the device-memory budget allows, releasing idle groups of other shapes to make
 * room), advances every group by one PCG iteration, and returns finished problems to their
 * callers.  Requests thus join and leave at iteration boundaries while others run, and each
 * result is computed exactly as if the problem were solved alone.  Precision: ST_FP64 or
 * ST_MIXED_PRECOND.  Host buffers must stay valid until the request is done.
 * --------------------------------------------------------------------------------------- */
typedef struct st_server_s* st_server;

/* Starts the worker on the current device.  slots_per_group: slots of a group (fewer for
 * large shapes: at most 2 slots N_t <= 65535 and a quarter of the budget per group);
 * memory_budget_gb: device memory the groups may hold in total. */
st_status st_server_start(st_server* out, const st_config* cfg, int slots_per_group, double memory_budget_gb);

/* Queues one solve (layout of st_solve_host; u_host receives u = W w).  *ticket identifies it. */
st_status st_server_submit(st_server s, int domain, int space_level, int time_level, const double* g_host,
                           const double* u0_host, double* u_host, int64_t* ticket);

/* The same with a deadline timeout_s seconds after submission (<= 0 or infinite: none).  A
 * request that has not finished by then fails with ST_ERR_TIMEOUT: before it starts, or at the
 * next iteration boundary while it runs (u_host is then not written). */
st_status st_server_submit_deadline(st_server s, int domain, int space_level, int time_level, const double* g_host,
                                    const double* u0_host, double* u_host, double timeout_s, int64_t* ticket);

/* Cancels a queued or running request: it fails with ST_ERR_CANCELLED before it starts or at the
 * next iteration boundary (u_host is not written).  No effect on a finished request. */
st_status st_server_cancel(st_server s, int64_t ticket);

/* State of a request: *state 0 queued, 1 running, 2 done, 3 failed; *status (may be NULL) its
 * st_status (ST_ERR_NOMEM: it cannot fit in the budget; ST_ERR_MAXIT, ST_ERR_BREAKDOWN,
 * ST_ERR_TIMEOUT, ST_ERR_CANCELLED); info->relres and iterations describe the solve.
 * *latency_s (may be NULL): seconds from submission to completion, or -1 if not finished. */
st_status st_server_poll(st_server s, int64_t ticket, int* state, int* status, st_solve_info* info,
                         double* latency_s);

/* Serves every submitted request, stops the worker and frees all device memory. */
st_status st_server_stop(st_server s);

/* Nested iteration (Sec. 4.4: with the algebraic error kept proportional to the discretisation
 * error, nested iteration after Hackbusch Ch. 5 makes the solve linear in N_t N_x; the paper
 * gives no procedure).  Solves on the meshes (K - m, J - m), m = levels-1 .. 0, of the handle's
 * domain with its st_config: level m's data are the fine nodal values g (B x N_t x N_x) and u0
 * (B x N_x) at that mesh's nodes (injection), its PCG starts from the previous level's solution
 * (coarse wavelet row i is fine row 2i, new details 0, rows prolongated by nested P1 in x) and
 * stops when sqrt(r^T K_X r) <= eps 2^(rate m) (Eq. 3.3, absolute; 2^rate is the expected ratio
 * of discretisation errors between consecutive levels).  w (B x N_t x N_x, wavelet order)
 * receives the finest solution; iters_per_level (levels ints, coarsest first; may be NULL) the
 * PCG iterations of each level.  The coarser handles are created on the first call and kept
 * with h (about 1/8, 1/64, ... of its memory).  Needs K - levels + 1 >= 1 (>= 2 on the L-shape)
 * and J - levels + 1 >= 1.  Synchronous.  Returns ST_ERR_MAXIT if some level stopped at maxit
 * (the finer levels still run), ST_ERR_BREAKDOWN or ST_ERR_CUDA on failure. */
st_status st_nested_solve(st_handle h, int levels, double eps, double rate, const double* g_nodal,
                          const double* u0_nodal, double* w, int* iters_per_level);

/* ---------------------------------------------------------------------------------------
 * Time-sharded building blocks.  The paper distributes the time axis over processes (Sec. 5.2).
 * A rank that owns the time rows [row0, row0 + nrows) of one problem (single-problem handle of the
 * full mesh, which supplies coefficient tables and scratch) applies the operators of a PCG
 * iteration to its rows; the wavelet transform acts along the whole time axis and is applied to a
 * block of columns after a rows-to-columns exchange; inner products are reduced by the caller.
 * The caller's vectors hold only its rows (N_x doubles each) or columns.  Errors: ST_ERR_ARG for
 * a batch handle, rows outside 0..N_t-1, null pointers.
 * --------------------------------------------------------------------------------------- */

/* Nodal rows of S (mode 0, Lemma 4.2: time mix, K_x, epilogue) or of the right-hand side before
 * the analysis (mode 1, Lemma 4.1: L^T G M and M_t G M, K_x, epilogue): y (nrows rows) from
 * u_halo, which holds rows row0 - 1 .. row0 + nrows (nrows + 2 rows; rows outside 0..N_t-1 are
 * not read).  u_row0: nodal row 0 of U (mode 0, Gamma_0 term) or u_0 (mode 1), used only when
 * row0 = 0. */
st_status st_rows_nodal(st_handle h, int mode, int64_t row0, int64_t nrows, const double* u_halo,
                        const double* u_row0, double* y);

/* z = K_X r on the wavelet rows row0 .. row0 + nrows - 1 (in-place row order; K_l of each row's
 * level, Thm. 3.1). */
st_status st_rows_KX(st_handle h, int64_t row0, int64_t nrows, const double* r, double* z);

/* Wavelet synthesis (synthesize != 0, u = W w) or analysis (w = W^T u) of an N_t x ncols block
 * of columns (row stride ncols, 1 <= ncols <= N_x; in-place wavelet row order). */
st_status st_wavelet_cols(st_handle h, int synthesize, int64_t ncols, const double* in, double* out);

/* *result = a^T b over n doubles (deterministic binary64 reduction; synchronous). */
st_status st_vec_dot(st_handle h, int64_t n, const double* a, const double* b, double* result);

/* y = alpha x + beta y over n doubles (asynchronous on the bound stream). */
st_status st_vec_axpby(st_handle h, int64_t n, double alpha, const double* x, double beta, double* y);

/* The whole time-sharded solve of one rank (Sec. 5.2's time distribution): right-hand side
 * (Lemma 4.1), PCG (Sec. 3.4, Eq. 3.3: scalars, stop test and updates all here) and synthesis
 * u = W w, on the rows [lo, hi) of rank `rank` of `nranks` (a power of two <= 2^J; m = 2^J /
 * nranks, lo = rank m, hi = lo + m, plus row 2^J on the last rank).  The communication goes
 * through the caller's st_comm: a neighbour row each side of the time mix, a rows <-> columns
 * exchange around each wavelet transform (rank s lifts the columns [s N_x / P, (s + 1) N_x / P)),
 * and a sum over the ranks of each inner product.  The rank's own kernels have finished whenever
 * a callback is called (no kernel waits on another rank).  g_rows, u_rows: device, (hi - lo) x N_x;
 * u0: device, N_x (read by the rank that owns row 0).  The handle (single problem, the full mesh)
 * supplies coefficient tables and scratch; the call allocates its row and column buffers for its
 * duration.  Stops by the handle's cfg.tol / tol_mode / maxit.  Synchronous.  Returns
 * ST_ERR_MAXIT, ST_ERR_BREAKDOWN, ST_ERR_ARG (bad partition), ST_ERR_CUDA, or ST_ERR_CANCELLED
 * when a callback reports failure. */
typedef struct {
  void* ctx;
  /* v[0 .. n) <- the sum over the ranks of v[0 .. n) (host memory); 0 on success */
  int (*allreduce_sum)(void* ctx, double* v, int n);
  /* for every rank s != own: send send_count[s] doubles from the device buffer send[s] to s and
   * receive recv_count[s] doubles from s into the device buffer recv[s] (count 0: nothing);
   * the sends and receives are complete when it returns; 0 on success */
  int (*exchange)(void* ctx, double* const* send, const int64_t* send_count, double* const* recv,
                  const int64_t* recv_count);
} st_comm;
st_status st_sharded_solve(st_handle h, const st_comm* comm, int rank, int nranks, const double* g_rows,
                           const double* u0, double* u_rows, int* iters, double* relres);

/* Autotuner (not in the paper).  Three Gauss-Seidel kernels compute identical sweeps:
 * shared-memory tiles (the default), a register wavefront, whose strips of 90 columns are cut into
 * row segments walked by separate warps, and register tiles, whose 96-column regions sit in the
 * registers of a block's warps (binary32: 12 rows x 8 warps, 8 x 12 or 6 x 16, the autotuner
 * trying each; binary64 and double-float: 6 rows x 8 warps).  Binary32 has one more register
 * block shape on the unit square: regions placed inside the grid, 192 columns x 96 rows of
 * whole warps on the levels with 2^k - 1 >= 192 and 96 x 96 of half-warps on those with
 * 2^k - 1 >= 96, whose lanes update two points of one colour with one paired binary32
 * instruction, and whose last pre-smoothing launch of a V-cycle also forms and restricts the
 * residual (on smaller levels it runs as the first shape).
 * For every multigrid level
 * above the coarsest, for binary64 and binary32 and for K_x (no mass couplings, 2 B N_t slices)
 * and K_l (mass couplings, B N_t slices), this times one pre-smoothing launch of each kernel (the
 * wavefront at ceil(n / q) rows per segment, q = 1 .. 12, n = 2^k - 1 on level k; the register
 * tiles in every block shape) on the handle's
 * workspace and keeps the fastest kernel and segment length for later calls on this handle.
 * Synchronous.
 * times_ms (may be NULL) receives 12 x 16 floats: times_ms[12 k + i] for level k and i = 0..11 in
 * the order (binary64 K_x: shared-memory tiles, wavefront, register tiles; binary64 K_l: the
 * same three; binary32 K_x: the same three; binary32 K_l: the same three), each the best over its
 * segment lengths or block shapes. */
st_status st_autotune(st_handle h, float* times_ms);

/* Forces one Gauss-Seidel kernel on every level of this handle: kind 0 shared-memory tiles (the
 * state after set-up, except binary32 on the unit square's levels with 2^k - 1 >= 96, which
 * start with kind 5), 1 register wavefront, 2, 3, 4 register tiles of block shape 0, 1, 2 (in
 * binary32 12 rows x 8 warps, 8 x 12, 6 x 16; binary64 and double-float always 6 x 8), 5 the
 * binary32 regions with paired arithmetic (unit square, levels with 2^k - 1 >= 96; shape 0
 * elsewhere and in binary64 and double-float).  All give bitwise the same sweeps and
 * coarse right-hand sides.  Returns ST_ERR_ARG for any other kind. */
st_status st_set_smoother(st_handle h, int kind);

/* Forces the register wavefront's rows per segment on every level of this handle (rows >= 1;
 * values above a level's n = 2^k - 1 mean one segment per strip; 0 restores the compiled
 * default of 64).  Any segment length gives bitwise the same sweeps.  Returns ST_ERR_ARG unless
 * 0 <= rows <= 65535. */
st_status st_set_wave_rows(st_handle h, int rows);

/* Measurement hooks (not part of the method).  Between st_profile_begin and st_profile_end the
 * handle counts every kernel it launches and brackets each finest-level Gauss-Seidel sweep
 * launch (the dominant kernel) with a pair of CUDA events on the bound stream, adding up the
 * launch's algorithmic work: per point and sweep 4 FP64 operations for K_x (2 adds, 2 fmas; 6
 * with the mass couplings of K_l: 1 more add and fma), and per point and launch 3 values moved
 * (read x and b, write x; 2 on a launch that starts from x = 0) of the storage type, plus the
 * coarse iterate read by a launch that adds the prolongated correction.  Launches computing in
 * binary64 or double-float and launches computing in binary32 (binary32 or bfloat16 storage)
 * are summed separately.  st_profile_end synchronises the stream and reports the sums, in total
 * and for the sweeps with mass couplings alone. */
typedef struct {
  int64_t launches;        /* kernels launched by the handle                        */
  int64_t sweep_launches;  /* finest-level binary64 Gauss-Seidel sweep launches     */
  double sweep_ms;         /* their summed CUDA-event durations                     */
  double sweep_fp64_ops;   /* their algorithmic FP64 operations (add, mul, fma = 1) */
  double sweep_bytes;      /* their algorithmic DRAM bytes                          */
  int64_t diag_launches;   /* the subset with mass couplings (K_l): launches        */
  double diag_ms;          /*   CUDA-event time                                     */
  double diag_fp64_ops;    /*   FP64 operations                                     */
  double diag_bytes;       /*   DRAM bytes                                          */
  int64_t f32_launches;    /* finest-level binary32 sweep launches                  */
  double f32_ms;           /*   CUDA-event time                                     */
  double f32_bytes;        /*   algorithmic DRAM bytes                              */
  int64_t f32_diag_launches; /* the binary32 subset with mass couplings (K_l)       */
  double f32_diag_ms;
  double f32_diag_bytes;
} st_profile;

st_status st_profile_begin(st_handle h);
st_status st_profile_end(st_handle h, st_profile* out);

/* Measurement hook (not part of the method): the device's sustained fused multiply-add rates,
 * from a throughput kernel of 4, 8 or 16 independent x <- x a + c chains per thread (the best
 * kept) and 8 blocks of 256 threads per SM, in binary64 (about 2.5e9 fmas a launch) and binary32
 * (32 times as many), each the best of 3 launches timed with CUDA events on cuda_stream after one
 * warm-up launch, on the current device.  *fp64_fma_per_s and *fp32_fma_per_s receive fmas per second (2 flops each).  Allocates
 * nothing (its results are folded into a file-scope device array).  Synchronous. */
st_status st_probe_fma_rates(void* cuda_stream, double* fp64_fma_per_s, double* fp32_fma_per_s);

/* Message describing the last failure on the calling thread ("" if none). */
const char* st_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ST_H */
