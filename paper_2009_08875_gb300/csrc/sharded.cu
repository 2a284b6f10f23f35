// st_sharded_solve: one rank's share of a solve whose time axis is split over ranks (the paper's
// time distribution, Sec. 5.2), with the whole PCG (scalars, stop test, updates) in this library
// and only the communication in the caller's st_comm callbacks.
//
// Rank r of P owns the time rows [lo, hi) (m = 2^J / P rows each, the last rank also row 2^J).
//  * nodal rows of S and of the right-hand side (Lemma 4.2, Lemma 4.1): the time matrices are
//    tridiagonal, so a rank needs one neighbour row each side (exchanged point to point);
//  * the wavelet transforms (Eq. 3.1) act along the whole time axis: the rows are exchanged into
//    blocks of columns (rank s owns the columns [s N_x / P, (s + 1) N_x / P)), each rank lifts its
//    columns over all N_t rows, and the result is exchanged back;
//  * K_X (Thm. 3.1) is block diagonal in the wavelet rows: no communication;
//  * inner products: a sum over the ranks of each rank's partial sum.
// Every callback is made after the rank's own kernels have finished, so no kernel ever waits on
// another rank.
#include <cmath>
#include <string>
#include <vector>

#include "st_internal.cuh"

using namespace st;

#define ST_CHECK_S(call)        \
  do {                          \
    st_status s_ = (call);      \
    if (s_ != ST_OK) return s_; \
  } while (0)

namespace {

struct Shard {
  st_handle h;
  const st_comm* comm;
  int rank, P;
  int64_t Nt, Nx;
  int64_t lo, hi, nrows;
  std::vector<int64_t> rlo, rhi, clo, chi;  // every rank's rows and columns
  int64_t ncols;                            // this rank's columns
  // device buffers (nrows x N_x unless noted)
  double *fhat = nullptr, *w = nullptr, *r = nullptr, *p = nullptr, *z = nullptr, *q = nullptr, *y = nullptr;
  double* halo = nullptr;  // (nrows + 2) x N_x
  double* colA = nullptr;  // N_t x ncols
  double* colB = nullptr;
  double* pack = nullptr;  // nrows x N_x: the pieces exchanged with the other ranks
  std::vector<void*> allocs;

  st_status alloc(double** ptr, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(double) * (count > 0 ? count : 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("st_sharded_solve: cudaMalloc failed: ") + cudaGetErrorString(e));
      return ST_ERR_NOMEM;
    }
    allocs.push_back(*ptr);
    return ST_OK;
  }
  ~Shard() {
    if (h) cudaStreamSynchronize(h->stream);
    for (void* a : allocs) cudaFree(a);
  }

  st_status sync() {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? ST_OK : cuda_fail("st_sharded_solve: stream synchronize", e);
  }
  st_status comm_fail(const char* what) {
    set_error(std::string("st_sharded_solve: the communicator's ") + what + " callback failed");
    return ST_ERR_CANCELLED;
  }

  // sum over the ranks
  st_status allreduce(double* v, int n) {
    if (comm->allreduce_sum(comm->ctx, v, n) != 0) return comm_fail("allreduce_sum");
    return ST_OK;
  }

  // this rank's rows (nrows x N_x) -> its columns over all N_t rows (N_t x ncols)
  st_status rows_to_cols(const double* X, double* C) {
    std::vector<double*> send(P, nullptr), recv(P, nullptr);
    std::vector<int64_t> ns(P, 0), nr(P, 0);
    int64_t at = 0;
    for (int s = 0; s < P; ++s) {
      const int64_t wc = chi[s] - clo[s];
      double* dst = (s == rank) ? C + lo * ncols : pack + at;
      cudaError_t e = cudaMemcpy2DAsync(dst, sizeof(double) * wc, X + clo[s], sizeof(double) * Nx, sizeof(double) * wc,
                                        nrows, cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) return cuda_fail("st_sharded_solve: pack columns", e);
      if (s != rank) {
        send[s] = dst;
        ns[s] = nrows * wc;
        at += nrows * wc;
        recv[s] = C + rlo[s] * ncols;  // rank s's rows of my columns, contiguous
        nr[s] = (rhi[s] - rlo[s]) * ncols;
      }
    }
    ST_CHECK_S(sync());
    if (P > 1 && comm->exchange(comm->ctx, send.data(), ns.data(), recv.data(), nr.data()) != 0)
      return comm_fail("exchange");
    return ST_OK;
  }

  // this rank's columns (N_t x ncols) -> its rows (nrows x N_x)
  st_status cols_to_rows(const double* C, double* X) {
    std::vector<double*> send(P, nullptr), recv(P, nullptr);
    std::vector<int64_t> ns(P, 0), nr(P, 0);
    int64_t at = 0;
    for (int s = 0; s < P; ++s) {
      if (s == rank) continue;
      send[s] = const_cast<double*>(C) + rlo[s] * ncols;
      ns[s] = (rhi[s] - rlo[s]) * ncols;
      recv[s] = pack + at;
      nr[s] = nrows * (chi[s] - clo[s]);
      at += nr[s];
    }
    // own block straight into place
    cudaError_t e = cudaMemcpy2DAsync(X + clo[rank], sizeof(double) * Nx, C + lo * ncols, sizeof(double) * ncols,
                                      sizeof(double) * ncols, nrows, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail("st_sharded_solve: own columns", e);
    ST_CHECK_S(sync());
    if (P > 1 && comm->exchange(comm->ctx, send.data(), ns.data(), recv.data(), nr.data()) != 0)
      return comm_fail("exchange");
    for (int s = 0; s < P; ++s) {
      if (s == rank) continue;
      const int64_t wc = chi[s] - clo[s];
      e = cudaMemcpy2DAsync(X + clo[s], sizeof(double) * Nx, recv[s], sizeof(double) * wc, sizeof(double) * wc, nrows,
                            cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) return cuda_fail("st_sharded_solve: unpack columns", e);
    }
    return ST_OK;
  }

  // halo = [row lo - 1; U; row hi] (zero rows beyond the time axis), from the neighbours
  st_status make_halo(const double* U) {
    cudaError_t e = cudaMemcpyAsync(halo + Nx, U, sizeof(double) * nrows * Nx, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(halo, 0, sizeof(double) * Nx, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(halo + (nrows + 1) * Nx, 0, sizeof(double) * Nx, h->stream);
    if (e != cudaSuccess) return cuda_fail("st_sharded_solve: halo", e);
    ST_CHECK_S(sync());
    std::vector<double*> send(P, nullptr), recv(P, nullptr);
    std::vector<int64_t> ns(P, 0), nr(P, 0);
    if (rank > 0) {
      send[rank - 1] = const_cast<double*>(U);  // my first row to the rank below
      ns[rank - 1] = Nx;
      recv[rank - 1] = halo;                    // its last row
      nr[rank - 1] = Nx;
    }
    if (rank < P - 1) {
      send[rank + 1] = const_cast<double*>(U) + (nrows - 1) * Nx;
      ns[rank + 1] = Nx;
      recv[rank + 1] = halo + (nrows + 1) * Nx;
      nr[rank + 1] = Nx;
    }
    if (P > 1 && comm->exchange(comm->ctx, send.data(), ns.data(), recv.data(), nr.data()) != 0)
      return comm_fail("exchange");
    return ST_OK;
  }

  // the operators on this rank's rows
  st_status synthesize(const double* Wr, double* Ur) {  // u = W w
    ST_CHECK_S(rows_to_cols(Wr, colA));
    cudaError_t e = wavelet_cols(h, 1, ncols, colA, colB);
    if (e != cudaSuccess) return cuda_fail("st_sharded_solve: wavelet synthesis", e);
    return cols_to_rows(colB, Ur);
  }
  st_status analyze(const double* Ur, double* Wr) {  // w = W^T u
    ST_CHECK_S(rows_to_cols(Ur, colA));
    cudaError_t e = wavelet_cols(h, 0, ncols, colA, colB);
    if (e != cudaSuccess) return cuda_fail("st_sharded_solve: wavelet analysis", e);
    return cols_to_rows(colB, Wr);
  }
  // nodal rows of S (mode 0) or of the right-hand side before the analysis (mode 1)
  st_status nodal(int mode, const double* Ur, const double* row0, double* Y) {
    ST_CHECK_S(make_halo(Ur));
    cudaError_t e = launch_timemix_rows(h, mode, (int)lo, (int)nrows, halo, h->Y);
    if (e == cudaSuccess) e = mg_apply<double>(h, (int)(2 * nrows), 0, h->Y, h->X);
    if (e == cudaSuccess) e = launch_epilogue_rows(h, (int)lo, (int)nrows, h->X, lo == 0 ? row0 : nullptr, Y);
    return e == cudaSuccess ? ST_OK : cuda_fail("st_sharded_solve: nodal rows", e);
  }
  st_status apply_Shat(const double* P_, double* Q) {
    ST_CHECK_S(synthesize(P_, Q));                       // Q holds u = W p for a moment
    ST_CHECK_S(nodal(0, Q, halo + Nx, y));               // row 0 of u: the halo's first own row
    return analyze(y, Q);
  }
  st_status apply_KX(const double* R, double* Z) {
    const int cls = (int)(-1 - lo);  // K_l of each wavelet row's level
    cudaError_t e = mg_apply<double>(h, (int)nrows, cls, R, h->X);
    if (e == cudaSuccess) e = launch_apply_A<double>(h, (int)nrows, h->X, h->Y);
    if (e == cudaSuccess) e = mg_apply<double>(h, (int)nrows, cls, h->Y, Z);
    return e == cudaSuccess ? ST_OK : cuda_fail("st_sharded_solve: K_X rows", e);
  }
  st_status dot(const double* a, const double* b, double* out) {
    cudaError_t e = launch_dot<double, double>(h, 0, 1, a, b, nrows * Nx, SC_OUTER, DOT_STORE);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, h->scal + SC_OUTER, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail("st_sharded_solve: inner product", e);
    ST_CHECK_S(sync());
    return allreduce(out, 1);
  }
  st_status axpby(double alpha, const double* x, double beta, double* yv) {
    cudaError_t e = launch_axpby(h, yv, x, alpha, beta, nrows * Nx);
    return e == cudaSuccess ? ST_OK : cuda_fail("st_sharded_solve: axpby", e);
  }

  // PCG on S_hat w = f_hat (Sec. 3.4), stopping as the single-handle solver (Eq. 3.3 with
  // cfg.tol_mode); the scalars are the sums over the ranks, so every rank takes the same steps
  st_status pcg(int* iters, double* relres) {
    const st_config& c = h->cfg;
    const int64_t n = nrows * Nx;
    cudaError_t e = cudaMemsetAsync(w, 0, sizeof(double) * n, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, fhat, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail("st_sharded_solve: initial residual", e);
    ST_CHECK_S(apply_KX(r, z));
    double rho = 0.0;
    ST_CHECK_S(dot(r, z, &rho));
    const double rho0 = rho;
    e = cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail("st_sharded_solve: p = z", e);
    *iters = 0;
    *relres = 0.0;
    if (!std::isfinite(rho0) || rho0 < 0.0) {
      set_error("st_sharded_solve: r_0^T K_X r_0 is negative or not finite");
      return ST_ERR_BREAKDOWN;
    }
    if (rho0 == 0.0 || (c.tol_mode == 1 && std::sqrt(rho0) <= c.tol)) return ST_OK;
    for (int it = 1; it <= c.maxit; ++it) {
      ST_CHECK_S(apply_Shat(p, q));
      double pq = 0.0;
      ST_CHECK_S(dot(p, q, &pq));
      if (!(pq > 0.0) || !std::isfinite(pq)) {
        set_error("st_sharded_solve: PCG breakdown, p^T S_hat p <= 0 or not finite");
        *iters = it;
        return ST_ERR_BREAKDOWN;
      }
      const double alpha = rho / pq;
      ST_CHECK_S(axpby(alpha, p, 1.0, w));
      ST_CHECK_S(axpby(-alpha, q, 1.0, r));
      ST_CHECK_S(apply_KX(r, z));
      double rho_new = 0.0;
      ST_CHECK_S(dot(r, z, &rho_new));
      *iters = it;
      if (!std::isfinite(rho_new) || rho_new < 0.0) {
        set_error("st_sharded_solve: PCG breakdown, r^T K_X r negative or not finite");
        return ST_ERR_BREAKDOWN;
      }
      *relres = std::sqrt(rho_new / rho0);
      if ((c.tol_mode == 1 && std::sqrt(rho_new) <= c.tol) || (c.tol_mode == 0 && *relres <= c.tol)) return ST_OK;
      ST_CHECK_S(axpby(1.0, z, rho_new / rho, p));
      rho = rho_new;
    }
    set_error("st_sharded_solve: PCG reached maxit before the tolerance");
    return ST_ERR_MAXIT;
  }
};

}  // namespace

extern "C" st_status st_sharded_solve(st_handle h, const st_comm* comm, int rank, int nranks, const double* g_rows,
                                      const double* u0, double* u_rows, int* iters, double* relres) {
  if (!h || !comm || !comm->allreduce_sum || !comm->exchange || !g_rows || !u0 || !u_rows || !iters || !relres) {
    set_error("st_sharded_solve: null argument");
    return ST_ERR_ARG;
  }
  if (h->B != 1 || nranks < 1 || (nranks & (nranks - 1)) || nranks > (1 << h->J) || rank < 0 || rank >= nranks ||
      nranks > h->Nx) {
    set_error("st_sharded_solve: needs a single-problem handle, a power-of-two number of ranks <= 2^J and <= N_x, "
              "and 0 <= rank < nranks");
    return ST_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
  Shard S;
  S.h = h;
  S.comm = comm;
  S.rank = rank;
  S.P = nranks;
  S.Nt = h->Nt;
  S.Nx = h->Nx;
  const int64_t m = ((int64_t)1 << h->J) / nranks;
  for (int s = 0; s < nranks; ++s) {
    S.rlo.push_back(s * m);
    S.rhi.push_back(s * m + m + (s == nranks - 1 ? 1 : 0));
    S.clo.push_back(s * S.Nx / nranks);
    S.chi.push_back((s + 1) * S.Nx / nranks);
  }
  S.lo = S.rlo[rank];
  S.hi = S.rhi[rank];
  S.nrows = S.hi - S.lo;
  S.ncols = S.chi[rank] - S.clo[rank];
  const size_t V = (size_t)(S.nrows * S.Nx);
  double** rows[] = {&S.fhat, &S.w, &S.r, &S.p, &S.z, &S.q, &S.y, &S.pack};
  for (double** b : rows) ST_CHECK_S(S.alloc(b, V));
  ST_CHECK_S(S.alloc(&S.halo, (size_t)(S.nrows + 2) * S.Nx));
  ST_CHECK_S(S.alloc(&S.colA, (size_t)(S.Nt * S.ncols)));
  ST_CHECK_S(S.alloc(&S.colB, (size_t)(S.Nt * S.ncols)));
  // f_hat = W^T (rows of Lemma 4.1's f), PCG, u = W w
  ST_CHECK_S(S.nodal(1, g_rows, u0, S.y));
  ST_CHECK_S(S.analyze(S.y, S.fhat));
  const st_status ps = S.pcg(iters, relres);
  if (ps != ST_OK && ps != ST_ERR_MAXIT) return ps;
  ST_CHECK_S(S.synthesize(S.w, u_rows));
  ST_CHECK_S(S.sync());
  return ps;
}
