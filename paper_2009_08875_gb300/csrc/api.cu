// C ABI of libst (declared in include/st.h): handle set-up, the operators of the Schur-complement
// PCG (Sec. 3.4, Lemma 4.2, Thm. 3.1, Eq. 3.1) and the host-side PCG driver.  Host code only
// validates arguments, sizes workspaces and enqueues kernels; all arithmetic runs on the GPU.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "st_internal.cuh"

namespace st {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

st_status cuda_fail(const char* where, cudaError_t e) {
  set_error(std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return ST_ERR_CUDA;
}

cudaError_t mg_set_attributes();

bool prof_start(const st_handle_s* h) {
  if (!h->prof_on) return false;
  if (h->prof_n + 2 > h->prof_cap) {
    // grow the event pool (outside steady state: st_profile_begin preallocates)
    int cap = h->prof_cap ? 2 * h->prof_cap : 4096;
    cudaEvent_t* ev = static_cast<cudaEvent_t*>(std::realloc(h->prof_ev, sizeof(cudaEvent_t) * cap));
    if (!ev) return false;
    for (int i = h->prof_cap; i < cap; ++i)
      if (cudaEventCreate(&ev[i]) != cudaSuccess) {
        h->prof_ev = ev;
        h->prof_cap = i;
        cudaGetLastError();
        return false;
      }
    h->prof_ev = ev;
    h->prof_cap = cap;
  }
  cudaEventRecord(h->prof_ev[h->prof_n], h->stream);
  return true;
}

void prof_stop(const st_handle_s* h, double ops, double bytes) {
  cudaEventRecord(h->prof_ev[h->prof_n + 1], h->stream);
  h->prof_n += 2;
  h->prof_ops += ops;
  h->prof_bytes += bytes;
}

}  // namespace st

using namespace st;

// ST_CHECK_CUDA(call, "where"): returns ST_ERR_CUDA with a message if the call failed.  Variadic
// so that template arguments with commas need no extra parentheses.
static inline st_status check_cuda_(cudaError_t e, const char* where) {
  return e == cudaSuccess ? ST_OK : cuda_fail(where, e);
}
#define ST_CHECK_CUDA(...)                      \
  do {                                          \
    st_status s_ = check_cuda_(__VA_ARGS__);    \
    if (s_ != ST_OK) return s_;                 \
  } while (0)

#define ST_REQUIRE(cond, msg)   \
  do {                          \
    if (!(cond)) {              \
      set_error(msg);           \
      return ST_ERR_ARG;        \
    }                           \
  } while (0)

namespace {

void free_all(st_handle_s* h) {
  double** bufs[] = {&h->U, &h->Y, &h->X, &h->Xalt, &h->Bs, &h->Z, &h->V1, &h->V2, &h->r, &h->p, &h->z, &h->q,
                     &h->g, &h->fhat, &h->w, &h->u0, &h->partials, &h->scal};
  for (double** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  for (int k = 0; k < 16; ++k) {
    if (h->mg.xc[k]) cudaFree(h->mg.xc[k]);
    if (h->mg.xc2[k]) cudaFree(h->mg.xc2[k]);
    if (h->mg.bc[k]) cudaFree(h->mg.bc[k]);
    h->mg.xc[k] = h->mg.xc2[k] = h->mg.bc[k] = nullptr;
  }
  if (h->coef) cudaFree(h->coef);
  h->coef = nullptr;
  if (h->coef32) cudaFree(h->coef32);
  h->coef32 = nullptr;
  float** fb[] = {&h->xi, &h->ri, &h->pi, &h->zi, &h->qi};
  for (float** b : fb) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  if (h->scal_host) cudaFreeHost(h->scal_host);
  h->scal_host = nullptr;
  for (int i = 0; i < h->prof_cap; ++i) cudaEventDestroy(h->prof_ev[i]);
  std::free(h->prof_ev);
  h->prof_ev = nullptr;
  h->prof_cap = h->prof_n = 0;
}

st_status alloc(double** p, size_t count, const char* what) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMalloc of ") + what + " failed: " + cudaGetErrorString(e));
    return ST_ERR_NOMEM;
  }
  return ST_OK;
}

st_status check_handle(st_handle h) {
  if (!h) {
    set_error("null handle");
    return ST_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
  return ST_OK;
}

template <typename T>
T* ws(double* p) {
  return reinterpret_cast<T*>(p);
}

template <typename T>
st_status apply_S_nodal_impl(st_handle h, const T* u, T* y) {
  ST_CHECK_CUDA(launch_timemix<T>(h, 0, u, ws<T>(h->Y)), "timemix");
  ST_CHECK_CUDA(mg_apply<T>(h, (int)(2 * h->Nt), 0, ws<T>(h->Y), ws<T>(h->X)), "K_x multigrid");
  ST_CHECK_CUDA(launch_epilogue<T>(h, ws<T>(h->X), u, y), "epilogue");
  return ST_OK;
}

template <typename T>
st_status apply_Shat_impl(st_handle h, const T* w, T* q) {
  ST_CHECK_CUDA(wavelet_synth<T>(h, w, ws<T>(h->U)), "wavelet synthesis");
  st_status s = apply_S_nodal_impl<T>(h, ws<T>(h->U), ws<T>(h->Z));
  if (s != ST_OK) return s;
  ST_CHECK_CUDA(wavelet_anal<T>(h, ws<T>(h->Z), q), "wavelet analysis");
  return ST_OK;
}

template <typename T>
st_status apply_KX_impl(st_handle h, const T* r, T* z) {
  const int nt = (int)h->Nt;
  ST_CHECK_CUDA(mg_apply<T>(h, nt, -1, r, ws<T>(h->X)), "K_l multigrid (1)");
  ST_CHECK_CUDA(launch_apply_A<T>(h, nt, ws<T>(h->X), ws<T>(h->Y)), "A_x");
  ST_CHECK_CUDA(mg_apply<T>(h, nt, -1, ws<T>(h->Y), z), "K_l multigrid (2)");
  return ST_OK;
}

st_status rhs_impl(st_handle h, const double* g, const double* u0, double* fhat) {
  ST_CHECK_CUDA(launch_timemix<double>(h, 1, g, h->Y), "timemix (rhs)");
  ST_CHECK_CUDA(mg_apply<double>(h, (int)(2 * h->Nt), 0, h->Y, h->X), "K_x multigrid (rhs)");
  ST_CHECK_CUDA(launch_epilogue<double>(h, h->X, u0, h->Z), "epilogue (rhs)");
  ST_CHECK_CUDA(wavelet_anal<double>(h, h->Z, fhat), "wavelet analysis (rhs)");
  return ST_OK;
}

st_status read_scalars(st_handle h) {
  ST_CHECK_CUDA(cudaMemcpyAsync(h->scal_host, h->scal, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost, h->stream),
                "scalar readback");
  ST_CHECK_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  return ST_OK;
}

st_status pcg64_impl(st_handle h, const double* fhat, double* w, int* iters, double* relres) {
  const int64_t n = h->Nt * h->Nx;
  const st_config& c = h->cfg;
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  ST_CHECK_CUDA(launch_zero<double>(h, w, n), "zero w");
  ST_CHECK_CUDA(launch_copy<double, double>(h, h->r, fhat, n), "copy r");
  st_status s = apply_KX_impl<double>(h, h->r, h->z);
  if (s != ST_OK) return s;
  ST_CHECK_CUDA(launch_dot<double, double>(h, h->r, h->z, n, SC_RHO, DOT_INIT), "dot r z");
  ST_CHECK_CUDA(launch_copy<double, double>(h, h->p, h->z, n), "copy p");
  if ((s = read_scalars(h)) != ST_OK) return s;
  const double rho0 = h->scal_host[SC_RHO0];
  if (!std::isfinite(rho0) || rho0 < 0.0) {
    set_error("PCG breakdown: initial r^T K_X r is negative or not finite");
    return ST_ERR_BREAKDOWN;
  }
  if (rho0 == 0.0 || (c.tol_mode == 1 && std::sqrt(rho0) <= c.tol)) return ST_OK;
  for (int it = 1; it <= c.maxit; ++it) {
    if ((s = apply_Shat_impl<double>(h, h->p, h->q)) != ST_OK) return s;
    ST_CHECK_CUDA(launch_dot<double, double>(h, h->p, h->q, n, SC_PQ, DOT_ALPHA), "dot p q");
    ST_CHECK_CUDA(launch_update_wr<double>(h, w, h->r, h->p, h->q, n), "update w r");
    if ((s = apply_KX_impl<double>(h, h->r, h->z)) != ST_OK) return s;
    ST_CHECK_CUDA(launch_dot<double, double>(h, h->r, h->z, n, SC_RHO_NEW, DOT_BETA), "dot r z");
    if ((s = read_scalars(h)) != ST_OK) return s;
    const double pq = h->scal_host[SC_PQ], rho = h->scal_host[SC_RHO_NEW];
    if (iters) *iters = it;
    if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rho) || rho < 0.0) {
      set_error("PCG breakdown: p^T S_hat p <= 0 or a non-finite scalar");
      return ST_ERR_BREAKDOWN;
    }
    const double rr = std::sqrt(rho / rho0);
    if (relres) *relres = rr;
    const bool done = c.tol_mode == 1 ? std::sqrt(rho) <= c.tol : rr <= c.tol;
    if (done) return ST_OK;
    ST_CHECK_CUDA(launch_update_p<double>(h, h->p, h->z, n), "update p");
  }
  set_error("PCG reached maxit before the tolerance");
  return ST_ERR_MAXIT;
}

// Binary32 PCG on S_hat x = ri from x = 0, with zi = K_X ri already formed; stops at a relative
// K_X-norm reduction of inner_tol or after inner_maxit iterations.  Inner products accumulate in
// binary64.  Returns the iteration count through *its.
st_status inner_pcg32(st_handle h, int* its) {
  const int64_t n = h->Nt * h->Nx;
  const st_config& c = h->cfg;
  *its = 0;
  ST_CHECK_CUDA(launch_zero<float>(h, h->xi, n), "zero inner x");
  ST_CHECK_CUDA(launch_copy<float, float>(h, h->pi, h->zi, n), "copy inner p");
  ST_CHECK_CUDA(launch_dot<float, float>(h, h->ri, h->zi, n, SC_RHO, DOT_INIT), "inner dot r z");
  st_status s;
  if ((s = read_scalars(h)) != ST_OK) return s;
  const double rho0 = h->scal_host[SC_RHO0];
  if (!(rho0 > 0.0) || !std::isfinite(rho0)) return ST_OK;  // nothing to correct (or caught by the outer test)
  for (int it = 1; it <= c.inner_maxit; ++it) {
    if ((s = apply_Shat_impl<float>(h, h->pi, h->qi)) != ST_OK) return s;
    ST_CHECK_CUDA(launch_dot<float, float>(h, h->pi, h->qi, n, SC_PQ, DOT_ALPHA), "inner dot p q");
    ST_CHECK_CUDA(launch_update_wr<float>(h, h->xi, h->ri, h->pi, h->qi, n), "inner update");
    if ((s = apply_KX_impl<float>(h, h->ri, h->zi)) != ST_OK) return s;
    ST_CHECK_CUDA(launch_dot<float, float>(h, h->ri, h->zi, n, SC_RHO_NEW, DOT_BETA), "inner dot r z");
    if ((s = read_scalars(h)) != ST_OK) return s;
    *its = it;
    const double pq = h->scal_host[SC_PQ], rho = h->scal_host[SC_RHO_NEW];
    if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rho) || rho < 0.0) {
      set_error("inner PCG breakdown: p^T S_hat p <= 0 or a non-finite scalar");
      return ST_ERR_BREAKDOWN;
    }
    if (std::sqrt(rho / rho0) <= c.inner_tol) break;
    ST_CHECK_CUDA(launch_update_p<float>(h, h->pi, h->zi, n), "inner update p");
  }
  return ST_OK;
}

// Iterative refinement: w = 0, r = f_hat; repeat { solve S_hat d = r in binary32; w += d;
// r = f_hat - S_hat w in binary64 } until sqrt(r^T K_X r) meets the tolerance (K_X in binary32,
// the inner product in binary64).
st_status pcg_mixed_impl(st_handle h, const double* fhat, double* w, int* iters, double* relres) {
  const int64_t n = h->Nt * h->Nx;
  const st_config& c = h->cfg;
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  ST_CHECK_CUDA(launch_zero<double>(h, w, n), "zero w");
  ST_CHECK_CUDA(launch_copy<double, double>(h, h->r, fhat, n), "copy r");
  ST_CHECK_CUDA(launch_copy<float, double>(h, h->ri, fhat, n), "round r");
  st_status s = apply_KX_impl<float>(h, h->ri, h->zi);
  if (s != ST_OK) return s;
  ST_CHECK_CUDA(launch_dot<double, float>(h, h->r, h->zi, n, SC_OUTER, DOT_STORE), "outer dot");
  if ((s = read_scalars(h)) != ST_OK) return s;
  const double rho0 = h->scal_host[SC_OUTER];
  if (!std::isfinite(rho0) || rho0 < 0.0) {
    set_error("PCG breakdown: initial r^T K_X r is negative or not finite");
    return ST_ERR_BREAKDOWN;
  }
  if (rho0 == 0.0 || (c.tol_mode == 1 && std::sqrt(rho0) <= c.tol)) return ST_OK;
  int total = 0;
  for (int outer = 1; total < c.maxit; ++outer) {
    int its = 0;
    if ((s = inner_pcg32(h, &its)) != ST_OK) return s;
    total += its;
    if (iters) *iters = total;
    h->last_outer = outer;
    ST_CHECK_CUDA(launch_add_correction(h, w, h->xi, n), "w += d");
    if ((s = apply_Shat_impl<double>(h, w, h->q)) != ST_OK) return s;
    ST_CHECK_CUDA(launch_residual_split(h, h->r, h->ri, fhat, h->q, n), "outer residual");
    if ((s = apply_KX_impl<float>(h, h->ri, h->zi)) != ST_OK) return s;
    ST_CHECK_CUDA(launch_dot<double, float>(h, h->r, h->zi, n, SC_OUTER, DOT_STORE), "outer dot");
    if ((s = read_scalars(h)) != ST_OK) return s;
    const double rho = h->scal_host[SC_OUTER];
    if (!std::isfinite(rho) || rho < 0.0) {
      set_error("PCG breakdown: outer r^T K_X r is negative or not finite");
      return ST_ERR_BREAKDOWN;
    }
    const double rr = std::sqrt(rho / rho0);
    if (relres) *relres = rr;
    const bool done = c.tol_mode == 1 ? std::sqrt(rho) <= c.tol : rr <= c.tol;
    if (done) return ST_OK;
    if (its == 0) break;  // the inner solve made no progress
  }
  set_error("mixed-precision refinement reached maxit before the tolerance");
  return ST_ERR_MAXIT;
}

st_status pcg_impl(st_handle h, const double* fhat, double* w, int* iters, double* relres) {
  int it = 0;
  double rr = 0.0;
  h->last_outer = 0;
  st_status s = h->cfg.precision == ST_MIXED_FP32 ? pcg_mixed_impl(h, fhat, w, &it, &rr)
                                                   : pcg64_impl(h, fhat, w, &it, &rr);
  h->last_iters = it;
  h->last_relres = rr;
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return s;
}

}  // namespace

extern "C" {

void st_default_config(st_config* cfg) {
  if (!cfg) return;
  cfg->alpha = 0.3;
  cfg->n_vcycles = 2;
  cfg->n_pre = 3;
  cfg->n_post = 3;
  cfg->tol = 1e-10;
  cfg->tol_mode = 0;
  cfg->maxit = 200;
  cfg->precision = ST_FP64;
  cfg->inner_tol = 1e-5;
  cfg->inner_maxit = 60;
}

const char* st_last_error(void) { return g_last_error.c_str(); }

st_status st_setup(st_handle* out, int domain, int space_level, int time_level, const st_config* cfg,
                   void* cuda_stream) {
  ST_REQUIRE(out != nullptr, "st_setup: null output pointer");
  *out = nullptr;
  ST_REQUIRE(domain == 0 || domain == 1, "st_setup: domain must be 0 (unit square) or 1 (L-shape)");
  ST_REQUIRE(space_level >= 1 && space_level <= 12, "st_setup: space level must be in 1..12");
  ST_REQUIRE(domain == 0 || space_level >= 2, "st_setup: the L-shape needs space level >= 2");
  ST_REQUIRE(time_level >= 1 && time_level <= 14, "st_setup: time level must be in 1..14");
  st_config c;
  st_default_config(&c);
  if (cfg) c = *cfg;
  ST_REQUIRE(c.n_vcycles >= 0 && c.n_vcycles <= 16 && c.n_pre >= 0 && c.n_pre <= 16 && c.n_post >= 0 &&
                 c.n_post <= 16,
             "st_setup: multigrid cycle / sweep counts must be in 0..16");
  ST_REQUIRE(c.alpha > 0.0 && std::isfinite(c.alpha), "st_setup: alpha must be positive");
  ST_REQUIRE(c.maxit >= 0 && c.tol >= 0.0 && (c.tol_mode == 0 || c.tol_mode == 1),
             "st_setup: invalid tolerance settings");
  ST_REQUIRE(c.precision == ST_FP64 || c.precision == ST_MIXED_FP32, "st_setup: unsupported precision");
  ST_REQUIRE(c.inner_tol > 0.0 && c.inner_tol < 1.0 && c.inner_maxit >= 1,
             "st_setup: inner_tol must be in (0, 1) and inner_maxit >= 1");

  st_handle_s* h = new (std::nothrow) st_handle_s();
  if (!h) {
    set_error("st_setup: host allocation failed");
    return ST_ERR_NOMEM;
  }
  std::memset(h, 0, sizeof(*h));
  h->domain = domain;
  h->K = space_level;
  h->J = time_level;
  h->n = (1 << space_level) - 1;
  h->Nx = (int64_t)h->n * h->n;
  h->Nt = ((int64_t)1 << time_level) + 1;
  h->cfg = c;
  h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail("cudaGetDevice", e);
  }
  h->mg.K = h->K;
  h->mg.kmin = domain == 1 ? 2 : 1;  // the L-shape has no unknown on level 1
  h->mg.max_slices = (int)(2 * h->Nt);

  const size_t V = (size_t)(h->Nt * h->Nx);
  st_status s = ST_OK;
  struct {
    double** p;
    size_t n;
    const char* name;
  } plan[] = {{&h->U, V, "U"},   {&h->Y, 2 * V, "Y"},  {&h->X, 2 * V, "X"}, {&h->Xalt, 2 * V, "Xalt"}, {&h->Bs, 2 * V, "Bs"},        {&h->Z, V, "Z"},
              {&h->V1, V, "V1"}, {&h->V2, V, "V2"},    {&h->r, V, "r"},            {&h->p, V, "p"},
              {&h->z, V, "z"},   {&h->q, V, "q"},      {&h->g, V, "g"},            {&h->fhat, V, "fhat"},
              {&h->w, V, "w"},   {&h->u0, (size_t)h->Nx, "u0"}, {&h->partials, (size_t)kDotBlocks, "partials"},
              {&h->scal, (size_t)SC_COUNT, "scalars"}};
  for (auto& a : plan)
    if (s == ST_OK) s = alloc(a.p, a.n, a.name);
  for (int k = h->mg.kmin; k <= h->K && s == ST_OK; ++k) {
    const size_t nk = (size_t)((1 << k) - 1) * ((1 << k) - 1) * (size_t)h->mg.max_slices;
    if (k < h->K) {
      s = alloc(&h->mg.xc[k], nk, "multigrid x");
      if (s == ST_OK) s = alloc(&h->mg.xc2[k], nk, "multigrid x (second buffer)");
      if (s == ST_OK) s = alloc(&h->mg.bc[k], nk, "multigrid b");
    }
  }
  // binary32 inner-solve vectors (every handle gets them: st_apply_S_f32 / st_apply_KX_f32 need none,
  // but a mixed-precision solve does)
  float** fplan[] = {&h->xi, &h->ri, &h->pi, &h->zi, &h->qi};
  for (float** fp : fplan) {
    if (s != ST_OK || c.precision != ST_MIXED_FP32) break;
    e = cudaMalloc(reinterpret_cast<void**>(fp), V * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of the binary32 inner-solve vectors failed");
      s = ST_ERR_NOMEM;
    }
  }
  if (s == ST_OK) {
    e = cudaMalloc(reinterpret_cast<void**>(&h->coef32), sizeof(Coef<float>) * (h->J + 2) * (h->K + 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of the coefficient table failed");
      s = ST_ERR_NOMEM;
    }
  }
  if (s == ST_OK) {
    e = cudaMalloc(reinterpret_cast<void**>(&h->coef), sizeof(Coef<double>) * (h->J + 2) * (h->K + 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of the coefficient table failed");
      s = ST_ERR_NOMEM;
    }
  }
  if (s == ST_OK) {
    e = cudaMallocHost(reinterpret_cast<void**>(&h->scal_host), sizeof(double) * SC_COUNT);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMallocHost of the scalar mirror failed");
      s = ST_ERR_NOMEM;
    }
  }
  if (s == ST_OK) {
    e = mg_set_attributes();
    if (e == cudaSuccess) e = launch_make_coef(h->coef, h->K, h->J, c.alpha, h->stream);
    if (e == cudaSuccess) e = launch_make_coef32(h->coef32, h->K, h->J, c.alpha, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->scal, 0, sizeof(double) * SC_COUNT, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) s = cuda_fail("st_setup", e);
  }
  if (s != ST_OK) {
    free_all(h);
    delete h;
    return s;
  }
  *out = h;
  return ST_OK;
}

st_status st_destroy(st_handle h) {
  if (!h) return ST_OK;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return ST_OK;
}

st_status st_dims(st_handle h, int64_t* Nt, int64_t* Nx) {
  ST_REQUIRE(h != nullptr, "st_dims: null handle");
  if (Nt) *Nt = h->Nt;
  if (Nx) *Nx = h->Nx;
  return ST_OK;
}

st_status st_apply_Kx(st_handle h, int nslices, const double* b, double* x) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(b && x, "st_apply_Kx: null pointer");
  ST_REQUIRE(nslices >= 1 && nslices <= 2 * h->Nt, "st_apply_Kx: nslices must be in 1..2 N_t");
  ST_CHECK_CUDA(mg_apply<double>(h, nslices, 0, b, x), "K_x multigrid");
  return ST_OK;
}

st_status st_apply_S_nodal(st_handle h, const double* u, double* y) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(u && y, "st_apply_S_nodal: null pointer");
  return apply_S_nodal_impl<double>(h, u, y);
}

st_status st_synthesize(st_handle h, const double* w, double* u) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(w && u, "st_synthesize: null pointer");
  ST_CHECK_CUDA(wavelet_synth<double>(h, w, u), "wavelet synthesis");
  return ST_OK;
}

st_status st_analyze(st_handle h, const double* u, double* w) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(w && u, "st_analyze: null pointer");
  ST_CHECK_CUDA(wavelet_anal<double>(h, u, w), "wavelet analysis");
  return ST_OK;
}

st_status st_apply_S(st_handle h, const double* w, double* q) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(w && q, "st_apply_S: null pointer");
  return apply_Shat_impl<double>(h, w, q);
}

st_status st_apply_S_f32(st_handle h, const float* w, float* q) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(w && q, "st_apply_S_f32: null pointer");
  return apply_Shat_impl<float>(h, w, q);
}

st_status st_apply_KX_f32(st_handle h, const float* r, float* z) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(r && z, "st_apply_KX_f32: null pointer");
  return apply_KX_impl<float>(h, r, z);
}

st_status st_solve_info_get(st_handle h, st_solve_info* out) {
  ST_REQUIRE(h != nullptr && out != nullptr, "st_solve_info_get: null pointer");
  out->iterations = h->last_iters;
  out->outer_iterations = h->last_outer;
  out->relres = h->last_relres;
  return ST_OK;
}

st_status st_apply_KX(st_handle h, const double* r, double* z) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(r && z, "st_apply_KX: null pointer");
  return apply_KX_impl<double>(h, r, z);
}

st_status st_rhs(st_handle h, const double* g, const double* u0, double* fhat) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(g && u0 && fhat, "st_rhs: null pointer");
  return rhs_impl(h, g, u0, fhat);
}

st_status st_pcg_solve(st_handle h, const double* fhat, double* w, int* iters, double* relres) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(fhat && w, "st_pcg_solve: null pointer");
  return pcg_impl(h, fhat, w, iters, relres);
}

st_status st_solve_host(st_handle h, const double* g_host, const double* u0_host, double* u_host, int* iters,
                        double* relres) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(g_host && u0_host && u_host, "st_solve_host: null pointer");
  const size_t V = (size_t)(h->Nt * h->Nx);
  ST_CHECK_CUDA(cudaMemcpyAsync(h->g, g_host, V * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy g");
  ST_CHECK_CUDA(cudaMemcpyAsync(h->u0, u0_host, (size_t)h->Nx * sizeof(double), cudaMemcpyHostToDevice, h->stream),
                "copy u0");
  if ((s = rhs_impl(h, h->g, h->u0, h->fhat)) != ST_OK) return s;
  st_status ps = pcg_impl(h, h->fhat, h->w, iters, relres);
  if (ps != ST_OK && ps != ST_ERR_MAXIT) return ps;
  ST_CHECK_CUDA(wavelet_synth<double>(h, h->w, h->g), "wavelet synthesis");
  ST_CHECK_CUDA(cudaMemcpyAsync(u_host, h->g, V * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy u");
  ST_CHECK_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  return ps;
}

st_status st_profile_begin(st_handle h) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  h->launches = 0;
  h->prof_n = 0;
  h->prof_ops = h->prof_bytes = 0.0;
  h->prof_on = true;
  // preallocate events so that recording inside the timed region never creates them
  if (h->prof_cap < 16384 && prof_start(h)) {
    // prof_start grew the pool to at least 4096; grow further by faking a full pool
    while (h->prof_cap < 16384) {
      h->prof_n = h->prof_cap;
      if (!prof_start(h)) break;
    }
  }
  ST_CHECK_CUDA(cudaStreamSynchronize(h->stream), "st_profile_begin");
  h->prof_n = 0;
  h->launches = 0;
  return ST_OK;
}

st_status st_profile_end(st_handle h, st_profile* out) {
  st_status s = check_handle(h);
  if (s != ST_OK) return s;
  ST_REQUIRE(out != nullptr, "st_profile_end: null output");
  ST_CHECK_CUDA(cudaStreamSynchronize(h->stream), "st_profile_end");
  double ms = 0.0;
  for (int i = 0; i + 1 < h->prof_n; i += 2) {
    float t = 0.f;
    ST_CHECK_CUDA(cudaEventElapsedTime(&t, h->prof_ev[i], h->prof_ev[i + 1]), "cudaEventElapsedTime");
    ms += t;
  }
  out->launches = h->launches;
  out->sweep_launches = h->prof_n / 2;
  out->sweep_ms = ms;
  out->sweep_fp64_ops = h->prof_ops;
  out->sweep_bytes = h->prof_bytes;
  h->prof_on = false;
  h->prof_n = 0;
  return ST_OK;
}

}  // extern "C"
