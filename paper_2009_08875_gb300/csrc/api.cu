// C ABI of libst (declared in include/st.h): handle set-up, the operators of the Schur-complement
// PCG (Sec. 3.4, Lemma 4.2, Thm. 3.1, Eq. 3.1) and the host-side PCG drivers.  Host code only
// validates arguments, sizes workspaces, enqueues kernels and reads back per-problem scalars for
// the stop tests; all arithmetic runs on the GPU.  A handle holds B >= 1 problems of the same
// domain, space level and time level, stored back to back; every operator acts on all of them.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <type_traits>

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
    unsigned char* cat = static_cast<unsigned char*>(std::realloc(h->prof_cat, cap));
    if (!cat) return false;
    h->prof_cat = cat;
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

void prof_stop(const st_handle_s* h, int cat, double ops, double bytes) {
  cudaEventRecord(h->prof_ev[h->prof_n + 1], h->stream);
  h->prof_cat[h->prof_n] = (unsigned char)cat;
  h->prof_n += 2;
  h->prof_ops[cat] += ops;
  h->prof_bytes[cat] += bytes;
}

}  // namespace st

using namespace st;

// ST_CHECK_CUDA(call, "where"): returns ST_ERR_CUDA with a message if the call failed.  Variadic
// so that template arguments with commas need no extra parentheses.
static inline st_status check_cuda_(cudaError_t e, const char* where) {
  return e == cudaSuccess ? ST_OK : cuda_fail(where, e);
}
#define ST_CHECK_CUDA(...)                   \
  do {                                       \
    st_status s_ = check_cuda_(__VA_ARGS__); \
    if (s_ != ST_OK) return s_;              \
  } while (0)

#define ST_CHECK(call)          \
  do {                          \
    st_status s_ = (call);      \
    if (s_ != ST_OK) return s_; \
  } while (0)

#define ST_REQUIRE(cond, msg) \
  do {                        \
    if (!(cond)) {            \
      set_error(msg);         \
      return ST_ERR_ARG;      \
    }                         \
  } while (0)

namespace {

// D = [[d11, d12], [d12, d22]] symmetric positive definite, c >= 0, all finite (Sec. 4)
bool check_phys(const st_config& c) {
  const double d11 = c.diffusion[0], d12 = c.diffusion[1], d22 = c.diffusion[2], r = c.reaction;
  return std::isfinite(d11) && std::isfinite(d12) && std::isfinite(d22) && std::isfinite(r) && d11 > 0.0 &&
         d22 > 0.0 && d11 * d22 - d12 * d12 > 0.0 && r >= 0.0;
}

void free_all(st_handle_s* h) {
  double** bufs[] = {&h->U, &h->Y, &h->X, &h->Xalt, &h->Bs,   &h->Z, &h->V1, &h->V2,       &h->r,
                     &h->p, &h->z, &h->q, &h->g,    &h->fhat, &h->w, &h->u0, &h->partials, &h->scal};
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
  if (h->coefdf) cudaFree(h->coefdf);
  h->coefdf = nullptr;
  float** fb[] = {&h->xi, &h->ri, &h->pi, &h->zi, &h->qi};
  for (float** b : fb) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  if (h->act) cudaFree(h->act);
  h->act = nullptr;
  if (h->scal_host) cudaFreeHost(h->scal_host);
  h->scal_host = nullptr;
  if (h->act_host) cudaFreeHost(h->act_host);
  h->act_host = nullptr;
  std::free(h->info_iters);
  std::free(h->info_outer);
  std::free(h->info_status);
  std::free(h->info_relres);
  h->info_iters = h->info_outer = h->info_status = nullptr;
  h->info_relres = nullptr;
  for (int i = 0; i < 3; ++i) {
    if (h->graph_exec[i]) cudaGraphExecDestroy(h->graph_exec[i]);
    h->graph_exec[i] = nullptr;
  }
  if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
  h->loop_exec = nullptr;
  if (h->ds_mem) cudaFree(h->ds_mem);
  h->ds_mem = nullptr;
  for (int i = 0; i < h->prof_cap; ++i) cudaEventDestroy(h->prof_ev[i]);
  std::free(h->prof_ev);
  std::free(h->prof_cat);
  h->prof_ev = nullptr;
  h->prof_cat = nullptr;
  h->prof_cap = h->prof_n = 0;
}

st_status alloc_bytes(void** p, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMalloc of ") + what + " failed: " + cudaGetErrorString(e));
    return ST_ERR_NOMEM;
  }
  return ST_OK;
}

st_status alloc(double** p, size_t count, const char* what) {
  return alloc_bytes(reinterpret_cast<void**>(p), count * sizeof(double), what);
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

// ---------------------------------------------------------------------------------------------
// operators on nb problems of a handle (all of them, or a range whose vectors start at problem b0;
// the workspace is scratch, so any range works)
// ---------------------------------------------------------------------------------------------
template <typename T>
st_status apply_S_nodal_impl(st_handle h, int nb, const T* u, T* y) {
  ST_CHECK_CUDA(launch_timemix<T>(h, nb, 0, u, ws<T>(h->Y)), "timemix");
  ST_CHECK_CUDA(mg_apply<T>(h, (int)(2 * nb * h->Nt), 0, ws<T>(h->Y), ws<T>(h->X)), "K_x multigrid");
  ST_CHECK_CUDA(launch_epilogue<T>(h, nb, ws<T>(h->X), u, h->Nt * h->Nx, y), "epilogue");
  return ST_OK;
}

template <typename T>
st_status apply_Shat_impl(st_handle h, int nb, const T* w, T* q) {
  ST_CHECK_CUDA(wavelet_synth<T>(h, nb, w, ws<T>(h->U)), "wavelet synthesis");
  ST_CHECK(apply_S_nodal_impl<T>(h, nb, ws<T>(h->U), ws<T>(h->Z)));
  ST_CHECK_CUDA(wavelet_anal<T>(h, nb, ws<T>(h->Z), q), "wavelet analysis");
  return ST_OK;
}

// K_l multigrid on `rows` slices; narrow: binary32 work with bfloat16 storage
template <typename T>
cudaError_t mg_kl(st_handle h, int rows, const T* b, T* x, bool narrow) {
  if constexpr (std::is_same<T, float>::value) {
    if (narrow) return mg_apply_bf16(h, rows, -1, b, x);
  }
  return mg_apply<T>(h, rows, -1, b, x);
}

template <typename T>
st_status apply_KX_impl(st_handle h, int nb, const T* r, T* z, bool narrow = false) {
  const int rows = (int)(nb * h->Nt);
  ST_CHECK_CUDA(mg_kl<T>(h, rows, r, ws<T>(h->X), narrow), "K_l multigrid (1)");
  ST_CHECK_CUDA(launch_apply_A<T>(h, rows, ws<T>(h->X), ws<T>(h->Y)), "A_x");
  ST_CHECK_CUDA(mg_kl<T>(h, rows, ws<T>(h->Y), z, narrow), "K_l multigrid (2)");
  return ST_OK;
}

// ---------------------------------------------------------------------------------------------
// per-problem PCG bookkeeping
// ---------------------------------------------------------------------------------------------
st_status read_scalars(st_handle h) {
  ST_CHECK_CUDA(cudaMemcpyAsync(h->scal_host, h->scal, sizeof(double) * SC_COUNT * h->B, cudaMemcpyDeviceToHost,
                                h->stream),
                "scalar readback");
  ST_CHECK_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  return ST_OK;
}

st_status push_act(st_handle h) {
  ST_CHECK_CUDA(cudaMemcpyAsync(h->act, h->act_host, sizeof(int) * h->B, cudaMemcpyHostToDevice, h->stream),
                "active flags");
  return ST_OK;
}

inline double sc(st_handle h, int b, int slot) { return h->scal_host[(size_t)b * SC_COUNT + slot]; }

// Destroys the captured graphs of a handle (the kernel choices or the vectors they name changed).
void drop_graphs(st_handle h) {
  for (int i = 0; i < 3; ++i) {
    if (h->graph_exec[i]) cudaGraphExecDestroy(h->graph_exec[i]);
    h->graph_exec[i] = nullptr;
  }
  if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
  h->loop_exec = nullptr;
}

// Runs one PCG iteration body.  With graphs enabled (on a stream other than the legacy and
// per-thread default streams, outside profiling) the first call captures the body's launches
// into a CUDA graph that later calls replay; `key` names the caller-owned vectors the body
// touches, and a different key captures again.
template <typename F>
st_status run_body(st_handle h, int slot, const void* key, F body) {
  const uintptr_t sv = reinterpret_cast<uintptr_t>(h->stream);
  const bool use = h->cfg.use_graphs && sv > 2 && !h->prof_on;
  if (!use) return body();
  if (h->graph_exec[slot] && h->graph_key[slot] != key) {
    cudaGraphExecDestroy(h->graph_exec[slot]);
    h->graph_exec[slot] = nullptr;
  }
  if (!h->graph_exec[slot]) {
    const int64_t before = h->launches;
    ST_CHECK_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin graph capture");
    st_status s = body();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (s != ST_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail("end graph capture", e);
    e = cudaGraphInstantiate(&h->graph_exec[slot], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->graph_exec[slot] = nullptr;
      return cuda_fail("graph instantiate", e);
    }
    h->graph_launches[slot] = h->launches - before;
    h->launches = before;
    h->graph_key[slot] = key;
  }
  ST_CHECK_CUDA(cudaGraphLaunch(h->graph_exec[slot], h->stream), "graph launch");
  h->launches += h->graph_launches[slot];
  return ST_OK;
}

bool any_active(st_handle h) {
  for (int b = 0; b < h->B; ++b)
    if (h->act_host[b]) return true;
  return false;
}

struct Tracker {
  std::vector<double> rho0;
  bool changed = false;
};

// Initial test of every problem from rho0 (r_0^T K_X r_0): sets the active flags.
void init_problems(st_handle h, Tracker& t, int slot) {
  const st_config& c = h->cfg;
  t.rho0.assign(h->B, 0.0);
  for (int b = 0; b < h->B; ++b) {
    h->info_iters[b] = 0;
    h->info_outer[b] = 0;
    h->info_relres[b] = 0.0;
    h->info_status[b] = ST_OK;
    const double r0 = sc(h, b, slot);
    t.rho0[b] = r0;
    h->act_host[b] = 1;
    if (!std::isfinite(r0) || r0 < 0.0) {
      h->info_status[b] = ST_ERR_BREAKDOWN;
      h->act_host[b] = 0;
    } else if (r0 == 0.0 || (c.tol_mode == 1 && std::sqrt(r0) <= c.tol)) {
      h->act_host[b] = 0;
    }
  }
}

// Stop test of problem b after an iteration with squared K_X-norm rho (and p^T q if checked).
void test_problem(st_handle h, Tracker& t, int b, double rho, double pq, bool check_pq) {
  const st_config& c = h->cfg;
  if ((check_pq && (!(pq > 0.0) || !std::isfinite(pq))) || !std::isfinite(rho) || rho < 0.0) {
    h->info_status[b] = ST_ERR_BREAKDOWN;
    h->act_host[b] = 0;
    t.changed = true;
    return;
  }
  const double rr = std::sqrt(rho / t.rho0[b]);
  h->info_relres[b] = rr;
  const bool done = c.tol_mode == 1 ? std::sqrt(rho) <= c.tol : rr <= c.tol;
  if (done) {
    h->act_host[b] = 0;
    t.changed = true;
  }
}

// Overall status: a breakdown in any problem, else maxit in any problem, else OK.
st_status finish(st_handle h) {
  int its = 0, outer = 0;
  double rr = 0.0;
  st_status s = ST_OK;
  for (int b = 0; b < h->B; ++b) {
    if (h->act_host[b] && h->info_status[b] == ST_OK) h->info_status[b] = ST_ERR_MAXIT;
    its = its > h->info_iters[b] ? its : h->info_iters[b];
    outer = outer > h->info_outer[b] ? outer : h->info_outer[b];
    rr = rr > h->info_relres[b] ? rr : h->info_relres[b];
    if (h->info_status[b] == ST_ERR_BREAKDOWN) s = ST_ERR_BREAKDOWN;
    if (h->info_status[b] == ST_ERR_MAXIT && s == ST_OK) s = ST_ERR_MAXIT;
  }
  h->last_iters = its;
  h->last_outer = outer;
  h->last_relres = rr;
  if (s == ST_ERR_BREAKDOWN) set_error("PCG breakdown: p^T S_hat p <= 0 or a non-finite scalar in some problem");
  if (s == ST_ERR_MAXIT) set_error("PCG reached maxit before the tolerance in some problem");
  return s;
}

// Initial residual: r = f_hat - S_hat w from the caller's w when h->use_guess is set (nested
// iteration), else w = 0 and r = f_hat.
st_status init_residual(st_handle h, const double* fhat, double* w) {
  const int64_t N = h->B * h->Nt * h->Nx;
  if (h->use_guess) {
    ST_CHECK(apply_Shat_impl<double>(h, h->B, w, h->q));
    ST_CHECK_CUDA(launch_residual_split(h, h->r, nullptr, fhat, h->q, N), "initial residual");
  } else {
    ST_CHECK_CUDA(launch_zero<double>(h, w, N), "zero w");
    ST_CHECK_CUDA(launch_copy<double, double>(h, h->r, fhat, N), "copy r");
  }
  return ST_OK;
}

// ---------------------------------------------------------------------------------------------
// PCG iteration bodies on all B problems: p = z + beta p, q = S_hat p, alpha, w and r updates,
// z = K_X r, rho and beta (problems whose active flag is clear keep their vectors)
// ---------------------------------------------------------------------------------------------
st_status body64(st_handle h, double* w, int nb) {
  const int64_t n = h->Nt * h->Nx;
  ST_CHECK_CUDA(launch_update_p<double>(h, 0, nb, h->p, h->z, n), "update p");
  ST_CHECK(apply_Shat_impl<double>(h, nb, h->p, h->q));
  ST_CHECK_CUDA(launch_dot<double, double>(h, 0, nb, h->p, h->q, n, SC_PQ, DOT_ALPHA), "dot p q");
  ST_CHECK_CUDA(launch_update_wr<double>(h, 0, nb, w, h->r, h->p, h->q, n), "update w r");
  ST_CHECK(apply_KX_impl<double>(h, nb, h->r, h->z));
  ST_CHECK_CUDA(launch_dot<double, double>(h, 0, nb, h->r, h->z, n, SC_RHO_NEW, DOT_BETA), "dot r z");
  return ST_OK;
}

st_status precond32(st_handle h, int nb, const double* r, double* z, float* ri, float* zi) {
  const int64_t N = nb * h->Nt * h->Nx;
  ST_CHECK_CUDA(launch_copy<float, double>(h, ri, r, N), "round r");
  ST_CHECK(apply_KX_impl<float>(h, nb, ri, zi));
  ST_CHECK_CUDA(launch_copy<double, float>(h, z, zi, N), "widen z");
  return ST_OK;
}

st_status body_precond(st_handle h, double* w, int nb) {
  const int64_t n = h->Nt * h->Nx;
  ST_CHECK_CUDA(launch_update_p<double>(h, 0, nb, h->p, h->z, n), "update p");
  ST_CHECK(apply_Shat_impl<double>(h, nb, h->p, h->q));
  ST_CHECK_CUDA(launch_dot<double, double>(h, 0, nb, h->p, h->q, n, SC_PQ, DOT_ALPHA), "dot p q");
  ST_CHECK_CUDA(launch_update_wr<double>(h, 0, nb, w, h->r, h->p, h->q, n), "update w r");
  ST_CHECK_CUDA(launch_dot<double, double>(h, 0, nb, h->r, h->z, n, SC_RZOLD, DOT_STORE), "dot r z_old");
  ST_CHECK(precond32(h, nb, h->r, h->z, h->ri, h->zi));
  ST_CHECK_CUDA(launch_dot<double, double>(h, 0, nb, h->r, h->z, n, SC_RHO_NEW, DOT_BETA_FLEX), "dot r z");
  return ST_OK;
}

// ---------------------------------------------------------------------------------------------
// FP64 PCG (Sec. 3.4), all B problems in lock step, each with its own scalars and stop test
// ---------------------------------------------------------------------------------------------
st_status pcg64_impl(st_handle h, const double* fhat, double* w) {
  const int nb = h->B;
  const int64_t n = h->Nt * h->Nx;
  const st_config& c = h->cfg;
  Tracker t;
  for (int b = 0; b < nb; ++b) h->act_host[b] = 1;
  ST_CHECK(push_act(h));
  ST_CHECK(init_residual(h, fhat, w));
  ST_CHECK(apply_KX_impl<double>(h, h->B, h->r, h->z));
  ST_CHECK_CUDA(launch_dot<double, double>(h, 0, nb, h->r, h->z, n, SC_RHO, DOT_INIT), "dot r z");
  ST_CHECK_CUDA(launch_zero<double>(h, h->p, n * nb), "zero p");  // first body: p = z + 0 p
  ST_CHECK(read_scalars(h));
  init_problems(h, t, SC_RHO0);
  ST_CHECK(push_act(h));
  auto body = [&]() -> st_status { return body64(h, w, nb); };
  for (int it = 1; it <= c.maxit && any_active(h); ++it) {
    ST_CHECK(run_body(h, 0, w, body));
    ST_CHECK(read_scalars(h));
    t.changed = false;
    for (int b = 0; b < nb; ++b) {
      if (!h->act_host[b]) continue;
      h->info_iters[b] = it;
      test_problem(h, t, b, sc(h, b, SC_RHO_NEW), sc(h, b, SC_PQ), true);
    }
    if (t.changed && any_active(h)) ST_CHECK(push_act(h));
  }
  return finish(h);
}

// ---------------------------------------------------------------------------------------------
// ST_MIXED_FP32: binary64 iterative refinement around a binary32 PCG (per problem)
// ---------------------------------------------------------------------------------------------
// One iteration of the inner binary32 PCG on all problems (narrow: the preconditioner stores its
// multigrid vectors as bfloat16 and beta takes the flexible form).
st_status body_inner32(st_handle h, bool narrow) {
  const int nb = h->B;
  const int64_t n = h->Nt * h->Nx;
  ST_CHECK_CUDA(launch_update_p<float>(h, 0, nb, h->pi, h->zi, n), "inner update p");
  ST_CHECK(apply_Shat_impl<float>(h, h->B, h->pi, h->qi));
  ST_CHECK_CUDA(launch_dot<float, float>(h, 0, nb, h->pi, h->qi, n, SC_PQ, DOT_ALPHA), "inner dot p q");
  ST_CHECK_CUDA(launch_update_wr<float>(h, 0, nb, h->xi, h->ri, h->pi, h->qi, n), "inner update");
  if (narrow)
    ST_CHECK_CUDA(launch_dot<float, float>(h, 0, nb, h->ri, h->zi, n, SC_RZOLD, DOT_STORE), "inner dot r z_old");
  ST_CHECK(apply_KX_impl<float>(h, h->B, h->ri, h->zi, narrow));
  ST_CHECK_CUDA(launch_dot<float, float>(h, 0, nb, h->ri, h->zi, n, SC_RHO_NEW, narrow ? DOT_BETA_FLEX : DOT_BETA),
                "inner dot r z");
  return ST_OK;
}

// Binary32 PCG on S_hat x = ri for the problems with out_act[b] set, from x = 0, with
// zi = K_X ri already formed; each stops at a relative reduction of inner_tol or inner_maxit.
// ST_MIXED_BF16: the preconditioner stores its multigrid vectors as bfloat16, which makes it
// slightly nonlinear, so beta takes the flexible (Polak-Ribiere) form r^T (z - z_old) / rho_old.
st_status inner_pcg32(st_handle h, const std::vector<int>& out_act, std::vector<int>& its) {
  const int nb = h->B;
  const int64_t n = h->Nt * h->Nx;
  const st_config& c = h->cfg;
  const bool narrow = c.precision == ST_MIXED_BF16;
  ST_CHECK_CUDA(launch_zero<float>(h, h->xi, n * nb), "zero inner x");
  ST_CHECK_CUDA(launch_zero<float>(h, h->pi, n * nb), "zero inner p");  // first body: p = z + 0 p
  ST_CHECK_CUDA(launch_dot<float, float>(h, 0, nb, h->ri, h->zi, n, SC_RHO, DOT_INIT), "inner dot r z");
  ST_CHECK(read_scalars(h));
  std::vector<double> rho0(nb);
  for (int b = 0; b < nb; ++b) {
    its[b] = 0;
    rho0[b] = sc(h, b, SC_RHO0);
    h->act_host[b] = out_act[b] && rho0[b] > 0.0 && std::isfinite(rho0[b]);
  }
  ST_CHECK(push_act(h));
  auto body = [&]() -> st_status { return body_inner32(h, narrow); };
  for (int it = 1; it <= c.inner_maxit && any_active(h); ++it) {
    ST_CHECK(run_body(h, 1, nullptr, body));
    ST_CHECK(read_scalars(h));
    bool changed = false;
    for (int b = 0; b < nb; ++b) {
      if (!h->act_host[b]) continue;
      its[b] = it;
      const double pq = sc(h, b, SC_PQ), rho = sc(h, b, SC_RHO_NEW);
      if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rho) || rho < 0.0 ||
          std::sqrt(rho / rho0[b]) <= c.inner_tol) {
        h->act_host[b] = 0;  // converged, or no further progress possible in binary32
        changed = true;
      }
    }
    if (changed && any_active(h)) ST_CHECK(push_act(h));
  }
  return ST_OK;
}

st_status pcg_mixed_impl(st_handle h, const double* fhat, double* w) {
  const int nb = h->B;
  const int64_t n = h->Nt * h->Nx;
  const st_config& c = h->cfg;
  Tracker t;
  ST_CHECK(init_residual(h, fhat, w));
  ST_CHECK_CUDA(launch_copy<float, double>(h, h->ri, h->r, n * nb), "round r");
  ST_CHECK(apply_KX_impl<float>(h, h->B, h->ri, h->zi));
  ST_CHECK_CUDA(launch_dot<double, float>(h, 0, nb, h->r, h->zi, n, SC_OUTER, DOT_STORE), "outer dot");
  ST_CHECK(read_scalars(h));
  init_problems(h, t, SC_OUTER);
  std::vector<int> out_act(h->act_host, h->act_host + nb), its(nb, 0);
  for (int step = 0; step < c.maxit; ++step) {
    bool any = false;
    for (int b = 0; b < nb; ++b) any = any || out_act[b];
    if (!any) break;
    ST_CHECK(inner_pcg32(h, out_act, its));
    bool progress = false;
    for (int b = 0; b < nb; ++b) {
      if (!out_act[b]) continue;
      h->info_iters[b] += its[b];
      h->info_outer[b] += 1;
      progress = progress || its[b] > 0;
    }
    ST_CHECK_CUDA(launch_add_correction(h, w, h->xi, n * nb), "w += d");
    ST_CHECK(apply_Shat_impl<double>(h, h->B, w, h->q));
    ST_CHECK_CUDA(launch_residual_split(h, h->r, h->ri, fhat, h->q, n * nb), "outer residual");
    ST_CHECK(apply_KX_impl<float>(h, h->B, h->ri, h->zi));
    ST_CHECK_CUDA(launch_dot<double, float>(h, 0, nb, h->r, h->zi, n, SC_OUTER, DOT_STORE), "outer dot");
    ST_CHECK(read_scalars(h));
    for (int b = 0; b < nb; ++b) {
      if (!out_act[b]) continue;
      h->act_host[b] = 1;
      test_problem(h, t, b, sc(h, b, SC_OUTER), 0.0, false);
      if (!h->act_host[b]) out_act[b] = 0;
      if (h->act_host[b] && h->info_iters[b] >= c.maxit) {
        h->info_status[b] = ST_ERR_MAXIT;
        out_act[b] = 0;
      }
    }
    if (!progress) break;
  }
  for (int b = 0; b < nb; ++b) h->act_host[b] = out_act[b];
  return finish(h);
}

// ---------------------------------------------------------------------------------------------
// ST_MIXED_PRECOND: binary64 flexible PCG (binary64 S_hat, recurrences, inner products) with the
// binary32 K_X as preconditioner; beta = r^T (z - z_old) / rho_old (Polak-Ribiere), which keeps
// the method convergent for a preconditioner that is only approximately linear
// ---------------------------------------------------------------------------------------------
st_status pcg_precond_impl(st_handle h, const double* fhat, double* w) {
  const int nb = h->B;
  const int64_t n = h->Nt * h->Nx;
  const st_config& c = h->cfg;
  Tracker t;
  for (int b = 0; b < nb; ++b) h->act_host[b] = 1;
  ST_CHECK(push_act(h));
  ST_CHECK(init_residual(h, fhat, w));
  ST_CHECK(precond32(h, nb, h->r, h->z, h->ri, h->zi));
  ST_CHECK_CUDA(launch_dot<double, double>(h, 0, nb, h->r, h->z, n, SC_RHO, DOT_INIT), "dot r z");
  ST_CHECK_CUDA(launch_zero<double>(h, h->p, n * nb), "zero p");  // first body: p = z + 0 p
  ST_CHECK(read_scalars(h));
  init_problems(h, t, SC_RHO0);
  ST_CHECK(push_act(h));
  auto body = [&]() -> st_status { return body_precond(h, w, nb); };
  for (int it = 1; it <= c.maxit && any_active(h); ++it) {
    ST_CHECK(run_body(h, 2, w, body));
    ST_CHECK(read_scalars(h));
    t.changed = false;
    for (int b = 0; b < nb; ++b) {
      if (!h->act_host[b]) continue;
      h->info_iters[b] = it;
      test_problem(h, t, b, sc(h, b, SC_RHO_NEW), sc(h, b, SC_PQ), true);
    }
    if (t.changed && any_active(h)) ST_CHECK(push_act(h));
  }
  return finish(h);
}

// ---------------------------------------------------------------------------------------------
// Device-driven solves (cfg.use_graphs = 2): the whole PCG loop is captured into one CUDA graph.
// A WHILE node repeats the iteration body, and a stop-test kernel at the end of each body takes
// the per-problem decisions of the host-driven loop above on the device and sets the node's
// condition, so a solve needs no host round trip per iteration (the refinement of ST_MIXED_FP32
// nests an inner WHILE node in the outer one).  The kernels and their order are those of the
// host-driven loop, so the results are bitwise the same.
// ---------------------------------------------------------------------------------------------
// Capture of work enqueued on the handle's stream into graph G after the nodes `leaves`; end()
// replaces `leaves` by the last nodes captured.
struct GraphCapture {
  st_handle h;
  cudaGraph_t G;
  std::vector<cudaGraphNode_t>* leaves;
  st_status begin() {
    ST_CHECK_CUDA(cudaStreamBeginCaptureToGraph(h->stream, G, leaves->empty() ? nullptr : leaves->data(), nullptr,
                                                leaves->size(), cudaStreamCaptureModeThreadLocal),
                  "begin capture");
    return ST_OK;
  }
  // ends the capture; `ok` is the status of the work enqueued (the capture ends either way)
  st_status end(st_status ok) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, nullptr, &deps, nullptr, &nd);
    std::vector<cudaGraphNode_t> out;
    if (e == cudaSuccess) out.assign(deps, deps + nd);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (ok != ST_OK) return ok;
    if (e != cudaSuccess) return cuda_fail("capture info", e);
    if (e2 != cudaSuccess) return cuda_fail("end capture", e2);
    *leaves = out;
    return ST_OK;
  }
};

// Appends a WHILE node with condition hc after `leaves` to G; *body receives its body graph and
// `leaves` becomes the node.
st_status add_while(cudaGraph_t G, std::vector<cudaGraphNode_t>& leaves, cudaGraphConditionalHandle hc,
                    cudaGraph_t* body) {
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = hc;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  ST_CHECK_CUDA(cudaGraphAddNode(&node, G, leaves.empty() ? nullptr : leaves.data(), nullptr, leaves.size(), &p),
                "add WHILE node");
  *body = p.conditional.phGraph_out[0];
  leaves.assign(1, node);
  return ST_OK;
}

// Captures `work` (enqueued on the handle's stream) into G after `leaves`.
template <typename F>
st_status capture_into(st_handle h, cudaGraph_t G, std::vector<cudaGraphNode_t>& leaves, F work) {
  GraphCapture c{h, G, &leaves};
  ST_CHECK(c.begin());
  return c.end(work());
}

// A loop: WHILE(hc) { body; test } after `leaves` in G.
template <typename F>
st_status capture_loop(st_handle h, cudaGraph_t G, std::vector<cudaGraphNode_t>& leaves,
                       cudaGraphConditionalHandle hc, F body) {
  cudaGraph_t bg = nullptr;
  ST_CHECK(add_while(G, leaves, hc, &bg));
  std::vector<cudaGraphNode_t> inner;
  return capture_into(h, bg, inner, body);
}

// The PCG program of the handle's precision into G after `leaves` (the solve of pcg_impl).
st_status capture_pcg(st_handle h, cudaGraph_t G, std::vector<cudaGraphNode_t>& leaves, const double* fhat,
                      double* w) {
  const int nb = h->B;
  const int64_t n = h->Nt * h->Nx;
  const int prec = h->cfg.precision;
  cudaGraphConditionalHandle hc;
  ST_CHECK_CUDA(cudaGraphConditionalHandleCreate(&hc, G, 0, 0), "conditional handle");
  if (prec == ST_MIXED_FP32 || prec == ST_MIXED_BF16) {
    const bool narrow = prec == ST_MIXED_BF16;
    ST_CHECK(capture_into(h, G, leaves, [&]() -> st_status {
      ST_CHECK(init_residual(h, fhat, w));
      ST_CHECK_CUDA(launch_copy<float, double>(h, h->ri, h->r, n * nb), "round r");
      ST_CHECK(apply_KX_impl<float>(h, nb, h->ri, h->zi));
      ST_CHECK_CUDA(launch_dot<double, float>(h, 0, nb, h->r, h->zi, n, SC_OUTER, DOT_STORE), "outer dot");
      ST_CHECK_CUDA(launch_loop_test(h, LOOP_INIT, SC_OUTER, false, true, hc), "outer test");
      return ST_OK;
    }));
    // outer step: inner binary32 PCG, then the binary64 residual and the outer test
    cudaGraph_t ob = nullptr;
    ST_CHECK(add_while(G, leaves, hc, &ob));
    cudaGraphConditionalHandle hi;
    ST_CHECK_CUDA(cudaGraphConditionalHandleCreate(&hi, ob, 0, 0), "conditional handle");
    std::vector<cudaGraphNode_t> ol;
    ST_CHECK(capture_into(h, ob, ol, [&]() -> st_status {
      ST_CHECK_CUDA(launch_zero<float>(h, h->xi, n * nb), "zero inner x");
      ST_CHECK_CUDA(launch_zero<float>(h, h->pi, n * nb), "zero inner p");
      ST_CHECK_CUDA(launch_dot<float, float>(h, 0, nb, h->ri, h->zi, n, SC_RHO, DOT_INIT), "inner dot r z");
      ST_CHECK_CUDA(launch_inner_test(h, LOOP_INIT, hi), "inner test");
      return ST_OK;
    }));
    ST_CHECK(capture_loop(h, ob, ol, hi, [&]() -> st_status {
      ST_CHECK(body_inner32(h, narrow));
      ST_CHECK_CUDA(launch_inner_test(h, LOOP_ITER, hi), "inner test");
      return ST_OK;
    }));
    return capture_into(h, ob, ol, [&]() -> st_status {
      ST_CHECK_CUDA(launch_refine_count(h), "refinement count");
      ST_CHECK_CUDA(launch_add_correction(h, w, h->xi, n * nb), "w += d");
      ST_CHECK(apply_Shat_impl<double>(h, nb, w, h->q));
      ST_CHECK_CUDA(launch_residual_split(h, h->r, h->ri, fhat, h->q, n * nb), "outer residual");
      ST_CHECK(apply_KX_impl<float>(h, nb, h->ri, h->zi));
      ST_CHECK_CUDA(launch_dot<double, float>(h, 0, nb, h->r, h->zi, n, SC_OUTER, DOT_STORE), "outer dot");
      ST_CHECK_CUDA(launch_loop_test(h, LOOP_ITER, SC_OUTER, false, true, hc), "outer test");
      return ST_OK;
    });
  }
  const bool pre = prec == ST_MIXED_PRECOND;
  ST_CHECK(capture_into(h, G, leaves, [&]() -> st_status {
    ST_CHECK(init_residual(h, fhat, w));
    if (pre)
      ST_CHECK(precond32(h, nb, h->r, h->z, h->ri, h->zi));
    else
      ST_CHECK(apply_KX_impl<double>(h, nb, h->r, h->z));
    ST_CHECK_CUDA(launch_dot<double, double>(h, 0, nb, h->r, h->z, n, SC_RHO, DOT_INIT), "dot r z");
    ST_CHECK_CUDA(launch_zero<double>(h, h->p, n * nb), "zero p");  // first body: p = z + 0 p
    ST_CHECK_CUDA(launch_loop_test(h, LOOP_INIT, SC_RHO0, false, false, hc), "stop test");
    return ST_OK;
  }));
  return capture_loop(h, G, leaves, hc, [&]() -> st_status {
    ST_CHECK(pre ? body_precond(h, w, nb) : body64(h, w, nb));
    ST_CHECK_CUDA(launch_loop_test(h, LOOP_ITER, SC_RHO_NEW, true, false, hc), "stop test");
    return ST_OK;
  });
}

// The device-driven solve of pcg_impl: one graph launch (the graph is kept for the next solve with
// the same vectors), then one read of the per-problem results.
st_status pcg_device(st_handle h, const double* fhat, double* w) {
  const void* key[3] = {fhat, w, reinterpret_cast<const void*>((uintptr_t)(h->use_guess ? 1 : 0))};
  if (h->loop_exec && (h->loop_key[0] != key[0] || h->loop_key[1] != key[1] || h->loop_key[2] != key[2])) {
    cudaGraphExecDestroy(h->loop_exec);
    h->loop_exec = nullptr;
  }
  if (!h->loop_exec) {
    cudaGraph_t G = nullptr;
    ST_CHECK_CUDA(cudaGraphCreate(&G, 0), "graph create");
    std::vector<cudaGraphNode_t> leaves;
    const int64_t before = h->launches;
    st_status s = capture_pcg(h, G, leaves, fhat, w);
    h->launches = before;
    if (s == ST_OK) {
      cudaError_t e = cudaGraphInstantiate(&h->loop_exec, G, 0);
      if (e != cudaSuccess) {
        h->loop_exec = nullptr;
        s = cuda_fail("graph instantiate", e);
      }
    }
    cudaGraphDestroy(G);
    if (s != ST_OK) return s;
    for (int i = 0; i < 3; ++i) h->loop_key[i] = key[i];
  }
  ST_CHECK_CUDA(cudaGraphLaunch(h->loop_exec, h->stream), "graph launch");
  ST_CHECK(solve_collect_enqueue(h, h->stream));
  ST_CHECK_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  return solve_collect_finish(h);
}

}  // namespace

namespace st {

st_status rhs_impl(st_handle h, int nb, const double* g, const double* u0, double* fhat) {
  ST_CHECK_CUDA(launch_timemix<double>(h, nb, 1, g, h->Y), "timemix (rhs)");
  ST_CHECK_CUDA(mg_apply<double>(h, (int)(2 * nb * h->Nt), 0, h->Y, h->X), "K_x multigrid (rhs)");
  ST_CHECK_CUDA(launch_epilogue<double>(h, nb, h->X, u0, h->Nx, h->Z), "epilogue (rhs)");
  ST_CHECK_CUDA(wavelet_anal<double>(h, nb, h->Z, fhat), "wavelet analysis (rhs)");
  return ST_OK;
}

// Reads back the per-problem results of a device-driven solve (enqueued on s) ...
st_status solve_collect_enqueue(st_handle h, cudaStream_t s) {
  const int B = h->B;
  const bool refine = h->cfg.precision == ST_MIXED_FP32 || h->cfg.precision == ST_MIXED_BF16;
  ST_CHECK_CUDA(cudaMemcpyAsync(h->info_iters, h->ds.iters, sizeof(int) * B, cudaMemcpyDeviceToHost, s), "results");
  ST_CHECK_CUDA(cudaMemcpyAsync(h->info_outer, h->ds.outer, sizeof(int) * B, cudaMemcpyDeviceToHost, s), "results");
  ST_CHECK_CUDA(cudaMemcpyAsync(h->info_status, h->ds.status, sizeof(int) * B, cudaMemcpyDeviceToHost, s),
                "results");
  ST_CHECK_CUDA(cudaMemcpyAsync(h->info_relres, h->ds.relres, sizeof(double) * B, cudaMemcpyDeviceToHost, s),
                "results");
  ST_CHECK_CUDA(cudaMemcpyAsync(h->act_host, refine ? h->ds.oact : h->act, sizeof(int) * B, cudaMemcpyDeviceToHost,
                                s),
                "results");
  return ST_OK;
}

// ... and, once they have arrived, sets the overall status as the host-driven loop does.
st_status solve_collect_finish(st_handle h) { return finish(h); }

st_status capture_solve(st_handle h, cudaGraph_t G, const std::vector<cudaGraphNode_t>& deps, const double* fhat,
                        double* w, st_status (*pre)(st_handle, void*), st_status (*post)(st_handle, void*), void* arg,
                        std::vector<cudaGraphNode_t>* leaves) {
  std::vector<cudaGraphNode_t> l = deps;
  if (pre) ST_CHECK(capture_into(h, G, l, [&]() { return pre(h, arg); }));
  ST_CHECK(capture_pcg(h, G, l, fhat, w));
  if (post) ST_CHECK(capture_into(h, G, l, [&]() { return post(h, arg); }));
  *leaves = l;
  return ST_OK;
}

st_status pcg_impl(st_handle h, const double* fhat, double* w, int* iters, double* relres) {
  st_status s;
  const bool device_loop =
      h->cfg.use_graphs == 2 && reinterpret_cast<uintptr_t>(h->stream) > 2 && !h->prof_on;
  if (device_loop) {
    s = pcg_device(h, fhat, w);
    if (iters) *iters = h->last_iters;
    if (relres) *relres = h->last_relres;
    return s;
  }
  switch (h->cfg.precision) {
    case ST_MIXED_FP32:
    case ST_MIXED_BF16:
      s = pcg_mixed_impl(h, fhat, w);
      break;
    case ST_MIXED_PRECOND:
      s = pcg_precond_impl(h, fhat, w);
      break;
    default:
      s = pcg64_impl(h, fhat, w);
  }
  if (iters) *iters = h->last_iters;
  if (relres) *relres = h->last_relres;
  return s;
}

// ---------------------------------------------------------------------------------------------
// slot-level operations for continuous batching (server.cu): problem b of a batched handle
// joins, all problems advance one iteration, a finished problem leaves
// ---------------------------------------------------------------------------------------------
// Starts problem b from the inputs already in its slots of h->g and h->u0: f_hat, w = 0,
// r = f_hat, z = K_X r, p = 0, rho = rho0 = r^T z, beta = 0 (so the next body sets p = z).
st_status slot_start(st_handle_s* h, int b) {
  const int64_t V = h->Nt * h->Nx;
  ST_CHECK(rhs_impl(h, 1, h->g + b * V, h->u0 + b * h->Nx, h->fhat + b * V));
  ST_CHECK_CUDA(launch_zero<double>(h, h->w + b * V, V), "zero w");
  ST_CHECK_CUDA(launch_zero<double>(h, h->p + b * V, V), "zero p");
  ST_CHECK_CUDA(launch_copy<double, double>(h, h->r + b * V, h->fhat + b * V, V), "copy r");
  if (h->cfg.precision == ST_MIXED_PRECOND)
    ST_CHECK(precond32(h, 1, h->r + b * V, h->z + b * V, h->ri + b * V, h->zi + b * V));
  else
    ST_CHECK(apply_KX_impl<double>(h, 1, h->r + b * V, h->z + b * V));
  ST_CHECK_CUDA(launch_dot<double, double>(h, b, 1, h->r + b * V, h->z + b * V, V, SC_RHO, DOT_INIT), "dot r z");
  return ST_OK;
}

// One iteration body for problems 0 .. nb - 1 of the handle (graph-captured; a different nb
// captures again), then the scalar readback enqueued on the handle's stream (not waited for).
st_status step_enqueue(st_handle_s* h, int nb) {
  // the graph key combines the vector it writes and the problem count
  const void* key = reinterpret_cast<const char*>(h->w) + nb;
  if (h->cfg.precision == ST_MIXED_PRECOND)
    ST_CHECK(run_body(h, 2, key, [&]() { return body_precond(h, h->w, nb); }));
  else
    ST_CHECK(run_body(h, 0, key, [&]() { return body64(h, h->w, nb); }));
  ST_CHECK_CUDA(cudaMemcpyAsync(h->scal_host, h->scal, sizeof(double) * SC_COUNT * nb, cudaMemcpyDeviceToHost,
                                h->stream),
                "scalar readback");
  return ST_OK;
}

// u = W w of problem b copied to u_host (enqueued, not waited for).
st_status slot_result(st_handle_s* h, int b, double* u_host) {
  const int64_t V = h->Nt * h->Nx;
  ST_CHECK_CUDA(wavelet_synth<double>(h, 1, h->w + b * V, h->U + b * V), "wavelet synthesis");
  ST_CHECK_CUDA(cudaMemcpyAsync(u_host, h->U + b * V, sizeof(double) * V, cudaMemcpyDeviceToHost, h->stream),
                "copy result");
  return ST_OK;
}

st_status push_active(st_handle_s* h) { return push_act(h); }

}  // namespace st

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
  cfg->use_graphs = 2;
  cfg->diffusion[0] = 1.0;
  cfg->diffusion[1] = 0.0;
  cfg->diffusion[2] = 1.0;
  cfg->reaction = 0.0;
  cfg->initial_guess = 0;
}

const char* st_last_error(void) { return g_last_error.c_str(); }

st_status st_setup_batch(st_handle* out, int domain, int space_level, int time_level, int batch,
                         const st_config* cfg, void* cuda_stream) {
  ST_REQUIRE(out != nullptr, "st_setup: null output pointer");
  *out = nullptr;
  ST_REQUIRE(domain == 0 || domain == 1 || domain == 2,
             "st_setup: domain must be 0 (unit square), 1 (L-shape) or 2 (unit cube)");
  ST_REQUIRE(domain != 2 || space_level <= 8, "st_setup: the cube needs space level <= 8");
  ST_REQUIRE(space_level >= 1 && space_level <= 12, "st_setup: space level must be in 1..12");
  ST_REQUIRE(domain != 1 || space_level >= 2, "st_setup: the L-shape needs space level >= 2");
  ST_REQUIRE(time_level >= 1 && time_level <= 14, "st_setup: time level must be in 1..14");
  const int64_t nt = ((int64_t)1 << time_level) + 1;
  ST_REQUIRE(batch >= 1 && 2 * batch * nt <= 65535,
             "st_setup: batch size must be >= 1 with 2 x batch x N_t <= 65535 slices per launch");
  st_config c;
  st_default_config(&c);
  if (cfg) c = *cfg;
  ST_REQUIRE(c.n_vcycles >= 0 && c.n_vcycles <= 16 && c.n_pre >= 0 && c.n_pre <= 16 && c.n_post >= 0 &&
                 c.n_post <= 16,
             "st_setup: multigrid cycle / sweep counts must be in 0..16");
  ST_REQUIRE(c.alpha > 0.0 && std::isfinite(c.alpha), "st_setup: alpha must be positive");
  ST_REQUIRE(c.maxit >= 0 && c.tol >= 0.0 && (c.tol_mode == 0 || c.tol_mode == 1),
             "st_setup: invalid tolerance settings");
  ST_REQUIRE(c.precision == ST_FP64 || c.precision == ST_MIXED_FP32 || c.precision == ST_MIXED_PRECOND ||
                 c.precision == ST_MIXED_BF16 || c.precision == ST_FP64_DF,
             "st_setup: unsupported precision");
  ST_REQUIRE(c.inner_tol > 0.0 && c.inner_tol < 1.0 && c.inner_maxit >= 1,
             "st_setup: inner_tol must be in (0, 1) and inner_maxit >= 1");
  ST_REQUIRE(check_phys(c), "st_setup: D must be symmetric positive definite and c >= 0 (finite)");
  ST_REQUIRE(domain != 2 || (c.diffusion[0] == 1.0 && c.diffusion[1] == 0.0 && c.diffusion[2] == 1.0),
             "st_setup: the cube supports D = Id only (c >= 0 is allowed)");
  ST_REQUIRE(domain != 2 || c.precision != ST_MIXED_BF16, "st_setup: ST_MIXED_BF16 is not available on the cube");

  st_handle_s* h = new (std::nothrow) st_handle_s();
  if (!h) {
    set_error("st_setup: host allocation failed");
    return ST_ERR_NOMEM;
  }
  std::memset(h, 0, sizeof(*h));
  h->domain = domain;
  h->K = space_level;
  h->J = time_level;
  h->B = batch;
  h->n = (1 << space_level) - 1;
  h->Nx = (int64_t)h->n * h->n * (domain == 2 ? h->n : 1);
  h->Nt = nt;
  h->cfg = c;
  h->phys = Phys{c.diffusion[0], c.diffusion[1], c.diffusion[2], c.reaction};
  h->diag0 = c.diffusion[1] != 0.0 || c.reaction != 0.0;
  h->mg_df = c.precision == ST_FP64_DF;
  h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail("cudaGetDevice", e);
  }
  h->mg.K = h->K;
  h->mg.kmin = domain == 1 ? 2 : 1;  // the L-shape has no unknown on level 1
  h->mg.max_slices = (int)(2 * batch * h->Nt);

  const size_t V = (size_t)(batch * h->Nt * h->Nx);
  st_status s = ST_OK;
  struct {
    double** p;
    size_t n;
    const char* name;
  } plan[] = {{&h->U, V, "U"},
              {&h->Y, 2 * V, "Y"},
              {&h->X, 2 * V, "X"},
              {&h->Xalt, 2 * V, "Xalt"},
              {&h->Bs, 2 * V, "Bs"},
              {&h->Z, V, "Z"},
              {&h->V1, V, "V1"},
              {&h->V2, V, "V2"},
              {&h->r, V, "r"},
              {&h->p, V, "p"},
              {&h->z, V, "z"},
              {&h->q, V, "q"},
              {&h->g, V, "g"},
              {&h->fhat, V, "fhat"},
              {&h->w, V, "w"},
              {&h->u0, (size_t)(batch * h->Nx), "u0"},
              {&h->partials, (size_t)batch * kDotBlocks, "partials"},
              {&h->scal, (size_t)batch * SC_COUNT, "scalars"}};
  for (auto& a : plan)
    if (s == ST_OK) s = alloc(a.p, a.n, a.name);
  for (int k = h->mg.kmin; k < h->K && s == ST_OK; ++k) {
    const size_t nkx = (size_t)((1 << k) - 1);
    const size_t nk = nkx * nkx * (domain == 2 ? nkx : 1) * (size_t)h->mg.max_slices;
    s = alloc(&h->mg.xc[k], nk, "multigrid x");
    if (s == ST_OK) s = alloc(&h->mg.xc2[k], nk, "multigrid x (second buffer)");
    if (s == ST_OK) s = alloc(&h->mg.bc[k], nk, "multigrid b");
  }
  // binary32 vectors: the five of the inner PCG (ST_MIXED_FP32) or the preconditioner's input
  // and output (ST_MIXED_PRECOND)
  std::vector<float**> fplan;
  if (c.precision == ST_MIXED_FP32 || c.precision == ST_MIXED_BF16) fplan = {&h->xi, &h->ri, &h->pi, &h->zi, &h->qi};
  if (c.precision == ST_MIXED_PRECOND) fplan = {&h->ri, &h->zi};
  for (float** fp : fplan)
    if (s == ST_OK) s = alloc_bytes(reinterpret_cast<void**>(fp), V * sizeof(float), "binary32 vectors");
  if (s == ST_OK)
    s = alloc_bytes(reinterpret_cast<void**>(&h->coef32), sizeof(Coef<float>) * (h->J + 2) * (h->K + 1),
                    "coefficient table");
  if (s == ST_OK)
    s = alloc_bytes(reinterpret_cast<void**>(&h->coef), sizeof(Coef<double>) * (h->J + 2) * (h->K + 1),
                    "coefficient table");
  if (s == ST_OK && h->mg_df)
    s = alloc_bytes(reinterpret_cast<void**>(&h->coefdf), sizeof(Coef<df64>) * (h->J + 2) * (h->K + 1),
                    "coefficient table");
  if (s == ST_OK) s = alloc_bytes(reinterpret_cast<void**>(&h->act), sizeof(int) * batch, "active flags");
  if (s == ST_OK) {
    // device loop state: 2 B doubles, then 4 counters and 5 B ints
    s = alloc_bytes(&h->ds_mem, sizeof(double) * 2 * batch + sizeof(int) * (4 + 5 * (size_t)batch), "loop state");
    if (s == ST_OK) {
      double* d = static_cast<double*>(h->ds_mem);
      h->ds.relres = d;
      h->ds.rho0 = d + batch;
      int* i = reinterpret_cast<int*>(d + 2 * batch);
      h->ds.ctr = i;
      h->ds.iters = i + 4;
      h->ds.outer = i + 4 + batch;
      h->ds.status = i + 4 + 2 * batch;
      h->ds.oact = i + 4 + 3 * batch;
      h->ds.its = i + 4 + 4 * batch;
    }
  }
  if (s == ST_OK) {
    e = cudaMallocHost(reinterpret_cast<void**>(&h->scal_host), sizeof(double) * SC_COUNT * batch);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->act_host), sizeof(int) * batch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMallocHost of the scalar mirrors failed");
      s = ST_ERR_NOMEM;
    }
  }
  if (s == ST_OK) {
    h->info_iters = static_cast<int*>(std::calloc(batch, sizeof(int)));
    h->info_outer = static_cast<int*>(std::calloc(batch, sizeof(int)));
    h->info_status = static_cast<int*>(std::calloc(batch, sizeof(int)));
    h->info_relres = static_cast<double*>(std::calloc(batch, sizeof(double)));
    if (!h->info_iters || !h->info_outer || !h->info_status || !h->info_relres) {
      set_error("st_setup: host allocation failed");
      s = ST_ERR_NOMEM;
    }
  }
  if (s == ST_OK) {
    e = mg_set_attributes();
    const int dim = domain == 2 ? 3 : 2;
    if (e == cudaSuccess) e = launch_make_coef(h->coef, h->K, h->J, c.alpha, h->phys, dim, h->stream);
    if (e == cudaSuccess) e = launch_make_coef32(h->coef32, h->K, h->J, c.alpha, h->phys, dim, h->stream);
    if (e == cudaSuccess && h->mg_df)
      e = launch_make_coef_df(h->coefdf, h->K, h->J, c.alpha, h->phys, dim, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->scal, 0, sizeof(double) * SC_COUNT * batch, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) s = cuda_fail("st_setup", e);
  }
  if (s != ST_OK) {
    free_all(h);
    delete h;
    return s;
  }
  // default Gauss-Seidel kernels: binary32 on the levels that hold a wide register region (the
  // autotuner's usual choice there), the shared-memory tiles everywhere else; all give the same
  // bits, so this only sets the speed of handles that are not autotuned (batches, the server)
  for (int k = 1; k <= h->K && k < 16; ++k)
    if (wide_fits(h, 0, k)) h->gs_kind[1][0][k] = h->gs_kind[1][1][k] = (unsigned char)(2 + 3);
  *out = h;
  return ST_OK;
}

st_status st_setup(st_handle* out, int domain, int space_level, int time_level, const st_config* cfg,
                   void* cuda_stream) {
  return st_setup_batch(out, domain, space_level, time_level, 1, cfg, cuda_stream);
}

st_status st_destroy(st_handle h) {
  if (!h) return ST_OK;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  for (int m = 0; m < 16; ++m)
    if (h->nest[m]) st_destroy(h->nest[m]);
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

st_status st_batch_size(st_handle h, int* B) {
  ST_REQUIRE(h != nullptr && B != nullptr, "st_batch_size: null pointer");
  *B = h->B;
  return ST_OK;
}

st_status st_apply_Kx(st_handle h, int nslices, const double* b, double* x) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(b && x, "st_apply_Kx: null pointer");
  ST_REQUIRE(nslices >= 1 && nslices <= 2 * h->B * h->Nt, "st_apply_Kx: nslices must be in 1..2 B N_t");
  ST_CHECK_CUDA(mg_apply<double>(h, nslices, 0, b, x), "K_x multigrid");
  return ST_OK;
}

st_status st_apply_S_nodal(st_handle h, const double* u, double* y) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(u && y, "st_apply_S_nodal: null pointer");
  return apply_S_nodal_impl<double>(h, h->B, u, y);
}

st_status st_synthesize(st_handle h, const double* w, double* u) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(w && u, "st_synthesize: null pointer");
  ST_CHECK_CUDA(wavelet_synth<double>(h, h->B, w, u), "wavelet synthesis");
  return ST_OK;
}

st_status st_analyze(st_handle h, const double* u, double* w) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(w && u, "st_analyze: null pointer");
  ST_CHECK_CUDA(wavelet_anal<double>(h, h->B, u, w), "wavelet analysis");
  return ST_OK;
}

st_status st_apply_S(st_handle h, const double* w, double* q) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(w && q, "st_apply_S: null pointer");
  return apply_Shat_impl<double>(h, h->B, w, q);
}

st_status st_apply_S_f32(st_handle h, const float* w, float* q) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(w && q, "st_apply_S_f32: null pointer");
  return apply_Shat_impl<float>(h, h->B, w, q);
}

st_status st_apply_KX_f32(st_handle h, const float* r, float* z) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(r && z, "st_apply_KX_f32: null pointer");
  return apply_KX_impl<float>(h, h->B, r, z);
}

st_status st_apply_KX_bf16(st_handle h, const float* r, float* z) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(r && z, "st_apply_KX_bf16: null pointer");
  ST_REQUIRE(h->domain != 2, "st_apply_KX_bf16: not available on the cube");
  return apply_KX_impl<float>(h, h->B, r, z, true);
}

st_status st_apply_KX(st_handle h, const double* r, double* z) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(r && z, "st_apply_KX: null pointer");
  return apply_KX_impl<double>(h, h->B, r, z);
}

st_status st_rhs(st_handle h, const double* g, const double* u0, double* fhat) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(g && u0 && fhat, "st_rhs: null pointer");
  return rhs_impl(h, h->B, g, u0, fhat);
}

st_status st_pcg_solve(st_handle h, const double* fhat, double* w, int* iters, double* relres) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(fhat && w, "st_pcg_solve: null pointer");
  h->use_guess = h->cfg.initial_guess != 0;
  const st_status s = pcg_impl(h, fhat, w, iters, relres);
  h->use_guess = false;
  return s;
}

st_status st_solve_info_get(st_handle h, st_solve_info* out) {
  ST_REQUIRE(h != nullptr && out != nullptr, "st_solve_info_get: null pointer");
  out->iterations = h->last_iters;
  out->outer_iterations = h->last_outer;
  out->relres = h->last_relres;
  return ST_OK;
}

st_status st_problem_info(st_handle h, int b, st_solve_info* out, int* status) {
  ST_REQUIRE(h != nullptr && out != nullptr, "st_problem_info: null pointer");
  ST_REQUIRE(b >= 0 && b < h->B, "st_problem_info: problem index out of range");
  out->iterations = h->info_iters[b];
  out->outer_iterations = h->info_outer[b];
  out->relres = h->info_relres[b];
  if (status) *status = h->info_status[b];
  return ST_OK;
}

st_status st_solve_host(st_handle h, const double* g_host, const double* u0_host, double* u_host, int* iters,
                        double* relres) {
  ST_CHECK(check_handle(h));
  ST_REQUIRE(g_host && u0_host && u_host, "st_solve_host: null pointer");
  const size_t V = (size_t)(h->B * h->Nt * h->Nx);
  ST_CHECK_CUDA(cudaMemcpyAsync(h->g, g_host, V * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy g");
  ST_CHECK_CUDA(cudaMemcpyAsync(h->u0, u0_host, (size_t)(h->B * h->Nx) * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream),
                "copy u0");
  ST_CHECK(rhs_impl(h, h->B, h->g, h->u0, h->fhat));
  st_status ps = pcg_impl(h, h->fhat, h->w, iters, relres);
  if (ps != ST_OK && ps != ST_ERR_MAXIT) return ps;
  ST_CHECK_CUDA(wavelet_synth<double>(h, h->B, h->w, h->g), "wavelet synthesis");
  ST_CHECK_CUDA(cudaMemcpyAsync(u_host, h->g, V * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy u");
  ST_CHECK_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  return ps;
}

st_status st_autotune(st_handle h, float* times_ms) {
  ST_CHECK(check_handle(h));
  float table[12 * 16] = {0};
  ST_CHECK_CUDA(mg_autotune(h, table), "autotune");
  drop_graphs(h);  // graphs captured with the old choices are stale
  if (times_ms) std::memcpy(times_ms, table, sizeof(table));
  return ST_OK;
}

st_status st_set_wave_rows(st_handle h, int rows) {
  ST_CHECK(check_handle(h));
  if (rows < 0 || rows > 65535) {
    set_error("st_set_wave_rows: rows must be in 0 .. 65535");
    return ST_ERR_ARG;
  }
  for (auto& a : h->gs_seg)
    for (auto& b : a)
      for (auto& c : b) c = (unsigned short)rows;
  drop_graphs(h);
  return ST_OK;
}

st_status st_set_smoother(st_handle h, int kind) {
  ST_CHECK(check_handle(h));
  if (kind < 0 || kind > 1 + kRegShapes) {
    set_error("st_set_smoother: kind must be 0 (shared-memory tiles), 1 (wavefront) or 2..5 (register tiles of "
              "block shape 0..3)");
    return ST_ERR_ARG;
  }
  std::memset(h->gs_kind, kind, sizeof(h->gs_kind));
  drop_graphs(h);
  return ST_OK;
}

st_status st_profile_begin(st_handle h) {
  ST_CHECK(check_handle(h));
  h->launches = 0;
  h->prof_n = 0;
  for (int c = 0; c < 4; ++c) h->prof_ops[c] = h->prof_bytes[c] = 0.0;
  h->prof_on = true;
  // preallocate events so that recording inside the timed region never creates them
  if (h->prof_cap < 16384 && prof_start(h)) {
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
  ST_CHECK(check_handle(h));
  ST_REQUIRE(out != nullptr, "st_profile_end: null output");
  ST_CHECK_CUDA(cudaStreamSynchronize(h->stream), "st_profile_end");
  double ms[4] = {0.0, 0.0, 0.0, 0.0};
  int64_t n[4] = {0, 0, 0, 0};
  for (int i = 0; i + 1 < h->prof_n; i += 2) {
    float t = 0.f;
    ST_CHECK_CUDA(cudaEventElapsedTime(&t, h->prof_ev[i], h->prof_ev[i + 1]), "cudaEventElapsedTime");
    ms[h->prof_cat[i]] += t;
    n[h->prof_cat[i]] += 1;
  }
  out->launches = h->launches;
  out->sweep_launches = n[0] + n[1];
  out->sweep_ms = ms[0] + ms[1];
  out->sweep_fp64_ops = h->prof_ops[0] + h->prof_ops[1];
  out->sweep_bytes = h->prof_bytes[0] + h->prof_bytes[1];
  out->diag_launches = n[1];
  out->diag_ms = ms[1];
  out->diag_fp64_ops = h->prof_ops[1];
  out->diag_bytes = h->prof_bytes[1];
  out->f32_launches = n[2] + n[3];
  out->f32_ms = ms[2] + ms[3];
  out->f32_bytes = h->prof_bytes[2] + h->prof_bytes[3];
  out->f32_diag_launches = n[3];
  out->f32_diag_ms = ms[3];
  out->f32_diag_bytes = h->prof_bytes[3];
  h->prof_on = false;
  h->prof_n = 0;
  return ST_OK;
}

}  // extern "C"
