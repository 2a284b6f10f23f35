// st_batch_*: many independent heat-equation solves of different shapes in one call.
//
// Problems are grouped by (domain, space level, time level); every group ("bucket") becomes one
// batched handle whose launches cover all of its problems at once.  Inside a bucket each problem
// keeps its own PCG scalars and stop test, and its result is bitwise the result of solving it
// alone.  With cfg.use_graphs = 2 (the default) all buckets run as the branches of one CUDA graph,
// launched once: each branch's PCG loop is a WHILE node driven by device-side stop tests, so the
// whole batch iterates on the GPU without host round trips.  Otherwise the buckets run
// concurrently from host threads (one per bucket and stream), each with a host-driven PCG loop
// (with cfg.use_graphs = 1 its iteration body is captured once as a CUDA graph and replayed).
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "st_internal.cuh"

namespace {

struct Problem {
  int domain, K, J;
  const double* g;   // host, N_t x N_x
  const double* u0;  // host, N_x
  double* u;         // host, N_t x N_x
  st_solve_info info;
  int status;
};

}  // namespace

struct st_batch_s {
  st_config cfg;
  int device;
  std::vector<Problem> probs;
  int buckets_last_run;
};

using namespace st;

namespace {

struct Bucket {
  int domain, K, J;
  std::vector<int> ids;  // problem ids, in slot order
  st_handle h = nullptr;
  cudaStream_t stream = nullptr;
  st_status status = ST_OK;
  std::string error;
};

// Solves one bucket: copy inputs into the handle, right-hand side, PCG, synthesis, copy out.
void run_bucket(st_batch_s* b, Bucket& bk) {
  cudaSetDevice(b->device);
  st_handle h = bk.h;
  const int64_t Nt = h->Nt, Nx = h->Nx;
  auto fail = [&](st_status s, const char* where, cudaError_t e) {
    bk.status = s;
    bk.error = std::string(where) + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string());
  };
  for (size_t i = 0; i < bk.ids.size(); ++i) {
    const Problem& p = b->probs[bk.ids[i]];
    cudaError_t e = cudaMemcpyAsync(h->g + i * Nt * Nx, p.g, sizeof(double) * Nt * Nx, cudaMemcpyHostToDevice,
                                    bk.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->u0 + i * Nx, p.u0, sizeof(double) * Nx, cudaMemcpyHostToDevice, bk.stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, "copy inputs", e);
  }
  st_status s = rhs_impl(h, h->B, h->g, h->u0, h->fhat);
  if (s != ST_OK) return fail(s, st_last_error(), cudaSuccess);
  st_status ps = pcg_impl(h, h->fhat, h->w, nullptr, nullptr);
  if (ps != ST_OK && ps != ST_ERR_MAXIT && ps != ST_ERR_BREAKDOWN) return fail(ps, st_last_error(), cudaSuccess);
  cudaError_t e = wavelet_synth<double>(h, h->B, h->w, h->g);
  if (e != cudaSuccess) return fail(ST_ERR_CUDA, "wavelet synthesis", e);
  for (size_t i = 0; i < bk.ids.size(); ++i) {
    Problem& p = b->probs[bk.ids[i]];
    e = cudaMemcpyAsync(p.u, h->g + i * Nt * Nx, sizeof(double) * Nt * Nx, cudaMemcpyDeviceToHost, bk.stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, "copy result", e);
    st_problem_info(h, (int)i, &p.info, &p.status);
  }
  e = cudaStreamSynchronize(bk.stream);
  if (e != cudaSuccess) return fail(ST_ERR_CUDA, "stream synchronize", e);
}

// Right-hand sides before the PCG and syntheses after it, as steps of the batch graph.
st_status batch_pre(st_handle h, void*) { return rhs_impl(h, h->B, h->g, h->u0, h->fhat); }
st_status batch_post(st_handle h, void*) {
  cudaError_t e = wavelet_synth<double>(h, h->B, h->w, h->g);
  return e == cudaSuccess ? ST_OK : cuda_fail("wavelet synthesis", e);
}

// Every bucket in one CUDA graph: each bucket is a branch (right-hand side, the device-driven
// PCG of capture_solve, synthesis) independent of the others, so the GPU runs the buckets
// concurrently and each iterates until its own problems stop, with no host round trip until the
// whole batch is done.  The host copies inputs in before the launch and results out after it.
st_status run_buckets_graph(st_batch_s* b, std::vector<Bucket>& buckets) {
  cudaStream_t ls = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail("cudaStreamCreate", e);
  cudaGraph_t G = nullptr;
  cudaGraphExec_t X = nullptr;
  st_status s = ST_OK;
  auto ck = [&](cudaError_t err, const char* where) {
    if (err != cudaSuccess && s == ST_OK) s = cuda_fail(where, err);
    return s == ST_OK;
  };
  for (Bucket& bk : buckets) {
    st_handle h = bk.h;
    const int64_t Nt = h->Nt, Nx = h->Nx;
    for (size_t i = 0; i < bk.ids.size() && s == ST_OK; ++i) {
      const Problem& p = b->probs[bk.ids[i]];
      ck(cudaMemcpyAsync(h->g + i * Nt * Nx, p.g, sizeof(double) * Nt * Nx, cudaMemcpyHostToDevice, ls), "copy g");
      ck(cudaMemcpyAsync(h->u0 + i * Nx, p.u0, sizeof(double) * Nx, cudaMemcpyHostToDevice, ls), "copy u0");
    }
  }
  if (ck(cudaGraphCreate(&G, 0), "graph create")) {
    for (Bucket& bk : buckets) {
      std::vector<cudaGraphNode_t> leaves;
      s = capture_solve(bk.h, G, {}, bk.h->fhat, bk.h->w, batch_pre, batch_post, nullptr, &leaves);
      if (s != ST_OK) break;
    }
  }
  if (s == ST_OK && ck(cudaGraphInstantiate(&X, G, 0), "graph instantiate")) ck(cudaGraphLaunch(X, ls), "graph launch");
  for (Bucket& bk : buckets) {
    st_handle h = bk.h;
    const int64_t Nt = h->Nt, Nx = h->Nx;
    for (size_t i = 0; i < bk.ids.size() && s == ST_OK; ++i)
      ck(cudaMemcpyAsync(b->probs[bk.ids[i]].u, h->g + i * Nt * Nx, sizeof(double) * Nt * Nx, cudaMemcpyDeviceToHost,
                         ls),
         "copy result");
    if (s == ST_OK) s = solve_collect_enqueue(h, ls);
  }
  if (s == ST_OK) ck(cudaStreamSynchronize(ls), "stream synchronize");
  for (Bucket& bk : buckets) {
    if (s != ST_OK) break;
    const st_status fs = solve_collect_finish(bk.h);
    if (fs != ST_OK && fs != ST_ERR_MAXIT && fs != ST_ERR_BREAKDOWN) s = fs;
    for (size_t i = 0; i < bk.ids.size(); ++i) {
      Problem& p = b->probs[bk.ids[i]];
      st_problem_info(bk.h, (int)i, &p.info, &p.status);
    }
  }
  if (X) cudaGraphExecDestroy(X);
  if (G) cudaGraphDestroy(G);
  cudaStreamSynchronize(ls);
  cudaStreamDestroy(ls);
  return s;
}

}  // namespace

extern "C" {

st_status st_batch_create(st_batch* out, const st_config* cfg) {
  if (!out) {
    set_error("st_batch_create: null output pointer");
    return ST_ERR_ARG;
  }
  st_batch_s* b = new (std::nothrow) st_batch_s();
  if (!b) {
    set_error("st_batch_create: host allocation failed");
    return ST_ERR_NOMEM;
  }
  st_default_config(&b->cfg);
  if (cfg) b->cfg = *cfg;
  b->buckets_last_run = 0;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail("cudaGetDevice", e);
  }
  *out = b;
  return ST_OK;
}

st_status st_batch_add(st_batch b, int domain, int space_level, int time_level, const double* g_host,
                       const double* u0_host, double* u_host, int* id) {
  if (!b || !g_host || !u0_host || !u_host) {
    set_error("st_batch_add: null pointer");
    return ST_ERR_ARG;
  }
  if ((domain != 0 && domain != 1 && domain != 2) || space_level < 1 || space_level > 12 ||
      (domain == 1 && space_level < 2) || (domain == 2 && space_level > 8) || time_level < 1 || time_level > 14) {
    set_error("st_batch_add: invalid domain or levels");
    return ST_ERR_ARG;
  }
  Problem p;
  std::memset(&p, 0, sizeof(p));
  p.domain = domain;
  p.K = space_level;
  p.J = time_level;
  p.g = g_host;
  p.u0 = u0_host;
  p.u = u_host;
  b->probs.push_back(p);
  if (id) *id = (int)b->probs.size() - 1;
  return ST_OK;
}

st_status st_batch_run(st_batch b) {
  if (!b) {
    set_error("st_batch_run: null batch");
    return ST_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
  // group by shape; split a group so that one launch covers at most 65535 slices (2 B N_t)
  std::map<std::tuple<int, int, int>, std::vector<int>> groups;
  for (size_t i = 0; i < b->probs.size(); ++i) {
    const Problem& p = b->probs[i];
    groups[std::make_tuple(p.domain, p.K, p.J)].push_back((int)i);
  }
  std::vector<Bucket> buckets;
  for (auto& kv : groups) {
    const int J = std::get<2>(kv.first);
    const int cap = (int)(65535 / (2 * ((1 << J) + 1)));
    for (size_t s = 0; s < kv.second.size(); s += cap) {
      Bucket bk;
      bk.domain = std::get<0>(kv.first);
      bk.K = std::get<1>(kv.first);
      bk.J = J;
      bk.ids.assign(kv.second.begin() + s, kv.second.begin() + std::min(kv.second.size(), s + cap));
      buckets.push_back(bk);
    }
  }
  st_status s = ST_OK;
  for (Bucket& bk : buckets) {
    e = cudaStreamCreateWithFlags(&bk.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      s = cuda_fail("cudaStreamCreate", e);
      break;
    }
    s = st_setup_batch(&bk.h, bk.domain, bk.K, bk.J, (int)bk.ids.size(), &b->cfg, bk.stream);
    if (s != ST_OK) break;
  }
  if (s == ST_OK && b->cfg.use_graphs == 2) {
    s = run_buckets_graph(b, buckets);
  } else if (s == ST_OK) {
    std::vector<std::thread> threads;
    for (Bucket& bk : buckets) threads.emplace_back(run_bucket, b, std::ref(bk));
    for (auto& t : threads) t.join();
    for (Bucket& bk : buckets)
      if (bk.status != ST_OK && s == ST_OK) {
        s = bk.status;
        set_error("st_batch_run: " + bk.error);
      }
  }
  for (Bucket& bk : buckets) {
    if (bk.h) st_destroy(bk.h);
    if (bk.stream) cudaStreamDestroy(bk.stream);
  }
  b->buckets_last_run = (int)buckets.size();
  if (s != ST_OK) return s;
  for (const Problem& p : b->probs)
    if (p.status != ST_OK) {
      set_error("st_batch_run: some problem did not converge (see st_batch_problem_info)");
      return (st_status)p.status;
    }
  return ST_OK;
}

st_status st_batch_problem_info(st_batch b, int id, st_solve_info* out, int* status) {
  if (!b || !out || id < 0 || id >= (int)b->probs.size()) {
    set_error("st_batch_problem_info: invalid argument");
    return ST_ERR_ARG;
  }
  *out = b->probs[id].info;
  if (status) *status = b->probs[id].status;
  return ST_OK;
}

st_status st_batch_buckets(st_batch b, int* n) {
  if (!b || !n) {
    set_error("st_batch_buckets: null pointer");
    return ST_ERR_ARG;
  }
  *n = b->buckets_last_run;
  return ST_OK;
}

st_status st_batch_destroy(st_batch b) {
  delete b;
  return ST_OK;
}

}  // extern "C"
