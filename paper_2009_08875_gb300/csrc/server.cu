// st_server_*: a continuous-batching solve server.
//
// Requests (one heat-equation solve each, any domain / space level / time level) are queued by
// st_server_submit and served by one worker thread.  Problems of one shape share a "group": a
// batched handle with a fixed number of slots whose CG state (w, r, p, z, q and the scalars)
// stays resident on the GPU.  Every round the worker
//   1. admits queued requests into free slots of their shape's group, creating a group when the
//      device-memory budget allows (idle groups of other shapes are released to make room);
//   2. starts the admitted problems (copy inputs, right-hand side, r, z, rho0 for that slot);
//   3. advances every group with an active slot by one PCG iteration (a CUDA graph, each group on
//      its own stream, all groups enqueued before any is waited for);
//   4. tests every active slot, and for each finished one synthesises u, copies it to the
//      caller's buffer and frees the slot.
// So requests join and leave at iteration boundaries while others are on the GPU, and each
// request's arithmetic is exactly that of solving it alone (its slot sees only its own data).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "st_internal.cuh"

using namespace st;

namespace {

using Clock = std::chrono::steady_clock;

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };

struct Request {
  int64_t ticket;
  int domain, K, J;
  const double* g;
  const double* u0;
  double* u;
  Clock::time_point submitted, started, finished;
  Clock::time_point deadline;  // meaningful if has_deadline
  bool has_deadline = false;
  bool cancel = false;         // set by st_server_cancel (under the server mutex)
  int state = REQ_QUEUED;
  st_solve_info info{};
  int status = ST_OK;
};

struct Group {
  int domain, K, J, slots;
  st_handle h = nullptr;
  cudaStream_t stream = nullptr;
  size_t bytes = 0;
  std::vector<Request*> slot;  // nullptr = free
  std::vector<int> joining;    // slots started this round
  Clock::time_point last_used;
  cudaEvent_t done = nullptr;  // recorded after the scalar readback of the iteration in flight
  bool in_flight = false;
};

// Device bytes of a group (the allocation plan of st_setup_batch, rounded up).
size_t group_bytes(int domain, int K, int J, int slots, int precision) {
  const int dim = domain == 2 ? 3 : 2;
  const double n = (double)((1 << K) - 1);
  const double Nt = (double)((1 << J) + 1);
  const double V = slots * Nt * std::pow(n, dim);
  double coarse = 0.0;
  for (int k = 1; k < K; ++k) coarse += 3.0 * 2.0 * slots * Nt * std::pow((double)((1 << k) - 1), dim);
  double floats = precision == ST_MIXED_PRECOND ? 2.0
                  : ((precision == ST_MIXED_FP32 || precision == ST_MIXED_BF16) ? 5.0 : 0.0);
  return (size_t)(8.0 * (26.0 * V + coarse) + 4.0 * floats * V + 64.0 * 1024 * 1024);
}

}  // namespace

struct st_server_s {
  st_config cfg;
  int device;
  int slots_per_group;
  size_t budget;
  size_t allocated = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;                    // submitted, not yet admitted
  std::vector<std::unique_ptr<Request>> all;     // every request, index = ticket
  std::vector<std::unique_ptr<Group>> groups;
  bool stopping = false;
  st_status error = ST_OK;
  std::string error_msg;
  std::thread worker;
  int64_t rounds = 0;
};

namespace {

int slots_for(st_server_s* s, int domain, int K, int J) {
  const int nt = (1 << J) + 1;
  int c = std::min(s->slots_per_group, 65535 / (2 * nt));
  // a group may use at most a quarter of the budget
  while (c > 1 && group_bytes(domain, K, J, c, s->cfg.precision) > s->budget / 4) c /= 2;
  return std::max(c, 1);
}

Group* find_group(st_server_s* s, const Request* r) {
  for (auto& g : s->groups)
    if (g->domain == r->domain && g->K == r->K && g->J == r->J)
      for (Request* q : g->slot)
        if (!q) return g.get();
  return nullptr;
}

bool group_idle(const Group* g) {
  if (g->in_flight) return false;
  for (Request* q : g->slot)
    if (q) return false;
  return true;
}

void release_group(st_server_s* s, size_t i) {
  Group* g = s->groups[i].get();
  st_destroy(g->h);
  if (g->done) cudaEventDestroy(g->done);
  cudaStreamDestroy(g->stream);
  s->allocated -= g->bytes;
  s->groups.erase(s->groups.begin() + i);
}

// Creates a group for r's shape if the budget allows, releasing idle groups (least recently
// used first) to make room.  Returns nullptr if it cannot be made now.
Group* make_group(st_server_s* s, const Request* r) {
  const int slots = slots_for(s, r->domain, r->K, r->J);
  const size_t need = group_bytes(r->domain, r->K, r->J, slots, s->cfg.precision);
  while (s->allocated + need > s->budget) {
    size_t victim = s->groups.size();
    for (size_t i = 0; i < s->groups.size(); ++i)
      if (group_idle(s->groups[i].get()) &&
          (victim == s->groups.size() || s->groups[i]->last_used < s->groups[victim]->last_used))
        victim = i;
    if (victim == s->groups.size()) return nullptr;
    release_group(s, victim);
  }
  auto g = std::make_unique<Group>();
  g->domain = r->domain;
  g->K = r->K;
  g->J = r->J;
  g->slots = slots;
  g->slot.assign(slots, nullptr);
  g->last_used = Clock::now();
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(g->stream);
    return nullptr;
  }
  if (st_setup_batch(&g->h, r->domain, r->K, r->J, slots, &s->cfg, g->stream) != ST_OK) {
    cudaEventDestroy(g->done);
    cudaStreamDestroy(g->stream);
    return nullptr;
  }
  for (int b = 0; b < slots; ++b) g->h->act_host[b] = 0;
  g->bytes = need;
  s->allocated += need;
  s->groups.push_back(std::move(g));
  return s->groups.back().get();
}

void fail_server(st_server_s* s, st_status st, const std::string& where) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->error == ST_OK) {
    s->error = st;
    s->error_msg = where + ": " + st_last_error();
  }
}

void finish_request(Request* r, int state) {
  r->finished = Clock::now();
  r->state = state;
}

void worker_loop(st_server_s* s) {
  cudaSetDevice(s->device);
  std::deque<Request*> waiting;  // admitted by the worker in arrival order
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool busy = !waiting.empty();
      for (auto& g : s->groups) busy = busy || !group_idle(g.get());
      if (!busy) s->cv.wait(lk, [&] { return s->stopping || !s->queue.empty(); });
      while (!s->queue.empty()) {
        waiting.push_back(s->queue.front());
        s->queue.pop_front();
      }
      // requests not yet started that were cancelled or are past their deadline
      const Clock::time_point now = Clock::now();
      for (auto it = waiting.begin(); it != waiting.end();) {
        Request* r = *it;
        if (r->cancel || (r->has_deadline && now >= r->deadline)) {
          r->status = r->cancel ? ST_ERR_CANCELLED : ST_ERR_TIMEOUT;
          finish_request(r, REQ_FAILED);
          it = waiting.erase(it);
        } else {
          ++it;
        }
      }
      busy = !waiting.empty();
      for (auto& g : s->groups) busy = busy || !group_idle(g.get());
      if (s->stopping && !busy) return;
      if (s->error != ST_OK) return;
    }
    // 1-2. admission and start of the admitted problems
    bool admitted = false;
    for (auto it = waiting.begin(); it != waiting.end();) {
      Request* r = *it;
      Group* g = find_group(s, r);
      if (!g) g = make_group(s, r);
      if (!g) {
        bool any_busy = false;
        for (auto& gp : s->groups) any_busy = any_busy || !group_idle(gp.get());
        if (!any_busy && s->allocated == 0) {  // it cannot fit even in an empty device budget
          std::lock_guard<std::mutex> lk(s->mu);
          r->status = ST_ERR_NOMEM;
          finish_request(r, REQ_FAILED);
          it = waiting.erase(it);
          continue;
        }
        ++it;  // no room now: try again next round
        continue;
      }
      if (g->in_flight) {  // joins when the group's current iteration has completed
        ++it;
        continue;
      }
      int b = 0;
      while (g->slot[b]) ++b;
      st_handle h = g->h;
      const int64_t V = h->Nt * h->Nx;
      cudaError_t e = cudaMemcpyAsync(h->g + b * V, r->g, sizeof(double) * V, cudaMemcpyHostToDevice, g->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->u0 + b * h->Nx, r->u0, sizeof(double) * h->Nx, cudaMemcpyHostToDevice, g->stream);
      if (e != cudaSuccess) return fail_server(s, cuda_fail("copy inputs", e), "admission");
      st_status st = slot_start(h, b);
      if (st != ST_OK) return fail_server(s, st, "slot start");
      g->slot[b] = r;
      g->joining.push_back(b);
      h->act_host[b] = 1;
      h->info_iters[b] = 0;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        r->started = Clock::now();
        r->state = REQ_RUNNING;
      }
      admitted = true;
      it = waiting.erase(it);
    }
    // 3. an iteration on every group that has occupied slots and none in flight; groups run
    // independently on their own streams, so a large problem does not hold back small ones
    bool progressed = admitted;
    for (auto& gp : s->groups) {
      Group* g = gp.get();
      if (g->in_flight) continue;
      bool occupied = false;
      for (Request* q : g->slot) occupied = occupied || q != nullptr;
      if (!occupied) continue;
      if (!g->joining.empty()) {
        st_status st = push_active(g->h);
        if (st != ST_OK) return fail_server(s, st, "active flags");
        g->joining.clear();
      }
      // only the occupied prefix of the slots is computed (free slots cost nothing)
      int nb = g->slots;
      while (nb > 0 && !g->slot[nb - 1]) --nb;
      st_status st = step_enqueue(g->h, nb);
      if (st != ST_OK) return fail_server(s, st, "iteration");
      cudaError_t e = cudaEventRecord(g->done, g->stream);
      if (e != cudaSuccess) return fail_server(s, cuda_fail("event record", e), "iteration");
      g->in_flight = true;
      g->last_used = Clock::now();
      progressed = true;
    }
    // 4. stop tests and results of every group whose iteration has completed
    for (auto& gp : s->groups) {
      Group* g = gp.get();
      if (!g->in_flight) continue;
      cudaError_t e = cudaEventQuery(g->done);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) return fail_server(s, cuda_fail("iteration", e), "iteration");
      g->in_flight = false;
      progressed = true;
      st_handle h = g->h;
      bool changed = false;
      std::vector<int> done;
      std::vector<char> stop(g->slots, 0);  // 1 cancelled, 2 past the deadline
      {
        std::lock_guard<std::mutex> lk(s->mu);
        const Clock::time_point now = Clock::now();
        for (int b = 0; b < g->slots; ++b)
          if (g->slot[b]) stop[b] = g->slot[b]->cancel ? 1 : ((g->slot[b]->has_deadline && now >= g->slot[b]->deadline) ? 2 : 0);
      }
      for (int b = 0; b < g->slots; ++b) {
        Request* r = g->slot[b];
        if (!r) continue;
        const double* sc = h->scal_host + (size_t)b * SC_COUNT;
        const int it = ++h->info_iters[b];
        if (stop[b]) {  // leaves at this iteration boundary without a result
          r->info.iterations = it;
          r->status = stop[b] == 1 ? ST_ERR_CANCELLED : ST_ERR_TIMEOUT;
          h->act_host[b] = 0;
          changed = true;
          done.push_back(b);
          continue;
        }
        const double rho0 = sc[SC_RHO0], rho = sc[SC_RHO_NEW], pq = sc[SC_PQ];
        int status = ST_OK;
        bool fin = false;
        if (!(rho0 >= 0.0) || !std::isfinite(rho0)) {
          status = ST_ERR_BREAKDOWN;
          fin = true;
        } else if (rho0 == 0.0) {
          fin = true;  // zero right-hand side: w = 0 is the solution
        } else if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rho) || rho < 0.0) {
          status = ST_ERR_BREAKDOWN;
          fin = true;
        } else {
          const double rr = std::sqrt(rho / rho0);
          r->info.relres = rr;
          const bool conv = s->cfg.tol_mode == 1 ? std::sqrt(rho) <= s->cfg.tol : rr <= s->cfg.tol;
          if (conv) fin = true;
          if (!conv && it >= s->cfg.maxit) {
            status = ST_ERR_MAXIT;
            fin = true;
          }
        }
        if (!fin) continue;
        r->info.iterations = (rho0 == 0.0) ? 0 : it;
        r->status = status;
        st_status st = slot_result(h, b, r->u);
        if (st != ST_OK) return fail_server(s, st, "result");
        h->act_host[b] = 0;
        changed = true;
        done.push_back(b);
      }
      if (!done.empty()) {
        e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return fail_server(s, cuda_fail("stream synchronize", e), "result");
        std::lock_guard<std::mutex> lk(s->mu);
        for (int b : done) {
          Request* r = g->slot[b];
          finish_request(r, r->status == ST_OK ? REQ_DONE : REQ_FAILED);
          g->slot[b] = nullptr;
        }
      }
      if (changed) {
        st_status st = push_active(h);
        if (st != ST_OK) return fail_server(s, st, "active flags");
      }
    }
    ++s->rounds;
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

st_status st_server_start(st_server* out, const st_config* cfg, int slots_per_group, double memory_budget_gb) {
  if (!out) {
    set_error("st_server_start: null output pointer");
    return ST_ERR_ARG;
  }
  *out = nullptr;
  st_config c;
  st_default_config(&c);
  if (cfg) c = *cfg;
  if (c.precision != ST_FP64 && c.precision != ST_MIXED_PRECOND) {
    set_error("st_server_start: the server runs ST_FP64 or ST_MIXED_PRECOND (single-phase iterations)");
    return ST_ERR_ARG;
  }
  if (slots_per_group < 1 || !(memory_budget_gb > 0.0)) {
    set_error("st_server_start: slots_per_group must be >= 1 and the memory budget positive");
    return ST_ERR_ARG;
  }
  st_server_s* s = new (std::nothrow) st_server_s();
  if (!s) {
    set_error("st_server_start: host allocation failed");
    return ST_ERR_NOMEM;
  }
  s->cfg = c;
  s->slots_per_group = slots_per_group;
  s->budget = (size_t)(memory_budget_gb * 1e9);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail("cudaGetDevice", e);
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return ST_OK;
}

st_status st_server_submit_deadline(st_server s, int domain, int space_level, int time_level, const double* g_host,
                                    const double* u0_host, double* u_host, double timeout_s, int64_t* ticket) {
  if (!s || !g_host || !u0_host || !u_host) {
    set_error("st_server_submit: null pointer");
    return ST_ERR_ARG;
  }
  if (std::isnan(timeout_s)) {
    set_error("st_server_submit: timeout must not be NaN");
    return ST_ERR_ARG;
  }
  if ((domain != 0 && domain != 1 && domain != 2) || space_level < 1 || space_level > 12 ||
      (domain == 1 && space_level < 2) || (domain == 2 && space_level > 8) || time_level < 1 || time_level > 14) {
    set_error("st_server_submit: invalid domain or levels");
    return ST_ERR_ARG;
  }
  auto r = std::make_unique<Request>();
  r->domain = domain;
  r->K = space_level;
  r->J = time_level;
  r->g = g_host;
  r->u0 = u0_host;
  r->u = u_host;
  r->submitted = Clock::now();
  if (timeout_s > 0.0 && std::isfinite(timeout_s)) {
    r->has_deadline = true;
    r->deadline = r->submitted + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->error != ST_OK) {
    set_error("st_server_submit: the server stopped after an error: " + s->error_msg);
    return s->error;
  }
  if (s->stopping) {
    set_error("st_server_submit: the server is stopping");
    return ST_ERR_ARG;
  }
  r->ticket = (int64_t)s->all.size();
  if (ticket) *ticket = r->ticket;
  s->queue.push_back(r.get());
  s->all.push_back(std::move(r));
  s->cv.notify_one();
  return ST_OK;
}

st_status st_server_submit(st_server s, int domain, int space_level, int time_level, const double* g_host,
                           const double* u0_host, double* u_host, int64_t* ticket) {
  return st_server_submit_deadline(s, domain, space_level, time_level, g_host, u0_host, u_host, 0.0, ticket);
}

st_status st_server_cancel(st_server s, int64_t ticket) {
  if (!s) {
    set_error("st_server_cancel: null server");
    return ST_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket < 0 || ticket >= (int64_t)s->all.size()) {
    set_error("st_server_cancel: unknown ticket");
    return ST_ERR_ARG;
  }
  Request* r = s->all[ticket].get();
  if (r->state < REQ_DONE) {
    r->cancel = true;
    s->cv.notify_one();
  }
  return ST_OK;
}

st_status st_server_poll(st_server s, int64_t ticket, int* state, int* status, st_solve_info* info,
                         double* latency_s) {
  if (!s || !state) {
    set_error("st_server_poll: null pointer");
    return ST_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket < 0 || ticket >= (int64_t)s->all.size()) {
    set_error("st_server_poll: unknown ticket");
    return ST_ERR_ARG;
  }
  const Request* r = s->all[ticket].get();
  *state = r->state;
  if (status) *status = r->status;
  if (info) *info = r->info;
  if (latency_s)
    *latency_s = (r->state >= REQ_DONE) ? std::chrono::duration<double>(r->finished - r->submitted).count() : -1.0;
  if (s->error != ST_OK) {
    set_error("st_server_poll: the server stopped after an error: " + s->error_msg);
    return s->error;
  }
  return ST_OK;
}

st_status st_server_stop(st_server s) {
  if (!s) return ST_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->cv.notify_one();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  while (!s->groups.empty()) release_group(s, s->groups.size() - 1);
  st_status e = s->error;
  if (e != ST_OK) set_error("st_server_stop: " + s->error_msg);
  delete s;
  return e;
}

}  // extern "C"
