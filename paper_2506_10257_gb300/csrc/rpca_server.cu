// rpca_server.cu -- served form: a request loop over sliding frame windows
// from several probes, with continuous batching, per-probe warm-start state
// resident on the device and admission by an HBM budget.
//
// Requests (one window each, with a probe key) are queued in arrival order.
// Progress is made inside every rpca_submit / rpca_poll / rpca_server_wait
// call (no background thread): finished requests are retired (their slot and
// their probe freed), then queued requests are started while a slot (a CUDA
// stream) is free and their probe's device state fits in the budget, so new
// arrivals join the GPU while earlier solves are still running and the
// solves of different probes overlap on the device.  A probe's requests run
// in order.  By default every window starts cold, so each result is the
// window's own solve.  With warm starts enabled (rpca_server_set_warm), a
// window starts from the previous window of the same probe: S0 and Y0 are the
// previous S and Y with the oldest frame dropped and a zero frame appended (a
// contiguous device copy in the frame-major layout), and the first mu is
// warm_mu_scale times the previous window's final mu.  A warm-started solve
// stops, like every solve, on the primal residual alone, and its end point
// depends on where it started: it is a different near-minimiser than the
// cold solve's (the oracle measures mask Dice 0.91-0.99 against the cold
// solves along a chain), hence off by default.
// Device memory per probe (the plan workspace plus the S, Y state) is charged
// against the budget; idle probes are evicted, least recently used first,
// when a new probe needs room, and a request that can never fit is refused
// with RPCA_ERR_BUDGET.
#include <cuda_runtime.h>
#include <string.h>

#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rpca.h"
#include "rpca_device.cuh"
#include "rpca_internal.h"

using rpca::Ctrl;

namespace {

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct Probe {
  int32_t key = 0;
  rpca_params p{};
  rpca_plan_t plan = nullptr;
  float* S_state = nullptr;   // final S of the probe's last window
  float* Y_state = nullptr;   // final Y of the probe's last window
  size_t bytes = 0;
  bool busy = false;          // a request of this probe is on the GPU
  bool have_prev = false;     // S_state, Y_state hold a finished window
  int64_t windows = 0;        // windows solved
  int pending = 0;            // queued + running requests
  uint64_t last_use = 0;
};

struct Request {
  uint64_t id = 0;
  int32_t key = 0;
  rpca_params p{};
  const void* X = nullptr;
  void* L = nullptr;
  void* S = nullptr;
  uint8_t* mask = nullptr;
  float theta = 0.f;
  int state = RQ_QUEUED;
  int slot = -1;
  int warm = 0;
  rpca_result res{};
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Ctrl* ctrl_host = nullptr;  // pinned copy of the finished solve's control block
  Request* req = nullptr;
};

bool same_shape(const rpca_params& a, const rpca_params& b) {
  return a.m == b.m && a.T == b.T && a.dtype == b.dtype && a.precision == b.precision &&
         a.mu_schedule == b.mu_schedule && a.drive == b.drive && a.max_iter == b.max_iter &&
         a.lambda == b.lambda && a.mu0_scale == b.mu0_scale && a.rho == b.rho &&
         a.mu_max_factor == b.mu_max_factor && a.tol == b.tol;
}

rpca_status cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return RPCA_OK;
  if (e == cudaErrorMemoryAllocation) return RPCA_ERR_NOMEM;
  return RPCA_ERR_CUDA;
}

}  // namespace

struct rpca_server_s {
  std::mutex mu;
  size_t budget = 0;
  size_t used = 0;
  size_t peak = 0;
  int warm = 0;                 // cold starts by default (see the top of this file)
  double warm_mu_scale = 0.1;
  int cold_every = 0;
  std::vector<Slot> slots;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::map<int32_t, std::unique_ptr<Probe>> probes;
  uint64_t next_id = 1;
  uint64_t tick = 0;
  int64_t started = 0, finished = 0, evicted = 0, refused = 0;
  int running = 0, max_running = 0;
};

namespace {

size_t probe_bytes(const rpca_params& p) {
  size_t ws = 0;
  if (rpca_workspace_size(&p, &ws) != RPCA_OK) return 0;
  return ws + 2 * sizeof(float) * (size_t)p.m * (size_t)p.T * (p.dtype == RPCA_C64 ? 2 : 1);
}

void free_probe(rpca_server_s* sv, Probe* pr) {
  if (pr->plan) rpca_plan_destroy(pr->plan);
  if (pr->S_state) cudaFree(pr->S_state);
  if (pr->Y_state) cudaFree(pr->Y_state);
  sv->used -= pr->bytes;
  pr->plan = nullptr;
  pr->S_state = pr->Y_state = nullptr;
  pr->bytes = 0;
  pr->have_prev = false;
}

// Evicts idle probes (least recently used first) until `need` more bytes fit.
bool make_room(rpca_server_s* sv, size_t need, int32_t keep_key) {
  while (sv->used + need > sv->budget) {
    Probe* victim = nullptr;
    for (auto& kv : sv->probes) {
      Probe* pr = kv.second.get();
      if (pr->key == keep_key || pr->busy || pr->pending > 0 || pr->bytes == 0) continue;
      if (!victim || pr->last_use < victim->last_use) victim = pr;
    }
    if (!victim) return false;
    free_probe(sv, victim);
    sv->evicted += 1;
  }
  return true;
}

// Device state of the request's probe, created (or re-created for new
// parameters) within the budget.  RPCA_PENDING: not now, memory is held by
// probes with work in flight.
rpca_status ensure_probe(rpca_server_s* sv, Request* rq, Probe** out) {
  auto it = sv->probes.find(rq->key);
  if (it == sv->probes.end()) it = sv->probes.emplace(rq->key, std::make_unique<Probe>()).first;
  Probe* pr = it->second.get();
  pr->key = rq->key;
  if (pr->plan && same_shape(pr->p, rq->p)) {
    *out = pr;
    return RPCA_OK;
  }
  if (pr->plan) free_probe(sv, pr);  // parameters changed: start this probe afresh
  const size_t need = probe_bytes(rq->p);
  if (need == 0) return RPCA_ERR_ARG;
  if (!make_room(sv, need, pr->key)) return RPCA_PENDING;
  rpca_params q = rq->p;
  q.warm_start = 1;  // every solve of a probe reads S0, Y0 (zero for a cold one)
  q.mu_init = 0.0;
  q.mu_prev_scale = 0.0;
  if (q.drive == RPCA_DRIVE_HOST) q.drive = RPCA_DRIVE_GRAPH;
  const size_t mT = sizeof(float) * (size_t)q.m * (size_t)q.T * (q.dtype == RPCA_C64 ? 2 : 1);
  rpca_status st = rpca_plan_create(&q, nullptr, 0, &pr->plan);
  if (st == RPCA_OK) st = cuda_st(cudaMalloc((void**)&pr->S_state, mT));
  if (st == RPCA_OK) st = cuda_st(cudaMalloc((void**)&pr->Y_state, mT));
  pr->bytes = need;
  sv->used += need;
  sv->peak = sv->used > sv->peak ? sv->used : sv->peak;
  if (st != RPCA_OK) {
    free_probe(sv, pr);
    return st;
  }
  pr->p = rq->p;
  pr->have_prev = false;
  pr->windows = 0;
  *out = pr;
  return RPCA_OK;
}

// Enqueues one request's solve on a free slot.
rpca_status start(rpca_server_s* sv, Request* rq, Probe* pr, int slot) {
  Slot& sl = sv->slots[slot];
  cudaStream_t s = sl.stream;
  const int T = rq->p.T;
  const int64_t m = rq->p.m * (rq->p.dtype == RPCA_C64 ? 2 : 1);  // floats per frame
  const size_t frame = sizeof(float) * (size_t)m;
  const bool warm = sv->warm && pr->have_prev && !(sv->cold_every > 0 && pr->windows % sv->cold_every == 0);
  cudaError_t e = cudaSuccess;
  if (warm) {
    // S0, Y0: drop the oldest frame, append a zero frame (frame-major => contiguous)
    float* S = (float*)rq->S;
    float* Y0 = (float*)rq->L;
    if (T > 1) {
      e = cudaMemcpyAsync(S, pr->S_state + m, frame * (T - 1), cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(Y0, pr->Y_state + m, frame * (T - 1), cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(S + (size_t)(T - 1) * m, 0, frame, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(Y0 + (size_t)(T - 1) * m, 0, frame, s);
  } else {
    e = cudaMemsetAsync(rq->S, 0, frame * T, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rq->L, 0, frame * T, s);
  }
  if (e != cudaSuccess) return cuda_st(e);
  rpca_status st = rpca::plan_solve_ex(pr->plan, rq->X, rq->L, rq->S, rq->mask, rq->theta, s, pr->S_state,
                                       pr->Y_state, warm ? sv->warm_mu_scale : 0.0, nullptr);
  if (st != RPCA_OK) return st;
  e = cudaMemcpyAsync(sl.ctrl_host, rpca::plan_ctrl(pr->plan), sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, s);
  if (e != cudaSuccess) return cuda_st(e);
  rq->state = RQ_RUNNING;
  rq->slot = slot;
  rq->warm = warm ? 1 : 0;
  sl.req = rq;
  pr->busy = true;
  pr->last_use = ++sv->tick;
  sv->started += 1;
  sv->running += 1;
  if (sv->running > sv->max_running) sv->max_running = sv->running;
  return RPCA_OK;
}

void finish(rpca_server_s* sv, Slot& sl, rpca_status err) {
  Request* rq = sl.req;
  Probe* pr = sv->probes[rq->key].get();
  rpca::PlanView v;
  rpca::plan_view(pr->plan, &v);
  if (err == RPCA_OK) {
    rpca::result_from_ctrl(v.lambda, *sl.ctrl_host, &rq->res, v.cplx);
  } else {
    memset(&rq->res, 0, sizeof(rq->res));
    rq->res.status = err;
  }
  rq->state = RQ_DONE;
  rq->slot = -1;
  sl.req = nullptr;
  pr->busy = false;
  pr->pending -= 1;
  pr->windows += 1;
  pr->have_prev = rq->res.status >= 0;
  sv->finished += 1;
  sv->running -= 1;
}

// Retire finished solves, then start queued requests while slots and memory allow.
void progress(rpca_server_s* sv) {
  for (Slot& sl : sv->slots) {
    if (!sl.req) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    finish(sv, sl, q == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA);
  }
  for (auto it = sv->queue.begin(); it != sv->queue.end();) {
    int slot = -1;
    for (int i = 0; i < (int)sv->slots.size(); ++i)
      if (!sv->slots[i].req) {
        slot = i;
        break;
      }
    if (slot < 0) break;
    Request* rq = *it;
    auto pit = sv->probes.find(rq->key);
    if (pit != sv->probes.end() && pit->second->busy) {  // keep each probe's windows in order
      ++it;
      continue;
    }
    bool earlier_same_probe = false;
    for (auto jt = sv->queue.begin(); jt != it; ++jt)
      if ((*jt)->key == rq->key) earlier_same_probe = true;
    if (earlier_same_probe) {
      ++it;
      continue;
    }
    Probe* pr = nullptr;
    rpca_status st = ensure_probe(sv, rq, &pr);
    if (st == RPCA_PENDING) {  // memory held by work in flight: try later
      ++it;
      continue;
    }
    if (st == RPCA_OK) st = start(sv, rq, pr, slot);
    if (st != RPCA_OK) {
      memset(&rq->res, 0, sizeof(rq->res));
      rq->res.status = st;
      rq->state = RQ_DONE;
      auto p2 = sv->probes.find(rq->key);
      if (p2 != sv->probes.end()) p2->second->pending -= 1;
    }
    it = sv->queue.erase(it);
  }
}

}  // namespace

extern "C" {

rpca_status rpca_server_create(size_t hbm_budget_bytes, int32_t max_slots, rpca_server_t* out) {
  if (!out || hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 256) return RPCA_ERR_ARG;
  *out = nullptr;
  rpca_server_s* sv = new rpca_server_s();
  sv->budget = hbm_budget_bytes;
  sv->slots.resize(max_slots);
  cudaError_t e = cudaSuccess;
  for (Slot& sl : sv->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.ctrl_host, sizeof(Ctrl));
  }
  if (e != cudaSuccess) {
    rpca_server_destroy(sv);
    return cuda_st(e);
  }
  *out = sv;
  return RPCA_OK;
}

rpca_status rpca_server_set_warm(rpca_server_t sv, int32_t warm, double warm_mu_scale, int32_t cold_every) {
  if (!sv || (warm != 0 && warm != 1) || !(warm_mu_scale >= 0.0) || cold_every < 0) return RPCA_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->warm = warm;
  sv->warm_mu_scale = warm_mu_scale;
  sv->cold_every = cold_every;
  return RPCA_OK;
}

rpca_status rpca_submit(rpca_server_t sv, const rpca_params* p, const void* X, void* L, void* S, uint8_t* mask,
                        float theta, int32_t stream_key, uint64_t* req_id) {
  if (!sv || !p || !X || !L || !S || !req_id) return RPCA_ERR_ARG;
  if (((uintptr_t)X | (uintptr_t)L | (uintptr_t)S) & 15u) return RPCA_ERR_ARG;
  if (X == L || X == S || L == S) return RPCA_ERR_ARG;
  size_t ws = 0;
  rpca_status st = rpca_workspace_size(p, &ws);
  if (st != RPCA_OK) return st;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (probe_bytes(*p) > sv->budget) {
    sv->refused += 1;
    return RPCA_ERR_BUDGET;
  }
  auto rq = std::make_unique<Request>();
  rq->id = sv->next_id++;
  rq->key = stream_key;
  rq->p = *p;
  rq->X = X;
  rq->L = L;
  rq->S = S;
  rq->mask = mask;
  rq->theta = theta;
  auto pit = sv->probes.find(stream_key);
  if (pit == sv->probes.end()) pit = sv->probes.emplace(stream_key, std::make_unique<Probe>()).first;
  pit->second->key = stream_key;
  pit->second->pending += 1;
  *req_id = rq->id;
  sv->queue.push_back(rq.get());
  sv->reqs.emplace(rq->id, std::move(rq));
  progress(sv);
  return RPCA_OK;
}

rpca_status rpca_poll(rpca_server_t sv, uint64_t req_id, rpca_result* out) {
  if (!sv) return RPCA_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  progress(sv);
  auto it = sv->reqs.find(req_id);
  if (it == sv->reqs.end()) return RPCA_ERR_NOTFOUND;
  Request* rq = it->second.get();
  if (rq->state != RQ_DONE) return RPCA_PENDING;
  if (out) *out = rq->res;
  const rpca_status st = (rpca_status)rq->res.status;
  sv->reqs.erase(it);
  return st;
}

rpca_status rpca_server_wait(rpca_server_t sv, uint64_t req_id, rpca_result* out) {
  if (!sv) return RPCA_ERR_ARG;
  for (;;) {
    cudaEvent_t ev = nullptr;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      progress(sv);
      auto it = sv->reqs.find(req_id);
      if (it == sv->reqs.end()) return RPCA_ERR_NOTFOUND;
      Request* rq = it->second.get();
      if (rq->state == RQ_DONE) {
        if (out) *out = rq->res;
        const rpca_status st = (rpca_status)rq->res.status;
        sv->reqs.erase(it);
        return st;
      }
      if (rq->state == RQ_RUNNING) ev = sv->slots[rq->slot].done;
      else {
        // queued: wait for any running solve to end
        for (Slot& sl : sv->slots)
          if (sl.req) {
            ev = sl.done;
            break;
          }
        // nothing running and still queued: its memory is held by probes
        // with queued work of their own that cannot start either
        if (!ev) return RPCA_ERR_BUDGET;
      }
    }
    if (ev) cudaEventSynchronize(ev);
    else std::this_thread::yield();
  }
}

rpca_status rpca_server_stats(rpca_server_t sv, int64_t* stats, int32_t n) {
  if (!sv || !stats || n < 0) return RPCA_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  progress(sv);
  const int64_t v[10] = {(int64_t)sv->used, (int64_t)sv->peak, (int64_t)sv->budget, (int64_t)sv->queue.size(),
                         (int64_t)sv->running, (int64_t)sv->max_running, sv->started, sv->finished,
                         sv->evicted, sv->refused};
  for (int i = 0; i < n && i < 10; ++i) stats[i] = v[i];
  return RPCA_OK;
}

void rpca_server_destroy(rpca_server_t sv) {
  if (!sv) return;
  for (Slot& sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  }
  for (auto& kv : sv->probes) free_probe(sv, kv.second.get());
  for (Slot& sl : sv->slots) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ctrl_host) cudaFreeHost(sl.ctrl_host);
  }
  delete sv;
}

}  // extern "C"
