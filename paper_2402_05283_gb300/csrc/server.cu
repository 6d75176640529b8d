// server.cu - serving loop: continuous batching of reconstructions.
//
// A host thread owned by the library runs rounds on one CUDA stream:
//   1. admission: queued requests become resident plans, in submission
//      order, while the device's free memory minus the plan's footprint
//      (iteration state + assembly buffers) stays above the reserve and the
//      active-request limit allows;
//   2. streaming: patterns pushed by the caller (copied into the request's
//      inbox at push time) are prepared on the device as soon as the request
//      is resident;
//   3. a request whose angles have all arrived joins the running set; every
//      round advances the whole running set together with one batched
//      iteration call (one launch per kernel and size group over all
//      (request, angle) tiles), so newcomers join at the next round while
//      others are mid-flight;
//   4. after its first episode a request gets a first 3D estimate, after its
//      whole schedule the final volume; both are reported as events.
// Each request computes exactly what a standalone plan computes.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "cpra_internal.h"

namespace {

enum ReqState { kQueued = 0, kResident = 1, kRunning = 2, kDone = 3, kFailed = 4 };

struct Chunk {
  int first = 0, count = 0;
  std::vector<float> I;
  std::vector<double> theta;
  bool has_theta = false;
};

struct Request {
  int64_t id = 0;
  cpra_config cfg{};
  ReqState state = kQueued;
  cpra_plan_t plan = nullptr;
  std::deque<Chunk> inbox;
  std::vector<uint8_t> arrived;
  int n_arrived = 0;
  int64_t total = 0, done = 0;
  bool first_done = false;
  int n_masked = -1;  // arrivals the plan's present mask follows (early start)
  double t_submit = 0, t_last_push = 0, t_admit = 0, t_first = -1, t_final = -1;
  std::string err;
};

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct cpra_server_s {
  cpra_server_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::map<int64_t, Request*> reqs;
  std::deque<int64_t> queue;
  std::vector<int64_t> running;
  std::deque<cpra_server_event> events;
  std::thread th;
  bool stop = false;
  int64_t next_id = 1;
  cpra_batch_t batch = nullptr;
  std::vector<int64_t> batch_ids;
  cpra_server_stats stats{};
  std::string err;
};

namespace {

void emit(cpra_server_s* s, const Request* r, int kind, double t) {
  cpra_server_event ev{};
  ev.id = r->id;
  ev.kind = kind;
  ev.t_event = t;
  ev.t_submit = r->t_submit;
  ev.t_last_pattern = r->t_last_push;
  s->events.push_back(ev);
}

void fail_request(cpra_server_s* s, Request* r, const std::string& why) {
  r->state = kFailed;
  r->err = why;
  emit(s, r, CPRA_EVENT_FAILED, now_s(s->t0));
}

// Early start: iterations a request may run before every angle arrived
// (the rest, at least one episode, wait for the last pattern)
int64_t hold_at(const cpra_server_s* s, const Request* r) {
  const int64_t e = r->cfg.n_ei;
  int64_t tail = s->cfg.early_tail > 0 ? s->cfg.early_tail : (r->total + 1) / 2;
  tail = std::max<int64_t>(e, (tail + e - 1) / e * e);
  return std::max<int64_t>(0, r->total - tail);
}

// One round of the loop; returns true when it did GPU work.
bool round(cpra_server_s* s) {
  std::vector<Request*> admit, resident, fresh_running;
  // admission in submission order, by free device memory.  Only this thread
  // admits, so the decision taken under the lock still holds when the plan
  // is made; cpra_plan itself (allocation, possibly a device-wide sync) runs
  // outside the lock, so submit, push, poll and wait never wait for it.
  for (;;) {
    Request* r = nullptr;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->queue.empty()) break;
      r = s->reqs[s->queue.front()];
      int active = 0;
      for (auto& kv : s->reqs)
        if (kv.second->state == kResident || kv.second->state == kRunning) ++active;
      if (s->cfg.max_active > 0 && active >= s->cfg.max_active) break;
      size_t it = 0, as = 0;
      cpra_plan_bytes(&r->cfg, &it, &as);
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      if (fr < it + as + s->cfg.hbm_reserve_bytes) break;
      s->queue.pop_front();
    }
    cpra_plan_t p = nullptr;
    const cpra_status st = cpra_plan(&r->cfg, s->stream, &p);
    const std::string msg = st == CPRA_OK ? std::string() : std::string(cpra_last_error(nullptr));
    std::lock_guard<std::mutex> lk(s->mu);
    if (st != CPRA_OK) {
      fail_request(s, r, msg.c_str());
      continue;
    }
    r->plan = p;
    r->state = kResident;
    r->t_admit = now_s(s->t0);
    s->stats.admitted++;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    // (a running request with early start still receives patterns)
    for (auto& kv : s->reqs)
      if ((kv.second->state == kResident || kv.second->state == kRunning) &&
          !kv.second->inbox.empty())
        resident.push_back(kv.second);
  }
  bool worked = false;
  // streaming: prepare the patterns that arrived for resident requests
  for (Request* r : resident) {
    std::deque<Chunk> chunks;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      chunks.swap(r->inbox);
    }
    for (Chunk& c : chunks) {
      cpra_status st = cpra_load_intensities(r->plan, c.I.data(), c.first, c.count,
                                             c.has_theta ? c.theta.data() : nullptr);
      worked = true;
      std::lock_guard<std::mutex> lk(s->mu);
      if (st != CPRA_OK) {
        fail_request(s, r, cpra_last_error(r->plan));
        break;
      }
      for (int i = 0; i < c.count; ++i)
        if (!r->arrived[c.first + i]) {
          r->arrived[c.first + i] = 1;
          r->n_arrived++;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->state == kResident &&
        (r->n_arrived == r->cfg.Np || (s->cfg.early_start && r->n_arrived > 0))) {
      r->state = kRunning;
      s->running.push_back(r->id);
    }
  }
  std::vector<Request*> run;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int64_t id : s->running) {
      Request* r = s->reqs[id];
      // early start: the tail of the schedule waits for every angle
      if (r->n_arrived < r->cfg.Np && r->done >= hold_at(s, r)) continue;
      run.push_back(r);
    }
  }
  // early start: each plan's present mask follows its arrivals
  for (Request* r : run) {
    if (r->n_masked == r->n_arrived) continue;
    const bool all = r->n_arrived == r->cfg.Np;
    if (all && r->n_masked < 0) {
      r->n_masked = r->n_arrived;
      continue;
    }
    cpra_status st = cpra_set_present(r->plan, all ? nullptr : r->arrived.data());
    std::lock_guard<std::mutex> lk(s->mu);
    if (st != CPRA_OK) {
      fail_request(s, r, cpra_last_error(r->plan));
      continue;
    }
    r->n_masked = r->n_arrived;
  }
  {
    std::vector<Request*> ok;
    for (Request* r : run)
      if (r->state == kRunning) ok.push_back(r);
    run.swap(ok);
  }
  if (run.empty()) return worked;
  // continuous batching: the batch follows the running set
  std::vector<int64_t> ids;
  for (Request* r : run) ids.push_back(r->id);
  if (ids != s->batch_ids) {
    if (s->batch) cpra_batch_destroy(s->batch);
    s->batch = nullptr;
    std::vector<cpra_plan_t> plans;
    for (Request* r : run) plans.push_back(r->plan);
    cpra_status st = cpra_batch_create(plans.data(), (int32_t)plans.size(), s->cfg.use_graph, &s->batch);
    if (st != CPRA_OK) {
      std::lock_guard<std::mutex> lk(s->mu);
      for (Request* r : run) fail_request(s, r, cpra_last_error(nullptr));
      s->running.clear();
      s->batch_ids.clear();
      return true;
    }
    s->batch_ids = ids;
  }
  int64_t n = s->cfg.iters_per_round > 0 ? s->cfg.iters_per_round : 10;
  for (Request* r : run) {
    n = std::min<int64_t>(n, r->total - r->done);
    const bool all = r->n_arrived == r->cfg.Np;
    if (!all) n = std::min<int64_t>(n, hold_at(s, r) - r->done);
    if (!r->first_done && all && r->done < r->cfg.n_ei) n = std::min<int64_t>(n, r->cfg.n_ei - r->done);
  }
  if (n < 1) n = 1;
  cpra_status st = cpra_batch_iterate(s->batch, (int32_t)n);
  if (st == CPRA_OK) st = cudaStreamSynchronize(s->stream) == cudaSuccess ? CPRA_OK : CPRA_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.rounds++;
    s->stats.max_batch = std::max<int64_t>(s->stats.max_batch, (int64_t)run.size());
    if (st != CPRA_OK) {
      for (Request* r : run) fail_request(s, r, "batched iteration failed");
      s->running.clear();
      return true;
    }
    for (Request* r : run) {
      r->done += n;
      s->stats.angle_iterations += n * r->n_masked;
    }
  }
  // first 3D estimates and final volumes
  for (Request* r : run) {
    const bool all = r->n_arrived == r->cfg.Np;
    const bool final = r->done >= r->total;
    const bool first = all && !r->first_done && (r->done >= r->cfg.n_ei || final);
    if (first || final) {
      cpra_status as = cpra_assemble_3d(r->plan, nullptr);
      if (as == CPRA_OK) as = cpra_sync(r->plan);
      std::lock_guard<std::mutex> lk(s->mu);
      if (as != CPRA_OK) {
        fail_request(s, r, cpra_last_error(r->plan));
        continue;
      }
      const double t = now_s(s->t0);
      if (first) {
        r->first_done = true;
        r->t_first = t;
        emit(s, r, CPRA_EVENT_FIRST_ESTIMATE, t);
      }
      if (final) {
        r->t_final = t;
        r->state = kDone;
        emit(s, r, CPRA_EVENT_FINAL, t);
        s->stats.completed++;
        continue;
      }
    }
  }
  {
    // requests held back this round stay in the running set
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<int64_t> still;
    for (int64_t id : s->running)
      if (s->reqs[id]->state == kRunning) still.push_back(id);
    s->running = still;
  }
  s->cv.notify_all();
  return true;
}

void loop(cpra_server_s* s) {
  cudaSetDevice(s->device);
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->stop) break;
    }
    const bool worked = round(s);
    if (!worked) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
  }
}

cpra_status sfail(cpra_server_s* s, cpra_status st, const std::string& msg) {
  if (s) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = msg;
  }
  return cpra::record_error(st, msg);
}

}  // namespace

extern "C" {

cpra_status cpra_server_default_config(cpra_server_config* c) {
  if (!c) return cpra::record_error(CPRA_ERR_INVALID_ARG, "config is NULL");
  std::memset(c, 0, sizeof(*c));
  c->hbm_reserve_bytes = (size_t)2 << 30;
  c->max_active = 0;
  c->iters_per_round = 10;
  c->use_graph = 1;
  c->stream = nullptr;
  return CPRA_OK;
}

cpra_status cpra_server_start(const cpra_server_config* cfg, cpra_server_t* out) {
  if (!cfg || !out) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (cfg->iters_per_round < 0 || cfg->max_active < 0 || cfg->early_tail < 0)
    return cpra::record_error(CPRA_ERR_INVALID_ARG, "negative limits");
  cpra_server_s* s = new (std::nothrow) cpra_server_s();
  if (!s) return cpra::record_error(CPRA_ERR_OUT_OF_MEMORY, "host allocation failed");
  s->cfg = *cfg;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) {
    if (cfg->stream) {
      s->stream = (cudaStream_t)cfg->stream;
    } else {
      e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
      s->own_stream = true;
    }
  }
  if (e != cudaSuccess) {
    delete s;
    return cpra::record_error(CPRA_ERR_CUDA, std::string("server stream: ") + cudaGetErrorString(e));
  }
  s->th = std::thread(loop, s);
  *out = s;
  return CPRA_OK;
}

cpra_status cpra_server_submit(cpra_server_t s, const cpra_config* cfg, int64_t* id) {
  if (!s || !cfg || !id) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  size_t a = 0, b = 0;
  cpra_status st = cpra_plan_bytes(cfg, &a, &b);
  if (st != CPRA_OK) return st;
  if (cfg->shrinkwrap_every > 0) return sfail(s, CPRA_ERR_UNSUPPORTED, "served requests run without shrink-wrap");
  if (cfg->sweep) return sfail(s, CPRA_ERR_UNSUPPORTED, "served requests run Jacobi episodes (sweep 0)");
  Request* r = new (std::nothrow) Request();
  if (!r) return sfail(s, CPRA_ERR_OUT_OF_MEMORY, "host allocation failed");
  r->cfg = *cfg;
  r->cfg.alloc = nullptr;  // the serving thread allocates with cudaMalloc
  r->cfg.free = nullptr;
  r->cfg.alloc_ctx = nullptr;
  r->arrived.assign(cfg->Np, 0);
  r->total = (int64_t)cfg->hio_iters + cfg->er_iters;
  if (r->total < 1) r->total = 1;
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->t_submit = now_s(s->t0);
  r->t_last_push = r->t_submit;
  s->reqs[r->id] = r;
  s->queue.push_back(r->id);
  s->stats.submitted++;
  *id = r->id;
  s->cv.notify_all();
  return CPRA_OK;
}

cpra_status cpra_server_push(cpra_server_t s, int64_t id, const float* I, int32_t first,
                             int32_t count, const double* theta) {
  if (!s || !I) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  int N = 0, Np = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(nullptr, CPRA_ERR_INVALID_ARG, "unknown request");
    N = it->second->cfg.N;
    Np = it->second->cfg.Np;
  }
  if (count < 1 || first < 0 || first + count > Np)
    return sfail(s, CPRA_ERR_INVALID_ARG, "bad pattern range");
  Chunk c;
  c.first = first;
  c.count = count;
  c.I.resize((size_t)count * N * N);
  cudaPointerAttributes pa;
  const bool dev = cudaPointerGetAttributes(&pa, I) == cudaSuccess &&
                   (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (dev) {
    if (cudaMemcpy(c.I.data(), I, c.I.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      return sfail(s, CPRA_ERR_CUDA, "pattern copy");
  } else {
    std::memcpy(c.I.data(), I, c.I.size() * sizeof(float));
  }
  if (theta) {
    c.has_theta = true;
    c.theta.assign(theta, theta + count);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  Request* r = s->reqs[id];
  if (r->state == kDone || r->state == kFailed) return sfail(nullptr, CPRA_ERR_INVALID_ARG, "request finished");
  r->inbox.push_back(std::move(c));
  r->t_last_push = now_s(s->t0);
  s->cv.notify_all();
  return CPRA_OK;
}

cpra_status cpra_server_poll(cpra_server_t s, cpra_server_event* ev, int32_t max_events, int32_t* got) {
  if (!s || !got || (max_events > 0 && !ev)) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int32_t k = 0;
  while (k < max_events && !s->events.empty()) {
    ev[k++] = s->events.front();
    s->events.pop_front();
  }
  *got = k;
  return CPRA_OK;
}

cpra_status cpra_server_wait(cpra_server_t s, int64_t id, double timeout_s) {
  if (!s) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(nullptr, CPRA_ERR_INVALID_ARG, "unknown request");
  Request* r = it->second;
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return r->state == kDone || r->state == kFailed;
  });
  if (!ok) return cpra::record_error(CPRA_ERR_TIMEOUT, "request not finished in time");
  if (r->state == kFailed) return cpra::record_error(CPRA_ERR_CUDA, r->err);
  return CPRA_OK;
}

cpra_status cpra_server_request_info(cpra_server_t s, int64_t id, cpra_server_request* info) {
  if (!s || !info) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return cpra::record_error(CPRA_ERR_INVALID_ARG, "unknown request");
  const Request* r = it->second;
  info->state = r->state;
  info->iterations_done = r->done;
  info->angles_arrived = r->n_arrived;
  info->t_submit = r->t_submit;
  info->t_admit = r->t_admit;
  info->t_last_pattern = r->t_last_push;
  info->t_first_estimate = r->t_first;
  info->t_final = r->t_final;
  return CPRA_OK;
}

cpra_status cpra_server_result(cpra_server_t s, int64_t id, int32_t what, void* dst, size_t bytes) {
  if (!s) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  cpra_plan_t p = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return cpra::record_error(CPRA_ERR_INVALID_ARG, "unknown request");
    if (it->second->state != kDone) return cpra::record_error(CPRA_ERR_NOT_READY, "request not finished");
    p = it->second->plan;
  }
  return cpra_result(p, what, dst, bytes);
}

cpra_status cpra_server_release(cpra_server_t s, int64_t id) {
  if (!s) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return cpra::record_error(CPRA_ERR_INVALID_ARG, "unknown request");
  Request* r = it->second;
  if (r->state != kDone && r->state != kFailed)
    return cpra::record_error(CPRA_ERR_NOT_READY, "request still active");
  if (r->plan) cpra_destroy(r->plan);
  delete r;
  s->reqs.erase(it);
  return CPRA_OK;
}

cpra_status cpra_server_get_stats(cpra_server_t s, cpra_server_stats* out) {
  if (!s || !out) return cpra::record_error(CPRA_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return CPRA_OK;
}

cpra_status cpra_server_stop(cpra_server_t s) {
  if (!s) return CPRA_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaStreamSynchronize(s->stream);
  if (s->batch) cpra_batch_destroy(s->batch);
  for (auto& kv : s->reqs) {
    if (kv.second->plan) cpra_destroy(kv.second->plan);
    delete kv.second;
  }
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
  return CPRA_OK;
}

}  // extern "C"
