// Rollout server: continuous batching of rollout requests over one batch of world
// slots per morphology (section "Architecture": world state stays on the device
// between steps; requests of different morphologies share the same launches).
//
// Host runtime only: admission, slot free lists, the tick loop, result hand-off. The
// physics runs in the batch's kernels through the public calls (b3p_reset,
// b3p_sample_targets, b3p_step, b3p_gather_state, b3p_set_idle) on the server's own
// stream. Every device buffer is allocated once at create; a tick enqueues work and
// allocates nothing on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/b3phys.h"
#include "b3p_internal.h"

// sets the calling thread's b3p_last_error message (b3p_host.cpp); returns code
b3p_status b3p_set_error(b3p_status code, const char *msg);

namespace {

struct Queued {
  int64_t id;
  b3p_request req;
  double t_submit;
};
struct Running {
  int64_t id;
  b3p_request req;
  std::vector<int> slots;   // local indices within the morphology's group, ascending
  int steps;
  double t_submit, t_admit;
};
struct Retired {
  int64_t id;
  b3p_request req;
  float *host;              // pinned block: qpos rows then qvel rows
  size_t capacity;          // floats the block holds
  cudaEvent_t ev;
  double t_submit, t_admit;
};
struct Finished {
  b3p_result r;
  float *host;
  size_t capacity;
};

}  // namespace

struct b3p_server {
  b3p_server_cfg cfg{};
  std::vector<const b3p_model *> models;
  std::vector<int> cap, nq, nv, nu, start;
  int total = 0, ctrl_floats = 0;
  void *dbuf = nullptr;
  b3p_batch *batch = nullptr;
  float *d_ctrl = nullptr, *d_sigma = nullptr, *d_gather = nullptr;
  int32_t *d_ids = nullptr, *h_ids = nullptr;
  int nring = 0;
  size_t ring_ints = 0, gather_floats = 0;
  cudaStream_t stream = nullptr;
  std::deque<cudaEvent_t> tick_ev;
  std::vector<cudaEvent_t> spare_ev;

  std::mutex mu;             // queues, free lists, counters
  std::mutex tick_mu;        // one tick at a time
  std::condition_variable cv;
  std::thread th;
  bool stop = false;

  std::deque<Queued> queue;
  std::vector<Running> running;
  std::vector<Retired> retired;
  std::map<int64_t, Finished> finished;     // handed out, not yet released
  std::vector<std::vector<int>> free_slots;
  std::multimap<size_t, float *> pool;      // pinned blocks by size

  int64_t next_id = 1, ticks = 0, world_steps = 0, submitted = 0, completed = 0;
  b3p_status err = B3P_OK;
  std::string errmsg;
  std::chrono::steady_clock::time_point t0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

b3p_status sfail(b3p_status code, const std::string &msg) { return b3p_set_error(code, msg.c_str()); }

// record the first error of a tick; the server stops
b3p_status stop_with(b3p_server *s, b3p_status code, const std::string &msg) {
  if (s->err == B3P_OK) {
    s->err = code;
    s->errmsg = msg;
  }
  return sfail(code, msg);
}

b3p_status cuda_err(b3p_server *s, cudaError_t e, const char *what) {
  return stop_with(s, B3P_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// pinned result blocks, reused by capacity (powers of two floats, at least 64)
float *pool_get(b3p_server *s, size_t floats, size_t *capacity) {
  auto it = s->pool.lower_bound(floats);
  if (it != s->pool.end()) {
    float *p = it->second;
    *capacity = it->first;
    s->pool.erase(it);
    return p;
  }
  size_t n = 64;
  while (n < floats) n <<= 1;
  void *p = nullptr;
  if (cudaMallocHost(&p, n * sizeof(float)) != cudaSuccess) return nullptr;
  *capacity = n;
  return (float *)p;
}

cudaEvent_t take_event(b3p_server *s) {
  if (!s->spare_ev.empty()) {
    cudaEvent_t e = s->spare_ev.back();
    s->spare_ev.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return e;
}

// one tick; tick_mu held by the caller
b3p_status tick_impl(b3p_server *s, int32_t *active_out) {
  // bound how far the host runs ahead of the GPU (outside the state lock)
  while ((int)s->tick_ev.size() >= std::max(1, s->cfg.max_inflight_ticks)) {
    cudaEvent_t e = s->tick_ev.front();
    cudaError_t ce = cudaEventSynchronize(e);
    s->tick_ev.pop_front();
    std::lock_guard<std::mutex> lk(s->mu);
    s->spare_ev.push_back(e);
    if (ce != cudaSuccess) return cuda_err(s, ce, "tick wait");
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->err != B3P_OK) return sfail(s->err, s->errmsg);
  const double t = s->now();
  const int area = (int)(s->ticks % s->nring);
  int32_t *h = s->h_ids + area * s->ring_ints, *d = s->d_ids + area * s->ring_ints;
  float *dg = s->d_gather + area * s->gather_floats;
  size_t off = 0;

  // admission in arrival order, first fit, lowest free slots
  struct Adm { size_t ids, rng; int n; uint64_t seed; };
  std::vector<Adm> adm;
  std::deque<Queued> left;
  while (!s->queue.empty()) {
    Queued q = s->queue.front();
    s->queue.pop_front();
    auto &fl = s->free_slots[q.req.model];
    if ((int)fl.size() < q.req.nworld) {
      left.push_back(q);
      continue;
    }
    std::sort(fl.begin(), fl.end());
    Running r{q.id, q.req, std::vector<int>(fl.begin(), fl.begin() + q.req.nworld), 0, q.t_submit, t};
    fl.erase(fl.begin(), fl.begin() + q.req.nworld);
    Adm a{off, off + (size_t)q.req.nworld, q.req.nworld, q.req.seed};
    for (int i = 0; i < q.req.nworld; i++) {
      h[a.ids + i] = s->start[q.req.model] + r.slots[i];
      h[a.rng + i] = i;
    }
    off += 2 * (size_t)q.req.nworld;
    adm.push_back(a);
    s->running.push_back(std::move(r));
  }
  s->queue.swap(left);

  // requests that reach their horizon with this tick's step
  struct Ret { size_t local, global; size_t gather; int idx; };
  std::vector<Ret> ret;
  size_t goff = 0;
  int nact = 0;
  for (int i = 0; i < (int)s->running.size(); i++) {
    Running &r = s->running[i];
    nact += r.req.nworld;
    if (r.steps + 1 < r.req.horizon) continue;
    Ret x{off, off + (size_t)r.req.nworld, goff, i};
    for (int k = 0; k < r.req.nworld; k++) {
      h[x.local + k] = r.slots[k];
      h[x.global + k] = s->start[r.req.model] + r.slots[k];
    }
    off += 2 * (size_t)r.req.nworld;
    goff += (size_t)r.req.nworld * (s->nq[r.req.model] + s->nv[r.req.model]);
    ret.push_back(x);
  }
  if (active_out) *active_out = nact;
  if (nact == 0) return B3P_OK;

  cudaError_t ce;
  if (off && (ce = cudaMemcpyAsync(d, h, off * sizeof(int32_t), cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
    return cuda_err(s, ce, "slot ids upload");
  b3p_status st;
  for (const Adm &a : adm)
    if ((st = b3p_reset(s->batch, a.seed, d + a.ids, d + a.rng, a.n, s->stream)) != B3P_OK)
      return stop_with(s, st, "reset of admitted slots");
  if ((st = b3p_sample_targets(s->batch, s->d_sigma, s->d_ctrl, s->stream)) != B3P_OK)
    return stop_with(s, st, "target sampling");
  if ((st = b3p_step(s->batch, s->d_ctrl, s->cfg.decimation, s->stream)) != B3P_OK)
    return stop_with(s, st, "step");
  s->world_steps += nact;
  for (Running &r : s->running) r.steps++;

  // retire: gather rows, copy to pinned memory behind an event, idle and free the slots
  std::vector<char> gone(s->running.size(), 0);
  for (const Ret &x : ret) {
    Running &r = s->running[x.idx];
    int g = r.req.model, n = r.req.nworld;
    size_t floats = (size_t)n * (s->nq[g] + s->nv[g]);
    float *dst = dg + x.gather;
    if ((st = b3p_gather_state(s->batch, g, B3P_FIELD_QPOS, d + x.local, n, dst, s->stream)) != B3P_OK ||
        (st = b3p_gather_state(s->batch, g, B3P_FIELD_QVEL, d + x.local, n, dst + (size_t)n * s->nq[g],
                               s->stream)) != B3P_OK)
      return stop_with(s, st, "result gather");
    size_t capacity = 0;
    float *hb = pool_get(s, floats, &capacity);
    if (!hb) return stop_with(s, B3P_ERR_CUDA, "pinned result block");
    if ((ce = cudaMemcpyAsync(hb, dst, floats * sizeof(float), cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess)
      return cuda_err(s, ce, "result copy");
    if ((st = b3p_set_idle(s->batch, d + x.global, n, 1, s->stream)) != B3P_OK)
      return stop_with(s, st, "idle retired slots");
    cudaEvent_t e = take_event(s);
    ce = cudaErrorUnknown;
    if (!e || (ce = cudaEventRecord(e, s->stream)) != cudaSuccess) {
      s->pool.emplace(capacity, hb);
      return cuda_err(s, ce, "result event");
    }
    s->retired.push_back(Retired{r.id, r.req, hb, capacity, e, r.t_submit, r.t_admit});
    auto &fl = s->free_slots[g];
    fl.insert(fl.end(), r.slots.begin(), r.slots.end());
    gone[x.idx] = 1;
  }
  if (!ret.empty()) {
    std::vector<Running> keep;
    for (size_t i = 0; i < s->running.size(); i++)
      if (!gone[i]) keep.push_back(std::move(s->running[i]));
    s->running.swap(keep);
  }
  cudaEvent_t e = take_event(s);
  ce = cudaErrorUnknown;
  if (!e || (ce = cudaEventRecord(e, s->stream)) != cudaSuccess) return cuda_err(s, ce, "tick event");
  s->tick_ev.push_back(e);
  s->ticks++;
  return B3P_OK;
}

void server_thread(b3p_server *s) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::milliseconds(1),
                     [&] { return s->stop || !s->queue.empty() || !s->running.empty(); });
      if (s->stop || s->err != B3P_OK) return;
      if (s->queue.empty() && s->running.empty()) continue;
    }
    std::lock_guard<std::mutex> tl(s->tick_mu);
    if (tick_impl(s, nullptr) != B3P_OK) return;
  }
}

void release_all(b3p_server *s) {
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto &r : s->retired) {
    cudaFreeHost(r.host);
    cudaEventDestroy(r.ev);
  }
  for (auto &f : s->finished) cudaFreeHost(f.second.host);
  for (auto &p : s->pool) cudaFreeHost(p.second);
  for (auto e : s->tick_ev) cudaEventDestroy(e);
  for (auto e : s->spare_ev) cudaEventDestroy(e);
  if (s->batch) b3p_batch_destroy(s->batch);
  cudaFree(s->dbuf);
  cudaFree(s->d_ctrl);
  cudaFree(s->d_sigma);
  cudaFree(s->d_gather);
  cudaFree(s->d_ids);
  cudaFreeHost(s->h_ids);
  if (s->stream) cudaStreamDestroy(s->stream);
}

}  // namespace

extern "C" {

b3p_status b3p_server_create(const b3p_server_cfg *cfg, b3p_server **out) {
  if (!cfg || !out || !cfg->models || !cfg->sigma_host || cfg->nmodels < 1 || cfg->nmodels > 16)
    return sfail(B3P_ERR_INVALID_ARG, "server config: null pointers or nmodels outside 1..16");
  if (cfg->decimation < 1 || cfg->hbm_budget_bytes <= 0 || cfg->max_worlds_per_model < 0)
    return sfail(B3P_ERR_INVALID_ARG, "server config: decimation, budget or slot cap out of range");
  if (cudaSetDevice(cfg->device) != cudaSuccess) return sfail(B3P_ERR_CUDA, "server device");
  auto *s = new b3p_server();
  s->cfg = *cfg;
  s->t0 = std::chrono::steady_clock::now();
  const int G = cfg->nmodels;
  s->models.assign(cfg->models, cfg->models + G);
  s->cfg.models = s->models.data();
  s->cap.assign(G, 0);
  s->nq.assign(G, 0);
  s->nv.assign(G, 0);
  s->nu.assign(G, 0);
  double share = cfg->hbm_budget_bytes / G;
  int any = 0;
  for (int g = 0; g < G; g++) {
    int32_t info[8];
    b3p_status st = b3p_model_info(s->models[g], info);
    if (st != B3P_OK) { delete s; return st; }
    s->nq[g] = info[0]; s->nv[g] = info[1]; s->nu[g] = info[2];
    // bytes the batch layout charges per world (1024-world plan, so fixed costs amortise)
    b3p_sizes sz{};
    int32_t nw = 1024;
    st = b3p_batch_plan(&s->models[g], &nw, 1, &cfg->options, &sz);
    if (st != B3P_OK) { delete s; return st; }
    double per = (double)sz.total_bytes / 1024.0;
    long long c = (long long)(share / per);
    if (cfg->max_worlds_per_model > 0) c = std::min<long long>(c, cfg->max_worlds_per_model);
    c = std::min<long long>(c, 1 << 22);
    s->cap[g] = (int)std::max<long long>(c, 0);
    any += s->cap[g];
  }
  if (any == 0) { delete s; return sfail(B3P_ERR_BUSY, "the HBM budget holds no world"); }
  std::vector<int32_t> nworld(G);
  for (int g = 0; g < G; g++) {
    nworld[g] = std::max(s->cap[g], 1);   // one slot keeps an empty pool's group valid
    s->start.push_back(s->total);
    s->total += nworld[g];
    s->ctrl_floats += nworld[g] * s->nu[g];
    s->free_slots.emplace_back();
    for (int i = 0; i < s->cap[g]; i++) s->free_slots[g].push_back(i);
  }
  b3p_sizes sz{};
  b3p_status st = b3p_batch_plan(s->models.data(), nworld.data(), G, &cfg->options, &sz);
  cudaError_t ce = cudaSuccess;
  auto bail = [&](b3p_status code, const char *what) {
    std::string m = what;
    if (ce != cudaSuccess) m += std::string(": ") + cudaGetErrorString(ce);
    release_all(s);
    delete s;
    return sfail(code, m);
  };
  if (st != B3P_OK) { delete s; return st; }
  if ((ce = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(B3P_ERR_CUDA, "stream");
  if ((ce = cudaMalloc(&s->dbuf, sz.total_bytes)) != cudaSuccess) return bail(B3P_ERR_CUDA, "slot batch buffer");
  b3p_buffers bufs{s->dbuf, sz.total_bytes};
  if ((st = b3p_batch_create(s->models.data(), nworld.data(), G, &cfg->options, &bufs, s->stream, &s->batch)) != B3P_OK)
    return bail(st, "slot batch");
  s->nring = std::max(1, cfg->max_inflight_ticks) + 1;
  s->ring_ints = 4 * (size_t)s->total;
  for (int g = 0; g < G; g++) s->gather_floats += (size_t)nworld[g] * (s->nq[g] + s->nv[g]);
  if ((ce = cudaMalloc(&s->d_ctrl, sizeof(float) * std::max(s->ctrl_floats, 1))) != cudaSuccess ||
      (ce = cudaMemset(s->d_ctrl, 0, sizeof(float) * std::max(s->ctrl_floats, 1))) != cudaSuccess ||
      (ce = cudaMalloc(&s->d_sigma, sizeof(float) * G)) != cudaSuccess ||
      (ce = cudaMemcpy(s->d_sigma, cfg->sigma_host, sizeof(float) * G, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMalloc(&s->d_gather, sizeof(float) * s->gather_floats * s->nring)) != cudaSuccess ||
      (ce = cudaMalloc(&s->d_ids, sizeof(int32_t) * s->ring_ints * s->nring)) != cudaSuccess ||
      (ce = cudaMallocHost(&s->h_ids, sizeof(int32_t) * s->ring_ints * s->nring)) != cudaSuccess)
    return bail(B3P_ERR_CUDA, "server buffers");
  // every slot starts reset and idle
  if ((st = b3p_reset(s->batch, 0, nullptr, nullptr, 0, s->stream)) != B3P_OK ||
      (st = b3p_set_idle(s->batch, nullptr, 0, 1, s->stream)) != B3P_OK)
    return bail(st, "slot initialisation");
  if ((ce = cudaStreamSynchronize(s->stream)) != cudaSuccess) return bail(B3P_ERR_CUDA, "slot initialisation");
  if (cfg->run_thread) s->th = std::thread(server_thread, s);
  *out = s;
  return B3P_OK;
}

void b3p_server_destroy(b3p_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  release_all(s);
  delete s;
}

b3p_status b3p_server_capacity(const b3p_server *s, int32_t *slots, int32_t cap) {
  if (!s || !slots) return sfail(B3P_ERR_INVALID_ARG, "null argument");
  if (cap < (int32_t)s->cap.size()) return sfail(B3P_ERR_INVALID_ARG, "capacity needs one entry per morphology");
  std::copy(s->cap.begin(), s->cap.end(), slots);
  return B3P_OK;
}

b3p_status b3p_server_submit(b3p_server *s, const b3p_request *r, int64_t *id) {
  if (!s || !r) return sfail(B3P_ERR_INVALID_ARG, "null argument");
  if (r->model < 0 || r->model >= (int)s->cap.size() || r->nworld < 1 || r->horizon < 1)
    return sfail(B3P_ERR_INVALID_ARG, "request: morphology index, nworld or horizon out of range");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err != B3P_OK) return sfail(s->err, s->errmsg);
    if (r->nworld > s->cap[r->model])
      return sfail(B3P_ERR_BUSY, "request of " + std::to_string(r->nworld) + " worlds never fits the " +
                                     std::to_string(s->cap[r->model]) + "-slot pool of morphology " +
                                     std::to_string(r->model));
    int64_t k = s->next_id++;
    s->queue.push_back(Queued{k, *r, s->now()});
    s->submitted++;
    if (id) *id = k;
  }
  s->cv.notify_all();
  return B3P_OK;
}

b3p_status b3p_server_tick(b3p_server *s, int32_t *active_worlds) {
  if (!s) return sfail(B3P_ERR_INVALID_ARG, "null server");
  if (s->cfg.run_thread) return sfail(B3P_ERR_UNSUPPORTED, "the server thread ticks this server");
  std::lock_guard<std::mutex> tl(s->tick_mu);
  return tick_impl(s, active_worlds);
}

b3p_status b3p_server_poll(b3p_server *s, b3p_result *out, int32_t max, int32_t *n) {
  if (!s || !n || (max > 0 && !out)) return sfail(B3P_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *n = 0;
  if (s->err != B3P_OK) return sfail(s->err, s->errmsg);
  std::vector<Retired> keep;
  cudaError_t bad = cudaSuccess;
  for (auto &r : s->retired) {
    if (*n >= max || bad != cudaSuccess) {
      keep.push_back(r);
      continue;
    }
    cudaError_t q = cudaEventQuery(r.ev);
    if (q == cudaErrorNotReady) {
      keep.push_back(r);
      continue;
    }
    if (q != cudaSuccess) {
      bad = q;
      keep.push_back(r);
      continue;
    }
    s->spare_ev.push_back(r.ev);
    b3p_result res{};
    res.id = r.id;
    res.model = r.req.model;
    res.nworld = r.req.nworld;
    res.qpos = r.host;
    res.qvel = r.host + (size_t)r.req.nworld * s->nq[r.req.model];
    res.t_submit = r.t_submit;
    res.t_admit = r.t_admit;
    res.t_done = s->now();
    s->finished[r.id] = Finished{res, r.host, r.capacity};
    out[(*n)++] = res;
    s->completed++;
  }
  s->retired.swap(keep);
  if (bad != cudaSuccess) return cuda_err(s, bad, "result event");
  return B3P_OK;
}

b3p_status b3p_server_release(b3p_server *s, int64_t id) {
  if (!s) return sfail(B3P_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->finished.find(id);
  if (it == s->finished.end()) return sfail(B3P_ERR_INVALID_ARG, "no unreleased result with that id");
  s->pool.emplace(it->second.capacity, it->second.host);
  s->finished.erase(it);
  return B3P_OK;
}

b3p_status b3p_server_get_stats(b3p_server *s, b3p_server_stats *out) {
  if (!s || !out) return sfail(B3P_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->ticks = s->ticks;
  out->world_steps = s->world_steps;
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->queued = (int32_t)s->queue.size();
  out->active = (int32_t)s->running.size();
  out->pending = (int32_t)s->retired.size();
  out->reserved = 0;
  return s->err == B3P_OK ? B3P_OK : sfail(s->err, s->errmsg);
}

double b3p_server_now(const b3p_server *s) { return s ? s->now() : 0.0; }

}  // extern "C"
