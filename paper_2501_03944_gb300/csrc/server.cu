// Serving runtime (include/mgfwa.h, "Serving"): a FIFO of optimisation
// requests, admission by free slot and device footprint, one handle and one
// stream per live run, every live run stepped each tick so that their
// kernels overlap on the GPU, and retirement at budget.  Host-side C++ only;
// every step of every run is the library's kernels on that run's stream.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "mgfwa.h"
#include "mgfwa_internal.cuh"

namespace {

double now_seconds() {
  using clk = std::chrono::steady_clock;
  static const clk::time_point t0 = clk::now();
  return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Request {
  int64_t id = 0;
  mgfwa_config cfg;
  // owned copy of the objective
  int32_t kind = 0, n_layers = 0;
  std::vector<int32_t> widths, acts, y;
  std::vector<float> X, params;
  int64_t n_samples = 0;
  mgfwa_objective obj() const {
    mgfwa_objective o;
    std::memset(&o, 0, sizeof(o));
    o.kind = kind;
    o.n_layers = n_layers;
    o.widths = widths.empty() ? nullptr : widths.data();
    o.acts = acts.empty() ? nullptr : acts.data();
    o.n_samples = n_samples;
    o.X = X.empty() ? nullptr : X.data();
    o.y = y.empty() ? nullptr : y.data();
    o.params = params.empty() ? nullptr : params.data();
    return o;
  }
  mgfwa_request_info info;
  int64_t per_gen = 0;       // evaluations per generation of one run
  mgfwa_t* h = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<float> best_x;
};

}  // namespace

struct mgfwa_server {
  int32_t max_live = 1;
  int64_t limit = 0;
  int64_t next_id = 1;
  std::deque<Request*> queue;
  std::vector<Request*> live;
  std::map<int64_t, Request*> all;
  mgfwa_server_stats st;
};

namespace {

void release(Request* r) {
  if (r->h) mgfwa_destroy(r->h);
  r->h = nullptr;
  if (r->stream) cudaStreamDestroy(r->stream);
  r->stream = nullptr;
}

// Admit waiting requests in order while a slot is free and the head fits.
void admit(mgfwa_server* s) {
  while (!s->queue.empty() && (int32_t)s->live.size() < s->max_live) {
    Request* r = s->queue.front();
    if (s->st.device_bytes_in_use + r->info.footprint > s->limit) break;
    s->queue.pop_front();
    r->info.t_admit = now_seconds();
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      r->info.state = MGFWA_REQ_FAILED;
      r->info.status = MGFWA_ECUDA;
      s->st.failed += 1;
      continue;
    }
    const mgfwa_objective o = r->obj();
    const mgfwa_status cs = mgfwa_create(&r->cfg, &o, r->stream, &r->h);
    if (cs != MGFWA_OK) {
      release(r);
      r->info.state = MGFWA_REQ_FAILED;
      r->info.status = cs;
      s->st.failed += 1;
      continue;
    }
    mgfwa_info hi;
    mgfwa_get_info(r->h, &hi);
    r->info.evals = hi.evals;
    r->info.state = MGFWA_REQ_RUNNING;
    s->st.device_bytes_in_use += r->info.footprint;
    s->st.admitted += 1;
    s->live.push_back(r);
  }
}

}  // namespace

extern "C" {

mgfwa_status mgfwa_server_create(int32_t max_live, int64_t device_bytes_limit, mgfwa_server_t** out) {
  if (!out || max_live < 1 || device_bytes_limit <= 0) {
    mgfwa::set_thread_error("server: need max_live >= 1 and a positive device-byte limit");
    return MGFWA_EINVAL;
  }
  mgfwa_server* s = new (std::nothrow) mgfwa_server();
  if (!s) return MGFWA_ENOMEM;
  s->max_live = max_live;
  s->limit = device_bytes_limit;
  std::memset(&s->st, 0, sizeof(s->st));
  now_seconds();
  *out = s;
  return MGFWA_OK;
}

mgfwa_status mgfwa_server_submit(mgfwa_server_t* s, const mgfwa_config* cfg, const mgfwa_objective* obj,
                                 int64_t* request_id) {
  if (!s || !cfg || !obj || !request_id) return MGFWA_EINVAL;
  int64_t fp = 0;
  mgfwa_status st = mgfwa_footprint(cfg, obj, &fp);
  if (st != MGFWA_OK) return st;
  if (fp > s->limit) {
    mgfwa::set_thread_error("server: the request's device footprint exceeds the server's limit");
    return MGFWA_EINVAL;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) return MGFWA_ENOMEM;
  r->id = s->next_id++;
  r->cfg = *cfg;
  r->kind = obj->kind;
  r->n_layers = obj->n_layers;
  if (obj->kind == MGFWA_OBJ_MLP_CE) {
    r->widths.assign(obj->widths, obj->widths + obj->n_layers + 1);
    r->acts.assign(obj->acts, obj->acts + (obj->n_layers > 1 ? obj->n_layers - 1 : 0));
    if (r->acts.empty()) r->acts.push_back(0);
    r->n_samples = obj->n_samples;
    r->X.assign(obj->X, obj->X + obj->n_samples * obj->widths[0]);
    r->y.assign(obj->y, obj->y + obj->n_samples);
  } else if (obj->kind == MGFWA_OBJ_NET_OUTPUT) {
    r->widths.assign(obj->widths, obj->widths + obj->n_layers + 1);
    r->acts.assign(obj->acts ? obj->acts : obj->widths, (obj->acts ? obj->acts : obj->widths) +
                                                           (obj->n_layers > 1 ? obj->n_layers - 1 : 0));
    if (r->acts.empty()) r->acts.push_back(0);
    int64_t n = 0;
    for (int l = 0; l < obj->n_layers; ++l) n += (int64_t)obj->widths[l] * obj->widths[l + 1] + obj->widths[l + 1];
    r->params.assign(obj->params, obj->params + n);
  }
  std::memset(&r->info, 0, sizeof(r->info));
  r->info.state = MGFWA_REQ_QUEUED;
  r->info.footprint = fp;
  r->info.t_submit = now_seconds();
  r->per_gen = (int64_t)cfg->n_fireworks * (cfg->sparks_per_firework + cfg->guiding_per_firework);
  s->queue.push_back(r);
  s->all[r->id] = r;
  s->st.submitted += 1;
  *request_id = r->id;
  return MGFWA_OK;
}

mgfwa_status mgfwa_server_tick(mgfwa_server_t* s, int32_t generations) {
  if (!s || generations < 1) return MGFWA_EINVAL;
  admit(s);
  // enqueue work for every live run first (their streams run concurrently) ...
  for (Request* r : s->live) {
    const int64_t left = (r->cfg.eval_budget - r->info.evals) / r->per_gen;
    const int32_t n = (int32_t)(left < generations ? left : generations);
    if (n <= 0) continue;
    const mgfwa_status st = mgfwa_step(r->h, n);
    if (st != MGFWA_OK && st != MGFWA_EBUDGET) {
      r->info.state = MGFWA_REQ_FAILED;
      r->info.status = st;
      continue;
    }
    r->info.evals += (int64_t)n * r->per_gen;
    s->st.sparks_evaluated += (int64_t)n * r->per_gen * r->cfg.n_runs;
  }
  // ... then retire the runs whose budget allows no further generation
  std::vector<Request*> still;
  mgfwa_status result = MGFWA_OK;
  for (Request* r : s->live) {
    const bool spent = r->info.evals + r->per_gen > r->cfg.eval_budget;
    if (r->info.state == MGFWA_REQ_FAILED) {
      release(r);
      s->st.failed += 1;
      s->st.device_bytes_in_use -= r->info.footprint;
      result = MGFWA_ECUDA;
      continue;
    }
    if (!spent) {
      still.push_back(r);
      continue;
    }
    r->best_x.resize((size_t)r->cfg.dim);
    int64_t ev = 0;
    const mgfwa_status st = mgfwa_best(r->h, r->best_x.data(), &r->info.best_f, &ev);
    r->info.t_done = now_seconds();
    if (st == MGFWA_OK) {
      r->info.evals = ev;
      r->info.state = MGFWA_REQ_DONE;
      s->st.completed += 1;
    } else {
      r->info.state = MGFWA_REQ_FAILED;
      r->info.status = st;
      s->st.failed += 1;
      result = st;
    }
    release(r);
    s->st.device_bytes_in_use -= r->info.footprint;
  }
  s->live.swap(still);
  admit(s);
  return result;
}

mgfwa_status mgfwa_server_poll(mgfwa_server_t* s, int64_t request_id, mgfwa_request_info* info, float* x_out) {
  if (!s || !info) return MGFWA_EINVAL;
  auto it = s->all.find(request_id);
  if (it == s->all.end()) {
    mgfwa::set_thread_error("server: unknown request id");
    return MGFWA_EINVAL;
  }
  const Request* r = it->second;
  *info = r->info;
  if (x_out && r->info.state == MGFWA_REQ_DONE)
    std::memcpy(x_out, r->best_x.data(), sizeof(float) * r->best_x.size());
  return MGFWA_OK;
}

mgfwa_status mgfwa_server_stats_get(const mgfwa_server_t* s, mgfwa_server_stats* stats) {
  if (!s || !stats) return MGFWA_EINVAL;
  *stats = s->st;
  stats->live = (int32_t)s->live.size();
  stats->queued = (int32_t)s->queue.size();
  return MGFWA_OK;
}

double mgfwa_server_now(const mgfwa_server_t*) { return now_seconds(); }

void mgfwa_server_destroy(mgfwa_server_t* s) {
  if (!s) return;
  for (auto& kv : s->all) {
    release(kv.second);
    delete kv.second;
  }
  delete s;
}

}  // extern "C"
