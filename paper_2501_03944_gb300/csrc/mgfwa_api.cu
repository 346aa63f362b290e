// C ABI of the library (include/mgfwa.h, include/mgfwa_debug.h): handle
// life cycle, device arena, the generation driver of Algorithm 1 and the
// reporting calls.  All device work is enqueued on the handle's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mgfwa.h"
#include "mgfwa_debug.h"
#include "fitness_tc.cuh"
#include "grad.cuh"
#include "mgfwa_internal.cuh"

using namespace mgfwa;

namespace {
thread_local std::string g_create_error;
}  // namespace

void mgfwa::set_thread_error(const char* msg) { g_create_error = msg ? msg : ""; }

struct mgfwa_handle {
  mgfwa_config cfg;
  Problem p;
  Mlp mlp;
  NetOut net;                   // testbed network objective (params point into the arena)
  int64_t net_count = 0;        // its parameter count
  float* net_act = nullptr;     // [2][PA][hmax] hidden activations
  uint32_t* net_x3_buf = nullptr;  // FP32X3: the layers' BF16 parts (activations ping-pong, weights)
  NetX3Plan net_x3;             // FP32X3: the testbed network's tensor-core layers
  int32_t kind = MGFWA_OBJ_MLP_CE;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool pooled = false;       // the arena came from the library's stream-ordered pool
  uint64_t fingerprint = 0;  // configuration + objective (checkpoints load only into the same problem)
  // device buffers (carved from the arena)
  float* X = nullptr;
  void* Xop = nullptr;          // [N][d_in] X as the tensor-core operand (BF16 or E4M3)
  int32_t* y = nullptr;
  float* fw_x = nullptr;
  float* fw_amp = nullptr;
  float* fw_f = nullptr;
  float* sparks = nullptr;  // [P][Dp]: explosion rows, then guiding rows
  void* op = nullptr;            // [P][w1_elems] first-layer operand (BF16 or E4M3)
  void* w2op = nullptr;          // [P][w2_rows][h1] BF16 W2 for the CTA-pair fitness kernel, or null
  int32_t w2_rows = 0;           // 16 or 32 (rows C.. are zero), or h2 with three layers
  void* w3op = nullptr;          // [P][w3_rows][h2] BF16 W3 for the three-layer CTA-pair kernel, or null
  int32_t w3_rows = 0;           // 16 (rows C.. are zero)
  int32_t op_kind = kOpNone;
  float inv_x = 1.0f, inv_w = 1.0f;  // E4M3: stored = E4M3(value * inv)
  float op_scale = 1.0f;             // layer-1 accumulator multiplier: 1 / (inv_x inv_w)
  float* fit = nullptr;         // [P]
  float* partial = nullptr;     // [mtiles][P]
  int32_t* top = nullptr;
  int32_t* bottom = nullptr;
  int32_t* winner = nullptr;
  float* f_old = nullptr;     // [B*mu] fitness before the selection (loser-out tournament)
  int32_t* loser = nullptr;   // [B*mu] 1 where the last tournament re-drew the firework
  float* gv = nullptr;        // [B*mu*m][Dp] lagged multi-guiding: the last recorded guiding vectors
  bool gv_ready = false;      // gv holds a generation's vectors
  bool lag_now = false;       // this generation guides from the previous one's vectors
  int32_t* elite = nullptr;     // [B*mu*E] spark rows picked for the FP32 re-score
  GradPlan rescore_plan;        // FP32 forward of the B*mu*E re-scored rows
  float* rescore_scratch = nullptr;
  L1Plan rescore_l1;            // their first layer on the tensor cores (over the spark rows)
  L1Plan refine_l1;             // the refinement's first layer on the tensor cores (over its rows)
  uint32_t* l1_xs = nullptr;    // X as three BF16 parts, for both (when the shape allows the layer)
  uint32_t* rescore_ws = nullptr;  // the re-scored rows' W1 parts
  uint32_t* refine_ws = nullptr;   // the refined rows' W1 parts
  float* best_x = nullptr;
  float* best_f = nullptr;
  double* ce64 = nullptr;
  double* f64 = nullptr;
  uint32_t* status = nullptr;
  uint32_t* gens_done = nullptr;  // device copy of the completed-generation count (Philox counter word)
  // hybrid refinement (refine_every > 0): one vector per run
  bool refine = false;
  GradPlan gp;
  float* rw = nullptr;        // [B][Dp] the vector being refined
  float* rg = nullptr;        // [B][Dp] its gradient
  float* rf = nullptr;        // [B] FP32 fitness of the refined vector
  int32_t* relite = nullptr;  // [B] firework refined, index within the run
  int32_t* rflags = nullptr;  // [B] refinement decisions
  float* gscratch = nullptr;  // backpropagation scratch (GradPlan)
  cudaGraphExec_t refine_exec = nullptr;  // the refinement's kernels, captured once
  bool capturing = false;                 // a graph (its own or a group's) is capturing a generation: no host counters
  bool grouped = false;                   // member of a group
  int64_t refine_kernels = 0;             // kernels in that graph
  cudaGraphExec_t gen_exec = nullptr;     // one generation (explode .. select), captured at the first step
  int64_t gen_kernels = 0;                // kernels in that graph
  bool want_op = false; // tensor-core path: operand copies of X and of the first-layer weights
  int64_t P = 0;       // sparks per generation of one run
  int64_t PA = 0;      // sparks per generation of all runs (rows of the spark buffers)
  int32_t mtiles = 0;  // sample tiles of 128
  int64_t evals = 0;
  int32_t gen = 0;
  int32_t mu_run = 0;                       // fireworks of the whole run (this handle holds a shard of them)
  mgfwa_reduce_best_fn reduce_best = nullptr;  // combines the shards' best keys (null: the handle is the run)
  void* reduce_ctx = nullptr;
  int32_t next_phase = MGFWA_PHASE_EXPLODE;
  int64_t launches = 0;
  bool broken = false;
  TcPlan tc;
  std::string err;
  // kernel-group timing (mgfwa_debug_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_next = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_marks;
};

namespace {

// MGFWA_TRACE=1 in the environment prints the steps of mgfwa_create to stderr.
bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char* v = getenv("MGFWA_TRACE");
    on = (v && v[0] == '1') ? 1 : 0;
  }
  return on == 1;
}
#define TRACE(...)                       \
  do {                                   \
    if (trace_on()) {                    \
      fprintf(stderr, "[mgfwa] " __VA_ARGS__); \
      fputc('\n', stderr);               \
      fflush(stderr);                    \
    }                                    \
  } while (0)

mgfwa_status fail(mgfwa_t* h, mgfwa_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) {
    h->err = buf;
    if (st == MGFWA_ECUDA) h->broken = true;
  } else {
    g_create_error = buf;
  }
  return st;
}

mgfwa_status cuda_fail(mgfwa_t* h, const char* what) {
  cudaError_t e = cudaGetLastError();
  return fail(h, MGFWA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CREATE_LAUNCH(expr, what)                         \
  do {                                                    \
    const int n_ = (expr);                                \
    if (n_ < 0) return bail(cuda_fail(h, (what)));        \
    h->launches += n_;                                    \
  } while (0)

#define MG_LAUNCH(h, expr, what)                          \
  do {                                                    \
    const int n_ = (expr);                                \
    if (n_ < 0) return cuda_fail((h), (what));            \
    (h)->launches += n_;                                  \
  } while (0)

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

enum { G_EXPLODE = 0, G_FIT_E = 1, G_FINISH = 2, G_RANK = 3, G_GUIDE = 4, G_FIT_G = 5, G_SELECT = 6, G_RESCORE = 7,
       G_REFINE = 8 };

// Brackets one kernel group with events when profiling is on.
struct Mark {
  mgfwa_t* h;
  int group;
  cudaEvent_t a = nullptr, b = nullptr;
  Mark(mgfwa_t* h_, int g) : h(h_), group(g) {
    if (!h->profiling || h->ev_next + 2 > h->ev_pool.size()) return;
    a = h->ev_pool[h->ev_next++];
    b = h->ev_pool[h->ev_next++];
    cudaEventRecord(a, h->stream);
  }
  ~Mark() {
    if (!a) return;
    cudaEventRecord(b, h->stream);
    h->ev_marks.push_back({group, {a, b}});
  }
};

int32_t subset_size(float sigma, int32_t g) {
  int32_t k = (int32_t)std::floor((double)sigma * (double)g + 0.5);
  if (k > g / 2) k = g / 2;
  if (k < 1) k = 1;
  return k;
}

bool use_tc(const mgfwa_t* h, int32_t precision) {
  return h->kind == MGFWA_OBJ_MLP_CE && (precision == MGFWA_BF16 || precision == MGFWA_FP8);
}

// Fitness of `count` consecutive spark rows starting at row `first` into
// fit[first..first+count); with defer_finish the per-tile sums stay in
// h->partial for the next kernel to finish (MLP objectives only).
mgfwa_status eval_rows(mgfwa_t* h, int64_t first, int32_t count, int32_t precision, bool defer_finish = false) {
  if (count <= 0) return MGFWA_OK;
  const float* rows = h->sparks + first * h->p.Dp;
  float* fit = h->fit + first;
  const int group = first == 0 ? G_FIT_E : G_FIT_G;
  if (h->kind == MGFWA_OBJ_SPHERE) {
    Mark mk(h, group);
    MG_LAUNCH(h, launch_fitness_sphere(rows, h->p.Dp, h->p.D, count, fit, h->stream), "sphere fitness");
    return MGFWA_OK;
  }
  if (h->kind == MGFWA_OBJ_NET_OUTPUT) {
    Mark mk(h, group);
    if (precision == MGFWA_FP32X3)
      MG_LAUNCH(h, launch_net_output_x3(h->net_x3, h->net, rows, h->p.Dp, count, fit, h->net_act, h->net.hmax,
                                        h->status, h->stream),
                "network output (tensor cores)");
    else
      MG_LAUNCH(h, launch_net_output(h->net, rows, h->p.Dp, count, fit, h->net_act, h->net.hmax, h->stream),
                "network output");
    return MGFWA_OK;
  }
  {
    Mark mk(h, group);
    if (use_tc(h, precision))
      MG_LAUNCH(h, launch_fitness_tc(h->tc, h->mlp, first, rows, h->p.Dp, count, h->op_scale, h->partial,
                                     h->status, h->stream),
                "tensor-core fitness");
    else
      MG_LAUNCH(h, launch_fitness_simt_main(h->mlp, rows, h->p.Dp, count, h->partial, h->stream), "FP32 fitness");
  }
  if (defer_finish) return MGFWA_OK;
  Mark mk(h, G_FINISH);
  MG_LAUNCH(h, launch_fitness_finish(h->partial, h->mtiles, count, h->mlp.N, fit, h->stream), "fitness finish");
  return MGFWA_OK;
}

// The generation's elite re-score runs (low precision, E > 0, MLP objective).
bool rescore_on(const mgfwa_t* h) {
  return h->cfg.precision != MGFWA_FP32 && h->cfg.elite_rescore > 0 && h->kind == MGFWA_OBJ_MLP_CE;
}

// In a captured generation the fitness means are finished by the kernel
// that first reads them (the explosion sparks' by the rank, the guiding
// sparks' by the elite pick when the re-score runs), one launch fewer
// each; phase-by-phase stepping keeps the separate finish so that every
// phase's buffers can be read.
bool finish_in_rank(const mgfwa_t* h) { return h->capturing && h->kind == MGFWA_OBJ_MLP_CE; }
bool finish_in_pick(const mgfwa_t* h) { return h->capturing && rescore_on(h); }

// Generation `gen` (1-based) ends with a hybrid refinement.
bool refine_due(const mgfwa_t* h, int32_t gen) {
  return h->refine && h->cfg.refine_steps > 0 && gen % h->cfg.refine_every == 0;
}

// Evaluations one refinement charges: 3 per gradient step, 1 for the result.
int64_t refine_cost(const mgfwa_t* h) { return 3 * (int64_t)h->cfg.refine_steps + 1; }

// The operand descriptor of rows [first, ...) (kind none without a tensor-core path).
OpDesc op_rows(const mgfwa_t* h, int64_t first) {
  OpDesc d;
  d.base = h->op;
  d.kind = h->op ? h->op_kind : kOpNone;
  d.inv_scale = h->inv_w;
  d.w1_elems = h->mlp.w1_elems;
  if (h->op && h->w2op) {
    d.w2 = h->w2op;
    d.w2_off = h->mlp.w_off[1];
    d.w2_h1 = h->mlp.widths[1];
    d.w2_classes = h->mlp.widths[2];
    d.w2_rows = h->w2_rows;
  }
  if (h->op && h->w3op) {
    d.w3 = h->w3op;
    d.w3_off = h->mlp.w_off[2];
    d.w3_k = h->mlp.widths[2];
    d.w3_classes = h->mlp.widths[3];
    d.w3_rows = h->w3_rows;
  }
  return d.from(first);
}

// Enqueue one refinement (pick, steps, fitness of the result, accept) on s;
// returns the kernels enqueued or -1.
int enqueue_refine(mgfwa_t* h, cudaStream_t s) {
  const Problem& p = h->p;
  const mgfwa_config& c = h->cfg;
  int n = 0, k;
  if ((k = launch_refine_pick(h->fw_x, h->fw_f, p.B, p.mu, p.Dp, h->rw, h->relite, s)) < 0) return -1;
  n += k;
  for (int32_t i = 0; i < c.refine_steps; ++i) {
    if ((k = launch_grad(h->gp, h->mlp, h->rw, p.Dp, h->gscratch, h->rg, nullptr, s, nullptr, &h->refine_l1,
                         h->status)) < 0)
      return -1;
    n += k;
    if ((k = launch_sgd(h->rw, h->rg, p.B, p.D, p.Dp, c.refine_lr, p.lb, p.ub, s)) < 0) return -1;
    n += k;
  }
  if ((k = launch_grad(h->gp, h->mlp, h->rw, p.Dp, h->gscratch, nullptr, h->rf, s, nullptr, &h->refine_l1,
                       h->status)) < 0)
    return -1;
  n += k;
  if ((k = launch_refine_accept(h->rw, h->rf, h->relite, h->rflags, h->fw_x, h->fw_f, h->best_x, h->best_f, p.B,
                                p.mu, p.Dp, s)) < 0)
    return -1;
  return n + k;
}

// Capture the refinement into h->refine_exec (on a private stream, so the
// caller's stream is never in capture mode).
mgfwa_status capture_refine(mgfwa_t* h) {
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(h, "capture stream");
  cudaGraph_t graph = nullptr;
  int n = -1;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    n = enqueue_refine(h, cs);
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) n = -1;
  }
  mgfwa_status st = MGFWA_OK;
  if (n < 0 || !graph || cudaGraphInstantiate(&h->refine_exec, graph, 0) != cudaSuccess) {
    h->refine_exec = nullptr;
    st = cuda_fail(h, "refine graph capture");
  } else {
    h->refine_kernels = n;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  return st;
}

mgfwa_status run_phase(mgfwa_t* h, int32_t phase) {
  const Problem& p = h->p;
  const int64_t n_e = (int64_t)p.B * p.mu * p.lam;  // explosion rows of all runs
  const int32_t prec = h->cfg.precision;
  switch (phase) {
    case MGFWA_PHASE_EXPLODE: {
      if (!h->capturing) h->gen += 1;
      // lagged multi-guiding: once a generation's vectors are recorded, the
      // guiding sparks come from them right after the explosion
      h->lag_now = h->cfg.lagged_guiding && h->gv_ready;
      Mark mk(h, G_EXPLODE);
      MG_LAUNCH(h, launch_explode(p, h->gens_done, h->fw_x, h->fw_amp, h->sparks, op_rows(h, 0), h->stream),
                "explode");
      if (h->lag_now)
        MG_LAUNCH(h, launch_guide(p, h->gens_done, h->fw_x, h->fw_amp, h->sparks, h->top, h->bottom,
                                  h->sparks + n_e * p.Dp, op_rows(h, n_e), h->stream, h->gv, nullptr),
                  "lagged guide");
      return MGFWA_OK;
    }
    case MGFWA_PHASE_EVAL_E:
      // lagged: explosion and guiding rows are contiguous and evaluated in one launch; the means are
      // finished by the rank and the elite pick when both fuse the finish, else here
      if (h->lag_now) return eval_rows(h, 0, (int32_t)(n_e + (int64_t)p.B * p.mu * p.m), prec, finish_in_pick(h));
      return eval_rows(h, 0, (int32_t)n_e, prec, finish_in_rank(h));
    case MGFWA_PHASE_RANK: {
      Mark mk(h, G_RANK);
      const bool fin = h->lag_now ? finish_in_pick(h) : finish_in_rank(h);
      const int64_t stride = h->lag_now ? n_e + (int64_t)p.B * p.mu * p.m : n_e;
      if (fin)
        MG_LAUNCH(h, launch_rank(p, h->fit, h->top, h->bottom, h->stream, h->partial, h->mtiles, h->mlp.N, stride),
                  "rank");
      else
        MG_LAUNCH(h, launch_rank(p, h->fit, h->top, h->bottom, h->stream), "rank");
      return MGFWA_OK;
    }
    case MGFWA_PHASE_GUIDE: {
      Mark mk(h, G_GUIDE);
      // lagged: record this generation's vectors only (its guiding sparks exist already)
      MG_LAUNCH(h, launch_guide(p, h->gens_done, h->fw_x, h->fw_amp, h->sparks, h->top, h->bottom,
                                h->lag_now ? nullptr : h->sparks + n_e * p.Dp, op_rows(h, n_e), h->stream, nullptr,
                                h->cfg.lagged_guiding ? h->gv : nullptr),
                "guide");
      if (h->cfg.lagged_guiding) h->gv_ready = true;
      return MGFWA_OK;
    }
    case MGFWA_PHASE_EVAL_G:
      if (h->lag_now) return MGFWA_OK;
      return eval_rows(h, n_e, p.B * p.mu * p.m, prec, finish_in_pick(h));
    case MGFWA_PHASE_RESCORE: {
      // low precision: each firework's elite candidates get their fitness in FP32
      const int32_t E = h->cfg.elite_rescore;
      if (!rescore_on(h)) return MGFWA_OK;
      Mark mk(h, G_RESCORE);
      if (finish_in_pick(h) && h->lag_now)
        MG_LAUNCH(h, launch_elite_pick(p, h->fit, h->fit + n_e, E, h->elite, h->stream, h->partial + n_e, h->mtiles,
                                       h->mlp.N, n_e + (int64_t)p.B * p.mu * p.m),
                  "elite pick");
      else if (finish_in_pick(h))
        MG_LAUNCH(h, launch_elite_pick(p, h->fit, h->fit + n_e, E, h->elite, h->stream, h->partial, h->mtiles,
                                       h->mlp.N),
                  "elite pick");
      else
        MG_LAUNCH(h, launch_elite_pick(p, h->fit, h->fit + n_e, E, h->elite, h->stream), "elite pick");
      MG_LAUNCH(h, launch_grad(h->rescore_plan, h->mlp, h->sparks, p.Dp, h->rescore_scratch, nullptr, h->fit,
                               h->stream, h->elite, &h->rescore_l1, h->status),
                "elite FP32 fitness");
      return MGFWA_OK;
    }
    case MGFWA_PHASE_SELECT: {
      Mark mk(h, G_SELECT);
      MG_LAUNCH(h, launch_select(p, h->fit, h->fit + n_e, h->sparks, h->sparks + n_e * p.Dp, h->fw_x, h->fw_amp,
                                 h->fw_f, h->winner, h->best_x, h->best_f, h->gens_done, h->f_old, h->loser,
                                 h->stream),
                "select");
      if (!h->capturing) h->evals += h->P;
      return MGFWA_OK;
    }
    case MGFWA_PHASE_REFINE: {
      // hybrid refinement of each run's elite: projected gradient descent,
      // kept on strict improvement.  Its ~12 launches per step do not
      // depend on the generation, so they are captured once as a CUDA graph.
      if (!refine_due(h, h->gen)) return MGFWA_OK;
      if (!h->refine_exec) {
        mgfwa_status st = capture_refine(h);
        if (st != MGFWA_OK) return st;
      }
      Mark mk(h, G_REFINE);
      if (cudaGraphLaunch(h->refine_exec, h->stream) != cudaSuccess) return cuda_fail(h, "refine graph launch");
      h->launches += h->refine_kernels;
      h->evals += refine_cost(h);
      return MGFWA_OK;
    }
  }
  return fail(h, MGFWA_EINVAL, "unknown phase %d", phase);
}

// Capture the phases explode .. select into h->gen_exec, on a private stream
// swapped in for the handle's (so the caller's stream is never in capture
// mode).  Nothing in them depends on the host's generation counter: the
// kernels read the generation from the device.
mgfwa_status capture_generation(mgfwa_t* h) {
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(h, "capture stream");
  cudaStream_t own = h->stream;
  const int64_t before = h->launches;
  cudaGraph_t graph = nullptr;
  mgfwa_status st = MGFWA_OK;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    h->stream = cs;
    h->capturing = true;
    for (int32_t ph = MGFWA_PHASE_EXPLODE; ph <= MGFWA_PHASE_SELECT && st == MGFWA_OK; ++ph) st = run_phase(h, ph);
    h->capturing = false;
    h->stream = own;
    ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && st == MGFWA_OK;
  }
  h->gen_kernels = h->launches - before;
  h->launches = before;
  if (!ok || !graph || cudaGraphInstantiate(&h->gen_exec, graph, 0) != cudaSuccess) {
    h->gen_exec = nullptr;
    if (st == MGFWA_OK) st = cuda_fail(h, "generation graph capture");
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  return st;
}

// One generation: explode .. select as one graph launch (direct launches
// while kernel groups are being timed), then the refinement when due.
mgfwa_status one_generation(mgfwa_t* h) {
  if (h->profiling) {
    for (int32_t ph = MGFWA_PHASE_EXPLODE; ph <= MGFWA_PHASE_REFINE; ++ph) {
      mgfwa_status st = run_phase(h, ph);
      if (st != MGFWA_OK) return st;
    }
    return MGFWA_OK;
  }
  if (h->cfg.lagged_guiding && !h->gv_ready) {
    // lagged multi-guiding's first generation has no vectors to guide from: it runs as written, kernel by
    // kernel, and the graph is captured at the next one
    for (int32_t ph = MGFWA_PHASE_EXPLODE; ph <= MGFWA_PHASE_REFINE; ++ph) {
      mgfwa_status st = run_phase(h, ph);
      if (st != MGFWA_OK) return st;
    }
    return MGFWA_OK;
  }
  if (!h->gen_exec) {
    mgfwa_status st = capture_generation(h);
    if (st != MGFWA_OK) return st;
  }
  h->gen += 1;
  if (cudaGraphLaunch(h->gen_exec, h->stream) != cudaSuccess) return cuda_fail(h, "generation graph launch");
  h->launches += h->gen_kernels;
  h->evals += h->P;
  return run_phase(h, MGFWA_PHASE_REFINE);
}

// The next generation fits: its sparks and, if due, its refinement.
bool budget_allows(const mgfwa_t* h) {
  if (h->cfg.n_shards > 1) {
    // a shard runs a generation when the whole run would (no refinement with shards)
    const int64_t P_run = (int64_t)h->mu_run * (h->p.lam + h->p.m);
    return (int64_t)h->mu_run + (int64_t)(h->gen + 1) * P_run <= h->cfg.eval_budget;
  }
  return h->evals + h->P + (refine_due(h, h->gen + 1) ? refine_cost(h) : 0) <= h->cfg.eval_budget;
}

mgfwa_status check_usable(mgfwa_t* h) {
  if (!h) return MGFWA_EINVAL;
  if (h->broken) return fail(h, MGFWA_ECUDA, "handle unusable after an earlier CUDA error: %s", h->err.c_str());
  return MGFWA_OK;
}

mgfwa_status check_status_word(mgfwa_t* h) {
  uint32_t st = 0;
  if (cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return cuda_fail(h, "synchronise");
  if (st != 0) {
    cudaMemsetAsync(h->status, 0, sizeof(uint32_t), h->stream);
    return fail(h, MGFWA_ETIMEOUT, "a bounded device wait gave up (code 0x%x)", st);
  }
  return MGFWA_OK;
}

mgfwa_status validate(const mgfwa_config* c, const mgfwa_objective* o) {
  if (!c || !o) return fail(nullptr, MGFWA_EINVAL, "null config or objective");
  if (c->dim < 1 || c->dim > (int64_t)1 << 31) return fail(nullptr, MGFWA_EINVAL, "dim %lld out of range", (long long)c->dim);
  if (!(c->lb < c->ub) || !std::isfinite(c->lb) || !std::isfinite(c->ub))
    return fail(nullptr, MGFWA_EINVAL, "bounds must be finite with lb < ub");
  if (c->n_fireworks < 1 || c->guiding_per_firework < 1 || c->sparks_per_firework < 2)
    return fail(nullptr, MGFWA_EINVAL, "need mu >= 1, m >= 1, lambda >= 2");
  if (c->sparks_per_firework % c->guiding_per_firework != 0)
    return fail(nullptr, MGFWA_EINVAL, "lambda (%d) must be a multiple of m (%d)", c->sparks_per_firework,
                c->guiding_per_firework);
  const int32_t g = c->sparks_per_firework / c->guiding_per_firework;
  if (g < 2 || g > 1024) return fail(nullptr, MGFWA_EINVAL, "group size lambda/m = %d must be in [2, 1024]", g);
  if (c->n_runs < 1) return fail(nullptr, MGFWA_EINVAL, "n_runs must be >= 1");
  if (c->elite_rescore < 0 || c->elite_rescore > 8 ||
      c->elite_rescore > c->sparks_per_firework + c->guiding_per_firework)
    return fail(nullptr, MGFWA_EINVAL, "elite_rescore must be in [0, min(8, lambda + m)]");
  if ((int64_t)c->n_runs * (c->n_fireworks + 1) > 65535 || c->sparks_per_firework > 65535)
    return fail(nullptr, MGFWA_EINVAL, "n_runs * (mu + 1) and lambda must each be <= 65535");
  const int64_t PA = (int64_t)c->n_runs * c->n_fireworks * (c->sparks_per_firework + c->guiding_per_firework);
  if (PA > (1 << 24)) return fail(nullptr, MGFWA_EINVAL, "n_runs mu (lambda + m) = %lld exceeds 2^24", (long long)PA);
  if (!(c->sigma > 0.0f) || !(c->sigma <= 0.5f)) return fail(nullptr, MGFWA_EINVAL, "sigma must be in (0, 0.5]");
  if (c->eval_budget < c->n_fireworks) return fail(nullptr, MGFWA_EINVAL, "eval_budget below the mu initial evaluations");
  if (c->precision != MGFWA_FP32 && c->precision != MGFWA_BF16 && c->precision != MGFWA_FP8 &&
      c->precision != MGFWA_FP32X3)
    return fail(nullptr, MGFWA_EINVAL, "precision %d not supported (FP32 = 0, BF16 = 1, FP8 = 2, FP32X3 = 3)",
                c->precision);
  if (c->precision == MGFWA_FP32X3 && o->kind != MGFWA_OBJ_NET_OUTPUT)
    return fail(nullptr, MGFWA_EINVAL, "FP32X3 is the testbed network objective's precision");
  if (c->refine_every < 0) return fail(nullptr, MGFWA_EINVAL, "refine_every must be >= 0");
  if (c->loser_out != 0 && c->loser_out != 1) return fail(nullptr, MGFWA_EINVAL, "loser_out must be 0 or 1");
  if (c->lagged_guiding != 0 && c->lagged_guiding != 1)
    return fail(nullptr, MGFWA_EINVAL, "lagged_guiding must be 0 or 1");
  if (c->n_shards < 0 || c->n_shards > c->n_fireworks)
    return fail(nullptr, MGFWA_EINVAL, "n_shards must be in [0, n_fireworks]");
  if (c->n_shards > 1) {
    if (c->shard_id < 0 || c->shard_id >= c->n_shards)
      return fail(nullptr, MGFWA_EINVAL, "shard_id must be in [0, n_shards)");
    if (c->loser_out || c->refine_every > 0)
      return fail(nullptr, MGFWA_EINVAL, "a shard of a run cannot use the loser-out tournament or refinement");
  } else if (c->shard_id != 0) {
    return fail(nullptr, MGFWA_EINVAL, "shard_id must be 0 without sharding");
  }
  if (c->refine_every > 0) {
    if (o->kind != MGFWA_OBJ_MLP_CE) return fail(nullptr, MGFWA_EINVAL, "refinement needs an MLP objective");
    if (c->refine_steps < 1 || c->refine_steps > 10000)
      return fail(nullptr, MGFWA_EINVAL, "refine_steps must be in [1, 10000]");
    if (!(c->refine_lr > 0.0f) || !std::isfinite(c->refine_lr))
      return fail(nullptr, MGFWA_EINVAL, "refine_lr must be positive and finite");
  }
  if (o->kind == MGFWA_OBJ_SPHERE) return MGFWA_OK;
  if (o->kind == MGFWA_OBJ_NET_OUTPUT) {
    const int32_t L = o->n_layers;
    if (L < 1 || L > kNetMaxLayers || !o->widths || (L > 1 && !o->acts) || !o->params)
      return fail(nullptr, MGFWA_EINVAL, "network objective needs 1 to %d layers, widths, acts and params",
                  kNetMaxLayers);
    for (int l = 0; l <= L; ++l)
      if (o->widths[l] < 1 || o->widths[l] > 4096)
        return fail(nullptr, MGFWA_EINVAL, "network width %d out of [1, 4096]", o->widths[l]);
    if (o->widths[0] != c->dim || o->widths[L] != 1)
      return fail(nullptr, MGFWA_EINVAL, "network widths must run from dim (%lld) to 1", (long long)c->dim);
    for (int l = 0; l + 1 < L; ++l)
      if (o->acts[l] != MGFWA_ACT_TANH && o->acts[l] != MGFWA_ACT_RELU && o->acts[l] != MGFWA_ACT_GELU)
        return fail(nullptr, MGFWA_EINVAL, "unknown activation %d", o->acts[l]);
    if (c->precision != MGFWA_FP32 && c->precision != MGFWA_FP32X3)
      return fail(nullptr, MGFWA_EINVAL, "the network objective runs in FP32 or FP32X3");
    if (c->precision == MGFWA_FP32X3) {
      bool any = false;
      for (int l = 0; l < L; ++l) any = any || net_x3_layer(o->widths[l], o->widths[l + 1]);
      if (!any)
        return fail(nullptr, MGFWA_EINVAL,
                    "FP32X3: no layer of this network has fan_in % 8 == 0 and an even fan_out >= 16");
    }
    return MGFWA_OK;
  }
  if (o->kind != MGFWA_OBJ_MLP_CE) return fail(nullptr, MGFWA_EINVAL, "unknown objective kind %d", o->kind);
  if (o->n_layers < 2 || o->n_layers > 3 || !o->widths || !o->acts || !o->X || !o->y)
    return fail(nullptr, MGFWA_EINVAL, "MLP objective needs 2 or 3 layers, widths, acts, X and y");
  if (o->n_samples < 1 || o->n_samples > mgfwa::kMaxSamples)
    return fail(nullptr, MGFWA_EINVAL, "n_samples must be in [1, %lld]", (long long)mgfwa::kMaxSamples);
  int64_t params = 0;
  for (int l = 0; l < o->n_layers; ++l) {
    if (o->widths[l] < 1 || o->widths[l + 1] < 1) return fail(nullptr, MGFWA_EINVAL, "layer widths must be >= 1");
    params += (int64_t)o->widths[l] * o->widths[l + 1] + o->widths[l + 1];
  }
  if (params != c->dim)
    return fail(nullptr, MGFWA_EINVAL, "dim %lld != MLP parameter count %lld", (long long)c->dim, (long long)params);
  if (o->widths[0] % 8 != 0) return fail(nullptr, MGFWA_EINVAL, "d_in (%d) must be a multiple of 8", o->widths[0]);
  for (int l = 1; l < o->n_layers; ++l) {
    if (o->widths[l] > 192) return fail(nullptr, MGFWA_EINVAL, "hidden width %d above 192", o->widths[l]);
    if (o->acts[l - 1] != MGFWA_ACT_TANH && o->acts[l - 1] != MGFWA_ACT_RELU)
      return fail(nullptr, MGFWA_EINVAL, "unknown activation %d", o->acts[l - 1]);
  }
  if (o->widths[o->n_layers] > 32 || o->widths[o->n_layers] < 2)
    return fail(nullptr, MGFWA_EINVAL, "class count must be in [2, 32]");
  const int C = o->widths[o->n_layers];
  for (int64_t n = 0; n < o->n_samples; ++n)
    if (o->y[n] < 0 || o->y[n] >= C) return fail(nullptr, MGFWA_EINVAL, "label y[%lld] out of range", (long long)n);
  if ((c->precision == MGFWA_BF16 || c->precision == MGFWA_FP8) && !tc_supported(o->widths, o->n_layers))
    return fail(nullptr, MGFWA_EINVAL,
                "tensor-core paths need d_in %% 8 == 0 and two layers with h1 in {32, 64, 128} (<= 32 classes) or "
                "three with (h1, h2) in {(128, 64), (64, 32)} (<= 16 classes)");
  if (c->precision == MGFWA_FP8 && o->widths[0] % 16 != 0)
    return fail(nullptr, MGFWA_EINVAL, "FP8 path needs d_in %% 16 == 0");
  return MGFWA_OK;
}

// Next 256-byte-aligned slice of `count` elements; with a null base only the
// offsets are computed (the sizing pass).
template <typename T>
T* carve(char*& cur, size_t count) {
  T* p = reinterpret_cast<T*>(cur);
  cur += round_up((int64_t)(count * sizeof(T)), 256);
  return p;
}

// The library's device memory pool (one per device, created on first use):
// arenas are allocated and freed in stream order from it, and freed memory
// stays in the pool for the next handle instead of returning to the driver,
// so creating a handle of a size seen before costs no driver allocation.
cudaMemPool_t arena_pool(int device) {
  constexpr int kMaxDevices = 64;
  static cudaMemPool_t pools[kMaxDevices] = {};
  static bool tried[kMaxDevices] = {};
  if (device < 0 || device >= kMaxDevices) return nullptr;
  if (!tried[device]) {
    tried[device] = true;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      pools[device] = pool;
    }
    cudaGetLastError();
  }
  return pools[device];
}

void arena_free(mgfwa_t* h) {
  if (!h->arena) return;
  if (h->pooled)
    cudaFreeAsync(h->arena, h->stream);
  else
    cudaFree(h->arena);
  h->arena = nullptr;
}

// FNV-1a over the configuration (but its budget), the network shape and
// (every 61st element of) the batch: a checkpoint is refused by a handle of
// another problem.
uint64_t problem_fingerprint(const mgfwa_config* cfg, const mgfwa_objective* obj) {
  uint64_t f = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) f = (f ^ b[i]) * 1099511628211ull;
  };
  // field by field (struct padding is not part of the problem); the budget is
  // left out so that a resumed run may be given a larger one
  mix(&cfg->dim, sizeof(cfg->dim));
  mix(&cfg->lb, sizeof(cfg->lb));
  mix(&cfg->ub, sizeof(cfg->ub));
  mix(&cfg->n_fireworks, sizeof(cfg->n_fireworks));
  mix(&cfg->sparks_per_firework, sizeof(cfg->sparks_per_firework));
  mix(&cfg->guiding_per_firework, sizeof(cfg->guiding_per_firework));
  mix(&cfg->sigma, sizeof(cfg->sigma));
  mix(&cfg->boost, sizeof(cfg->boost));
  mix(&cfg->amp_init, sizeof(cfg->amp_init));
  mix(&cfg->c_amplify, sizeof(cfg->c_amplify));
  mix(&cfg->c_reduce, sizeof(cfg->c_reduce));
  mix(&cfg->seed, sizeof(cfg->seed));
  mix(&cfg->precision, sizeof(cfg->precision));
  mix(&cfg->elite_rescore, sizeof(cfg->elite_rescore));
  mix(&cfg->n_runs, sizeof(cfg->n_runs));
  mix(&cfg->refine_every, sizeof(cfg->refine_every));
  mix(&cfg->refine_steps, sizeof(cfg->refine_steps));
  mix(&cfg->refine_lr, sizeof(cfg->refine_lr));
  mix(&cfg->loser_out, sizeof(cfg->loser_out));
  mix(&cfg->lagged_guiding, sizeof(cfg->lagged_guiding));
  mix(&cfg->shard_id, sizeof(cfg->shard_id));
  mix(&cfg->n_shards, sizeof(cfg->n_shards));
  mix(&obj->kind, sizeof(obj->kind));
  mix(&obj->n_layers, sizeof(obj->n_layers));
  if (obj->kind == MGFWA_OBJ_MLP_CE) {
    mix(obj->widths, sizeof(int32_t) * (size_t)(obj->n_layers + 1));
    mix(obj->acts, sizeof(int32_t) * (size_t)(obj->n_layers > 1 ? obj->n_layers - 1 : 0));
    mix(&obj->n_samples, sizeof(obj->n_samples));
    const int64_t nx = obj->n_samples * (int64_t)obj->widths[0];
    for (int64_t e = 0; e < nx; e += 61) mix(obj->X + e, sizeof(float));
    for (int64_t e = 0; e < obj->n_samples; e += 61) mix(obj->y + e, sizeof(int32_t));
  } else if (obj->kind == MGFWA_OBJ_NET_OUTPUT) {
    mix(obj->widths, sizeof(int32_t) * (size_t)(obj->n_layers + 1));
    if (obj->n_layers > 1) mix(obj->acts, sizeof(int32_t) * (size_t)(obj->n_layers - 1));
    int64_t n = 0;
    for (int l = 0; l < obj->n_layers; ++l) n += (int64_t)obj->widths[l] * obj->widths[l + 1] + obj->widths[l + 1];
    for (int64_t e = 0; e < n; e += 61) mix(obj->params + e, sizeof(float));
  }
  return f;
}

// Fill the handle's problem description and sizes from a validated
// configuration (no allocation).
void plan_handle(mgfwa_t* h, const mgfwa_config* cfg, const mgfwa_objective* obj) {
  h->cfg = *cfg;
  h->kind = obj->kind;
  cudaGetDevice(&h->device);

  Problem& p = h->p;
  p.D = cfg->dim;
  p.Dp = round_up(cfg->dim, 64);
  p.lb = cfg->lb;
  p.ub = cfg->ub;
  p.mu = cfg->n_fireworks;
  p.fw_off = 0;
  h->mu_run = cfg->n_fireworks;
  if (cfg->n_shards > 1) {
    // this shard's fireworks: [shard_id mu / n_shards, (shard_id + 1) mu / n_shards) of the run
    const int64_t lo = (int64_t)cfg->shard_id * cfg->n_fireworks / cfg->n_shards;
    const int64_t hi = (int64_t)(cfg->shard_id + 1) * cfg->n_fireworks / cfg->n_shards;
    p.mu = (int32_t)(hi - lo);
    p.fw_off = (int32_t)lo;
  }
  p.lam = cfg->sparks_per_firework;
  p.m = cfg->guiding_per_firework;
  p.g = p.lam / p.m;
  p.k = subset_size(cfg->sigma, p.g);
  p.beta = cfg->boost;
  p.amp0 = cfg->amp_init > 0.0f ? cfg->amp_init : cfg->ub - cfg->lb;
  p.c_a = cfg->c_amplify;
  p.c_r = cfg->c_reduce;
  p.B = cfg->n_runs;
  p.seed = cfg->seed;
  h->P = (int64_t)p.mu * (p.lam + p.m);
  // loser-out tournament: the generations the budget allows at P evaluations each (0 = off)
  p.lo_gmax = 0;
  if (cfg->loser_out) {
    const int64_t g = (cfg->eval_budget - p.mu) / h->P;
    p.lo_gmax = (int32_t)(g < 1 ? 1 : (g > (1 << 30) ? (1 << 30) : g));
  }
  h->PA = (int64_t)p.B * h->P;

  Mlp& mlp = h->mlp;
  std::memset(&mlp, 0, sizeof(mlp));
  int64_t N = 0;
  if (obj->kind == MGFWA_OBJ_MLP_CE) {
    mlp.n_layers = obj->n_layers;
    for (int l = 0; l <= obj->n_layers; ++l) mlp.widths[l] = obj->widths[l];
    for (int l = 0; l + 1 < obj->n_layers; ++l) mlp.acts[l] = obj->acts[l];
    int64_t off = 0;
    for (int l = 0; l < obj->n_layers; ++l) {
      mlp.w_off[l] = off;
      off += (int64_t)obj->widths[l] * obj->widths[l + 1];
      mlp.b_off[l] = off;
      off += obj->widths[l + 1];
    }
    mlp.N = obj->n_samples;
    mlp.w1_elems = (int64_t)obj->widths[0] * obj->widths[1];
    N = obj->n_samples;
    h->mtiles = (int32_t)((N + 127) / 128);
  } else {
    h->mtiles = 1;
  }
  NetOut& net = h->net;
  std::memset(&net, 0, sizeof(net));
  h->net_count = 0;
  if (obj->kind == MGFWA_OBJ_NET_OUTPUT) {
    net.n_layers = obj->n_layers;
    net.hmax = 1;
    int64_t off = 0;
    for (int l = 0; l <= obj->n_layers; ++l) {
      net.widths[l] = obj->widths[l];
      if (obj->widths[l] > net.wmax) net.wmax = obj->widths[l];
      if (l > 0 && l < obj->n_layers && obj->widths[l] > net.hmax) net.hmax = obj->widths[l];
    }
    for (int l = 0; l < obj->n_layers; ++l) {
      if (l + 1 < obj->n_layers) net.acts[l] = obj->acts[l];
      net.w_off[l] = off;
      off += (int64_t)obj->widths[l] * obj->widths[l + 1];
      net.b_off[l] = off;
      off += obj->widths[l + 1];
    }
    h->net_count = off;
  }
  h->fingerprint = problem_fingerprint(cfg, obj);
  h->want_op = obj->kind == MGFWA_OBJ_MLP_CE && (cfg->precision == MGFWA_BF16 || cfg->precision == MGFWA_FP8);
  h->op_kind = !h->want_op ? kOpNone : (cfg->precision == MGFWA_FP8 ? kOpFp8 : kOpBf16);
  if (h->op_kind == kOpFp8) {
    // E4M3 scales: X by its largest magnitude, the weights by the box bound
    // (every coordinate lies in [lb, ub], so no spark exceeds it)
    float amax = 0.0f;
    for (int64_t e = 0; e < obj->n_samples * (int64_t)obj->widths[0]; ++e) amax = std::fmax(amax, std::fabs(obj->X[e]));
    const float bound = std::fmax(std::fabs(cfg->lb), std::fabs(cfg->ub));
    h->inv_x = amax > 0.0f ? 448.0f / amax : 1.0f;
    h->inv_w = 448.0f / bound;
    h->op_scale = (float)(1.0 / ((double)h->inv_x * (double)h->inv_w));
  }
  h->refine = cfg->refine_every > 0 && obj->kind == MGFWA_OBJ_MLP_CE;
  const bool rescore = h->want_op && cfg->elite_rescore > 0;
  if (h->refine || rescore) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      sms = 152;  // sizing without a device: a GB300's SM count
    }
    if (h->refine) h->gp = grad_plan(mlp, p.B, sms);
    if (rescore) h->rescore_plan = grad_plan(mlp, p.B * p.mu * cfg->elite_rescore, sms, true);
  }
}

// One arena for all device state; sizing (null base) and carving share this
// one layout pass.
size_t carve_all(mgfwa_t* h, char* base) {
  const Problem& p = h->p;
  const Mlp& mlp = h->mlp;
  const mgfwa_config* cfg = &h->cfg;
  const bool want_op = h->want_op;
  const int64_t N = mlp.N, d_in = mlp.widths[0];
  char* cur = base;
  h->X = carve<float>(cur, N * d_in);
  const int64_t esize = h->op_kind == kOpFp8 ? 1 : 2;
  h->Xop = want_op ? carve<uint8_t>(cur, N * d_in * esize) : nullptr;
  h->y = carve<int32_t>(cur, N);
  const int64_t F = (int64_t)p.B * p.mu;  // fireworks of all runs
  h->fw_x = carve<float>(cur, F * p.Dp);
  h->fw_amp = carve<float>(cur, F);
  h->fw_f = carve<float>(cur, F);
  h->sparks = carve<float>(cur, h->PA * p.Dp);
  h->op = want_op ? carve<uint8_t>(cur, h->PA * mlp.w1_elems * esize) : nullptr;
  // the CTA-pair fitness kernel reads W2 as BF16 from its own copy
  const bool pair = want_op && tc_pair_supported(mlp.widths, mlp.n_layers);
  h->w2_rows = pair ? tc_pair_w2_rows(mlp.widths, mlp.n_layers) : 0;
  h->w2op = h->w2_rows ? carve<uint16_t>(cur, h->PA * h->w2_rows * mlp.widths[1]) : nullptr;
  h->w3_rows = pair && mlp.n_layers == 3 ? tc_pair_logit_rows(mlp.widths[3]) : 0;
  h->w3op = h->w3_rows ? carve<uint16_t>(cur, h->PA * h->w3_rows * mlp.widths[2]) : nullptr;
  h->fit = carve<float>(cur, h->PA);
  h->partial = carve<float>(cur, (size_t)h->mtiles * h->PA);
  h->top = carve<int32_t>(cur, F * p.m * p.k);
  h->bottom = carve<int32_t>(cur, F * p.m * p.k);
  h->winner = carve<int32_t>(cur, F + p.B + 1);  // per firework, per run, the generation (the selection's decisions)
  h->f_old = carve<float>(cur, F);
  h->loser = carve<int32_t>(cur, F);
  h->gv = cfg->lagged_guiding ? carve<float>(cur, F * p.m * p.Dp) : nullptr;
  h->elite = carve<int32_t>(cur, F * (cfg->elite_rescore > 0 ? cfg->elite_rescore : 1));
  const bool rescore = want_op && cfg->elite_rescore > 0;
  h->rescore_scratch = rescore ? carve<float>(cur, (size_t)h->rescore_plan.floats) : nullptr;
  // the FP32-accurate tensor-core first layer's BF16 operand parts (sized by shape, whatever the device)
  const bool l1 = (rescore || h->refine) && h->kind == MGFWA_OBJ_MLP_CE && l1_fp32x3_supported(mlp);
  h->l1_xs = l1 ? carve<uint32_t>(cur, (size_t)l1_fp32x3_x_words(mlp)) : nullptr;
  h->rescore_ws = l1 && rescore ? carve<uint32_t>(cur, (size_t)l1_fp32x3_w_words(mlp, h->rescore_plan.R)) : nullptr;
  h->refine_ws = l1 && h->refine ? carve<uint32_t>(cur, (size_t)l1_fp32x3_w_words(mlp, p.B)) : nullptr;
  if (h->kind == MGFWA_OBJ_NET_OUTPUT) {
    h->net.params = carve<float>(cur, (size_t)h->net_count);
    h->net_act = h->net.n_layers > 1 ? carve<float>(cur, (size_t)(2 * h->PA * h->net.hmax)) : nullptr;
    h->net_x3_buf =
        h->cfg.precision == MGFWA_FP32X3 ? carve<uint32_t>(cur, (size_t)net_x3_words(h->net, h->PA)) : nullptr;
  }
  h->best_x = carve<float>(cur, (int64_t)p.B * p.Dp);
  h->best_f = carve<float>(cur, p.B);
  h->ce64 = carve<double>(cur, N > 0 ? N : 1);
  h->f64 = carve<double>(cur, 1);
  h->status = carve<uint32_t>(cur, 1);
  h->gens_done = carve<uint32_t>(cur, 1);
  if (h->refine) {
    h->rw = carve<float>(cur, (int64_t)p.B * p.Dp);
    h->rg = carve<float>(cur, (int64_t)p.B * p.Dp);
    h->rf = carve<float>(cur, p.B);
    h->relite = carve<int32_t>(cur, p.B);
    h->rflags = carve<int32_t>(cur, p.B);
    h->gscratch = carve<float>(cur, (size_t)h->gp.floats);
  }
  return (size_t)(cur - base);
}

}  // namespace

extern "C" {

mgfwa_status mgfwa_config_init(mgfwa_config* cfg) {
  if (!cfg) return MGFWA_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->sigma = 0.2f;
  cfg->boost = 1.0f;
  cfg->amp_init = 0.0f;
  cfg->c_amplify = 1.2f;
  cfg->c_reduce = 0.9f;
  cfg->precision = MGFWA_FP32;
  cfg->elite_rescore = 2;
  cfg->n_runs = 1;
  return MGFWA_OK;
}

mgfwa_status mgfwa_footprint(const mgfwa_config* cfg, const mgfwa_objective* obj, int64_t* bytes_out) {
  if (!bytes_out) return fail(nullptr, MGFWA_EINVAL, "null output pointer");
  g_create_error.clear();
  mgfwa_status st = validate(cfg, obj);
  if (st != MGFWA_OK) return st;
  mgfwa_t* h = new (std::nothrow) mgfwa_t();
  if (!h) return fail(nullptr, MGFWA_ENOMEM, "host allocation failed");
  plan_handle(h, cfg, obj);
  *bytes_out = (int64_t)carve_all(h, nullptr);
  delete h;
  return MGFWA_OK;
}

mgfwa_status mgfwa_create(const mgfwa_config* cfg, const mgfwa_objective* obj, void* cuda_stream, mgfwa_t** out) {
  if (!out) return fail(nullptr, MGFWA_EINVAL, "null output handle pointer");
  *out = nullptr;
  g_create_error.clear();
  TRACE("create: validate");
  mgfwa_status st = validate(cfg, obj);
  if (st != MGFWA_OK) return st;
  TRACE("create: validated");
  mgfwa_t* h = new (std::nothrow) mgfwa_t();
  if (!h) return fail(nullptr, MGFWA_ENOMEM, "host allocation failed");
  plan_handle(h, cfg, obj);
  const Problem& p = h->p;
  Mlp& mlp = h->mlp;
  const bool want_op = h->want_op;
  const int64_t N = mlp.N, d_in = mlp.widths[0];
  const size_t bytes = carve_all(h, nullptr);
  h->arena_bytes = bytes;
  TRACE("create: arena %zu bytes, Dp %lld, P %lld, N %lld, d_in %lld", bytes, (long long)p.Dp, (long long)h->P,
        (long long)N, (long long)d_in);

  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail(nullptr, MGFWA_ECUDA, "cudaStreamCreate failed");
    }
    h->own_stream = true;
  }
  {
    void* mem = nullptr;
    cudaMemPool_t pool = arena_pool(h->device);
    if (pool && cudaMallocFromPoolAsync(&mem, bytes, pool, h->stream) == cudaSuccess) {
      h->pooled = true;
    } else {
      cudaGetLastError();
      mem = nullptr;
      if (cudaMalloc(&mem, bytes) != cudaSuccess) mem = nullptr;
    }
    h->arena = static_cast<char*>(mem);
  }
  if (!h->arena) {
    cudaGetLastError();
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return fail(nullptr, MGFWA_ENOMEM, "device allocation of %zu bytes failed", bytes);
  }
  if (carve_all(h, h->arena) != bytes) {
    arena_free(h);
    cudaStreamSynchronize(h->stream);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return fail(nullptr, MGFWA_EINVAL, "internal: arena layout mismatch");
  }

  mlp.X = h->X;
  mlp.Xop = h->Xop;
  mlp.y = h->y;

  auto bail = [&](mgfwa_status s) {
    std::string e = h->err;
    mgfwa_destroy(h);
    g_create_error = e;
    return s;
  };
  TRACE("create: allocated");
  if (cudaMemsetAsync(h->arena, 0, bytes, h->stream) != cudaSuccess) return bail(cuda_fail(h, "memset arena"));
  TRACE("create: memset");
  if (N > 0) {
    if (cudaMemcpyAsync(h->X, obj->X, sizeof(float) * N * d_in, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->y, obj->y, sizeof(int32_t) * N, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      return bail(cuda_fail(h, "copy batch"));
    if (want_op) CREATE_LAUNCH(launch_f32_to_op(h->X, N * d_in, h->op_kind, h->inv_x, h->Xop, h->stream), "X operand");
  }
  if (h->kind == MGFWA_OBJ_NET_OUTPUT &&
      cudaMemcpyAsync(const_cast<float*>(h->net.params), obj->params, sizeof(float) * h->net_count,
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return bail(cuda_fail(h, "copy network parameters"));
  if (h->net_x3_buf) {
    // FP32X3: the tensor-core layers' maps, and the weights' BF16 parts once
    if (!net_x3_plan(h->net_x3, h->net, h->PA, h->net_x3_buf))
      return bail(fail(h, MGFWA_EINVAL, "FP32X3 needs a Blackwell (sm_10x) GPU"));
    CREATE_LAUNCH(launch_net_x3_split_w(h->net_x3, h->net, h->stream), "FP32X3 weight parts");
  }
  if (h->w2op &&
      cudaMemsetAsync(h->w2op, 0, sizeof(uint16_t) * h->PA * h->w2_rows * h->mlp.widths[1], h->stream) != cudaSuccess)
    return bail(cuda_fail(h, "clear the W2 copy"));
  if (h->w3op &&
      cudaMemsetAsync(h->w3op, 0, sizeof(uint16_t) * h->PA * h->w3_rows * h->mlp.widths[2], h->stream) != cudaSuccess)
    return bail(cuda_fail(h, "clear the W3 copy"));
  if (want_op) {
    st = tc_plan(h->tc, h->mlp, op_rows(h, 0), h->sparks, p.Dp, h->PA);
    if (st != MGFWA_OK) {
      h->err = tc_last_error();
      return bail(st);
    }
    if (tc_prepare(h->tc, h->mlp) != cudaSuccess) return bail(cuda_fail(h, "tensor-core kernel attributes"));
    if (h->tc.pair) {
      // the pair kernel's tile shape and depth, timed on one explosion's worth of rows (all give the same
      // fitness; the rows are not yet the run's)
      st = tc_pair_tune(h->tc, h->mlp, h->sparks, p.Dp, (int32_t)((int64_t)p.B * p.mu * p.lam), h->op_scale,
                        h->partial, h->status, h->stream);
      if (st != MGFWA_OK) {
        h->err = tc_last_error();
        return bail(st);
      }
    }
  }
  // the FP32-accurate first layer of the elite re-score and of the refinement on the tensor cores
  // (where the shape allows; otherwise they keep the CUDA-core products)
  if (h->rescore_ws)
    l1_fp32x3_plan(h->rescore_l1, h->mlp, h->sparks, p.Dp, h->rescore_plan.R, h->l1_xs, h->rescore_ws);
  if (h->refine_ws) l1_fp32x3_plan(h->refine_l1, h->mlp, h->rw, p.Dp, p.B, h->l1_xs, h->refine_ws);
  if (h->rescore_l1.ready || h->refine_l1.ready)
    CREATE_LAUNCH(launch_l1_split_x(h->rescore_l1.ready ? h->rescore_l1 : h->refine_l1, h->mlp, h->stream),
                  "X parts");
  TRACE("create: batch copied");
  // Algorithm 1, init: mu fireworks uniform in the box, evaluated.
  CREATE_LAUNCH(launch_init(p, h->fw_x, h->fw_amp, h->stream), "init");
  TRACE("create: init launched");
  const int32_t F = p.B * p.mu;
  if (cudaMemcpy2DAsync(h->sparks, sizeof(float) * p.Dp, h->fw_x, sizeof(float) * p.Dp, sizeof(float) * p.Dp, F,
                        cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
    return bail(cuda_fail(h, "stage init rows"));
  if (want_op) CREATE_LAUNCH(launch_to_operand(h->sparks, p.Dp, F, op_rows(h, 0), h->stream), "init operand");
  TRACE("create: staged");
  // with an FP32 elite re-score the initial fireworks are scored in FP32 too
  st = eval_rows(h, 0, F, cfg->elite_rescore > 0 && h->kind == MGFWA_OBJ_MLP_CE ? MGFWA_FP32 : cfg->precision);
  if (st != MGFWA_OK) return bail(st);
  TRACE("create: evaluated");
  if (cudaMemcpyAsync(h->fw_f, h->fit, sizeof(float) * F, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
    return bail(cuda_fail(h, "init fitness"));
  CREATE_LAUNCH(launch_run_best_init(p, h->fw_x, h->fw_f, h->best_x, h->best_f, h->stream), "init best");
  h->evals = p.mu;
  TRACE("create: best launched");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(cuda_fail(h, "create synchronise"));
  TRACE("create: synchronised");
  st = check_status_word(h);
  if (st != MGFWA_OK) return bail(st);
  *out = h;
  return MGFWA_OK;
}

mgfwa_status mgfwa_step(mgfwa_t* h, int32_t n_generations) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  if (n_generations < 0) return fail(h, MGFWA_EINVAL, "negative generation count");
  if (h->next_phase != MGFWA_PHASE_EXPLODE) return fail(h, MGFWA_EINVAL, "a debug generation is in progress");
  if (n_generations > 0 && !budget_allows(h)) return fail(h, MGFWA_EBUDGET, "budget spent");
  for (int32_t i = 0; i < n_generations && budget_allows(h); ++i) {
    st = one_generation(h);
    if (st != MGFWA_OK) return st;
  }
  return MGFWA_OK;
}

mgfwa_status mgfwa_run(mgfwa_t* h) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  if (h->next_phase != MGFWA_PHASE_EXPLODE) return fail(h, MGFWA_EINVAL, "a debug generation is in progress");
  while (budget_allows(h)) {
    st = one_generation(h);
    if (st != MGFWA_OK) return st;
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "run synchronise");
  return check_status_word(h);
}

mgfwa_status mgfwa_best_run(mgfwa_t* h, int32_t run, float* x_out, double* f_out, int64_t* evals_out) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  if (run < 0 || run >= h->p.B) return fail(h, MGFWA_EINVAL, "run %d out of range [0, %d)", run, h->p.B);
  const float* bx = h->best_x + (int64_t)run * h->p.Dp;
  if (f_out) {
    if (h->kind == MGFWA_OBJ_SPHERE)
      MG_LAUNCH(h, launch_sphere_f64(bx, h->p.D, h->f64, h->stream), "FP64 sphere");
    else if (h->kind == MGFWA_OBJ_NET_OUTPUT)
      MG_LAUNCH(h, launch_net_output_f64(h->net, bx, h->f64, h->stream), "FP64 network output");
    else
      MG_LAUNCH(h, launch_fitness_f64(h->mlp, bx, h->ce64, h->f64, h->stream), "FP64 fitness");
    if (cudaMemcpyAsync(f_out, h->f64, sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
      return cuda_fail(h, "read best fitness");
  }
  if (x_out && cudaMemcpyAsync(x_out, bx, sizeof(float) * h->p.D, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return cuda_fail(h, "read best position");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "best synchronise");
  if (evals_out) *evals_out = h->evals;
  return check_status_word(h);
}

// ---------------------------------------------------------------------------
// The run's best over shards.

mgfwa_status mgfwa_reduce_best_keys(const mgfwa_best_key* keys, int32_t n, mgfwa_best_key* out) {
  if (!keys || !out || n < 1) return MGFWA_EINVAL;
  auto before = [](const mgfwa_best_key& a, const mgfwa_best_key& b) {
    const float fa = std::isnan(a.f) ? INFINITY : a.f, fb = std::isnan(b.f) ? INFINITY : b.f;
    if (fa != fb) return fa < fb;
    if (std::isnan(a.f) != std::isnan(b.f)) return !std::isnan(a.f);  // +inf before NaN
    if (a.shard != b.shard) return a.shard < b.shard;
    return a.run < b.run;
  };
  mgfwa_best_key best = keys[0];
  for (int32_t i = 1; i < n; ++i)
    if (before(keys[i], best)) best = keys[i];
  *out = best;
  return MGFWA_OK;
}

mgfwa_status mgfwa_shard_key(mgfwa_t* h, int32_t run, mgfwa_best_key* key_out) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  if (!key_out || run < 0 || run >= h->p.B) return fail(h, MGFWA_EINVAL, "shard key: bad run or null output");
  float f = 0.0f;
  if (cudaMemcpyAsync(&f, h->best_f + run, sizeof(float), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return cuda_fail(h, "read the run's best");
  key_out->f = f;
  key_out->shard = h->cfg.n_shards > 1 ? h->cfg.shard_id : 0;
  key_out->run = run;
  key_out->pad = 0;
  return check_status_word(h);
}

mgfwa_status mgfwa_set_reduce_best(mgfwa_t* h, mgfwa_reduce_best_fn fn, void* ctx) {
  if (!h) return MGFWA_EINVAL;
  h->reduce_best = fn;
  h->reduce_ctx = fn ? ctx : nullptr;
  return MGFWA_OK;
}

mgfwa_status mgfwa_global_best_key(mgfwa_t* h, int32_t run, mgfwa_best_key* key_out) {
  mgfwa_status st = mgfwa_shard_key(h, run, key_out);
  if (st != MGFWA_OK || !h->reduce_best) return st;
  if (h->reduce_best(h->reduce_ctx, key_out) != 0) return fail(h, MGFWA_ECUDA, "the reduce_best hook failed");
  return MGFWA_OK;
}

mgfwa_status mgfwa_best(mgfwa_t* h, float* x_out, double* f_out, int64_t* evals_out) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  int32_t run = 0;
  if (h->p.B > 1) {
    // the run whose FP32 best-so-far is lowest (the first on ties)
    std::vector<float> bf((size_t)h->p.B);
    if (cudaMemcpyAsync(bf.data(), h->best_f, sizeof(float) * h->p.B, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return cuda_fail(h, "read run bests");
    for (int32_t b = 1; b < h->p.B; ++b) {
      const float kb = std::isnan(bf[b]) ? INFINITY : bf[b];
      const float kr = std::isnan(bf[run]) ? INFINITY : bf[run];
      if (kb < kr) run = b;
    }
  }
  return mgfwa_best_run(h, run, x_out, f_out, evals_out);
}

mgfwa_status mgfwa_evaluate(mgfwa_t* h, const float* xs, int64_t count, int32_t precision, float* f_out) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  if (!xs || !f_out || count < 0 || count > h->PA)
    return fail(h, MGFWA_EINVAL, "evaluate: bad arguments (count <= %lld)", (long long)h->PA);
  if (precision != MGFWA_FP32 && precision != MGFWA_BF16 && precision != MGFWA_FP8 && precision != MGFWA_FP32X3)
    return fail(h, MGFWA_EINVAL, "evaluate: bad precision");
  if (precision == MGFWA_FP32X3 && !h->net_x3.ready)
    return fail(h, MGFWA_EINVAL, "evaluate: FP32X3 needs a testbed-network handle created in FP32X3");
  if (use_tc(h, precision) && (!h->op || precision != h->cfg.precision))
    return fail(h, MGFWA_EINVAL, "evaluate: the handle's tensor-core operand is not of precision %d", precision);
  if (h->next_phase != MGFWA_PHASE_EXPLODE) return fail(h, MGFWA_EINVAL, "a debug generation is in progress");
  if (count == 0) return MGFWA_OK;
  if (cudaMemcpy2DAsync(h->sparks, sizeof(float) * h->p.Dp, xs, sizeof(float) * h->p.D, sizeof(float) * h->p.D, count,
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return cuda_fail(h, "evaluate: copy rows");
  if (use_tc(h, precision))
    MG_LAUNCH(h, launch_to_operand(h->sparks, h->p.Dp, (int32_t)count, op_rows(h, 0), h->stream), "evaluate operand");
  st = eval_rows(h, 0, (int32_t)count, precision);
  if (st != MGFWA_OK) return st;
  if (cudaMemcpyAsync(f_out, h->fit, sizeof(float) * count, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return cuda_fail(h, "evaluate: read fitness");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "evaluate synchronise");
  return check_status_word(h);
}

// ---------------------------------------------------------------------------
// Checkpoints: header, then fw_x [B*mu][D], fw_amp, fw_f [B*mu], best_x [B][D],
// best_f [B] (FP32), packed.

namespace {
struct CkptHeader {
  uint64_t magic;
  uint64_t fingerprint;
  int64_t evals;
  int64_t launches;
  int32_t gen;
  uint32_t gens_done;
  int64_t payload_bytes;
};
constexpr uint64_t kCkptMagic = 0x31544b43415746ull;  // "FWACKT1"

int64_t ckpt_payload(const mgfwa_t* h) {
  const int64_t F = (int64_t)h->p.B * h->p.mu, B = h->p.B, D = h->p.D;
  return (int64_t)sizeof(float) * (F * D + 2 * F + B * D + B);
}
}  // namespace

mgfwa_status mgfwa_checkpoint_size(const mgfwa_t* h, int64_t* bytes) {
  if (!h || !bytes) return MGFWA_EINVAL;
  *bytes = (int64_t)sizeof(CkptHeader) + ckpt_payload(h);
  return MGFWA_OK;
}

mgfwa_status mgfwa_checkpoint_save(mgfwa_t* h, void* host, int64_t bytes) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  const int64_t need = (int64_t)sizeof(CkptHeader) + ckpt_payload(h);
  if (!host || bytes != need) return fail(h, MGFWA_EINVAL, "checkpoint: buffer must hold %lld bytes", (long long)need);
  if (h->next_phase != MGFWA_PHASE_EXPLODE) return fail(h, MGFWA_EINVAL, "a debug generation is in progress");
  if (h->cfg.lagged_guiding) return fail(h, MGFWA_EINVAL, "checkpoint: not supported with lagged_guiding");
  CkptHeader hd{kCkptMagic, h->fingerprint, h->evals, h->launches, h->gen, 0u, ckpt_payload(h)};
  char* out = static_cast<char*>(host) + sizeof(CkptHeader);
  const int64_t F = (int64_t)h->p.B * h->p.mu, B = h->p.B;
  const size_t rb = sizeof(float) * h->p.D, pitch = sizeof(float) * h->p.Dp;
  cudaError_t e = cudaMemcpyAsync(&hd.gens_done, h->gens_done, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(out, rb, h->fw_x, pitch, rb, F, cudaMemcpyDeviceToHost, h->stream);
  out += rb * F;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->fw_amp, sizeof(float) * F, cudaMemcpyDeviceToHost, h->stream);
  out += sizeof(float) * F;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->fw_f, sizeof(float) * F, cudaMemcpyDeviceToHost, h->stream);
  out += sizeof(float) * F;
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(out, rb, h->best_x, pitch, rb, B, cudaMemcpyDeviceToHost, h->stream);
  out += rb * B;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->best_f, sizeof(float) * B, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "checkpoint save");
  std::memcpy(host, &hd, sizeof(hd));
  return check_status_word(h);
}

mgfwa_status mgfwa_checkpoint_load(mgfwa_t* h, const void* host, int64_t bytes) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  const int64_t need = (int64_t)sizeof(CkptHeader) + ckpt_payload(h);
  if (!host || bytes != need) return fail(h, MGFWA_EINVAL, "checkpoint: buffer must hold %lld bytes", (long long)need);
  if (h->next_phase != MGFWA_PHASE_EXPLODE || h->grouped)
    return fail(h, MGFWA_EINVAL, "checkpoint: not between generations, or the handle is in a group");
  if (h->cfg.lagged_guiding) return fail(h, MGFWA_EINVAL, "checkpoint: not supported with lagged_guiding");
  CkptHeader hd;
  std::memcpy(&hd, host, sizeof(hd));
  if (hd.magic != kCkptMagic || hd.payload_bytes != ckpt_payload(h))
    return fail(h, MGFWA_EINVAL, "checkpoint: not a checkpoint of this layout");
  if (hd.fingerprint != h->fingerprint)
    return fail(h, MGFWA_EINVAL, "checkpoint: made for another configuration or objective");
  const char* in = static_cast<const char*>(host) + sizeof(CkptHeader);
  const int64_t F = (int64_t)h->p.B * h->p.mu, B = h->p.B;
  const size_t rb = sizeof(float) * h->p.D, pitch = sizeof(float) * h->p.Dp;
  // the staged host copy must outlive the asynchronous copies: synchronise below
  cudaError_t e = cudaMemcpyAsync(h->gens_done, &hd.gens_done, sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(h->fw_x, pitch, in, rb, rb, F, cudaMemcpyHostToDevice, h->stream);
  in += rb * F;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->fw_amp, in, sizeof(float) * F, cudaMemcpyHostToDevice, h->stream);
  in += sizeof(float) * F;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->fw_f, in, sizeof(float) * F, cudaMemcpyHostToDevice, h->stream);
  in += sizeof(float) * F;
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(h->best_x, pitch, in, rb, rb, B, cudaMemcpyHostToDevice, h->stream);
  in += rb * B;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->best_f, in, sizeof(float) * B, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "checkpoint load");
  h->evals = hd.evals;
  h->gen = hd.gen;
  h->launches = hd.launches;
  return MGFWA_OK;
}

mgfwa_status mgfwa_get_info(const mgfwa_t* h, mgfwa_info* info) {
  if (!h || !info) return MGFWA_EINVAL;
  info->evals = h->evals;
  info->generations = h->gen;
  info->k = h->p.k;
  info->dim_padded = h->p.Dp;
  info->sparks_per_gen = h->PA;
  info->device_bytes = (int64_t)h->arena_bytes;
  info->kernel_launches = h->launches;
  info->n_runs = h->p.B;
  info->fp8_inv_scale_x = h->op_kind == kOpFp8 ? h->inv_x : 0.0f;
  info->fp8_inv_scale_w = h->op_kind == kOpFp8 ? h->inv_w : 0.0f;
  return MGFWA_OK;
}

void mgfwa_destroy(mgfwa_t* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  tc_release(h->tc);
  if (h->refine_exec) cudaGraphExecDestroy(h->refine_exec);
  if (h->gen_exec) cudaGraphExecDestroy(h->gen_exec);
  arena_free(h);
  if (h->stream) cudaStreamSynchronize(h->stream);  // the pool's free completes in stream order
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  cudaGetLastError();
  delete h;
}

const char* mgfwa_last_error(const mgfwa_t* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

// ---------------------------------------------------------------------------
// Groups: many handles (any shapes) stepped together, one CUDA graph per step.

}  // extern "C"

struct mgfwa_group {
  std::vector<mgfwa_t*> members;
  cudaStream_t stream = nullptr;          // where the graph runs
  std::vector<cudaStream_t> branch;       // capture branches, one per member
  std::vector<cudaEvent_t> join, mid_a, mid_b;  // per member: end, after its explosion, after its guide
  cudaEvent_t fork = nullptr, done = nullptr, fit_e = nullptr, fit_g = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> live;                  // members captured in exec
  std::vector<int64_t> kernels;           // kernels per generation of each member
  int64_t group_kernels = 0;              // grouped fitness launches per generation
  PairMember* table = nullptr;            // device: the grouped launches' members (explosion, then guiding)
  int32_t table_cap = 0;
  std::string err;
};

namespace {

void group_release(mgfwa_group* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  for (cudaStream_t b : g->branch) if (b) cudaStreamDestroy(b);
  for (auto* v : {&g->join, &g->mid_a, &g->mid_b})
    for (cudaEvent_t e : *v) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {g->fork, g->done, g->fit_e, g->fit_g}) if (e) cudaEventDestroy(e);
  if (g->table) cudaFree(g->table);
  g->table = nullptr;
  if (g->stream) cudaStreamDestroy(g->stream);
  cudaGetLastError();
}

mgfwa_status group_fail(mgfwa_group* g, mgfwa_status st, const char* what) {
  g->err = what;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) g->err += std::string(": ") + cudaGetErrorString(e);
  set_thread_error(g->err.c_str());
  return st;
}

// Members whose sparks one grouped launch of the CTA-pair fitness kernel
// can evaluate with the others': an MLP on the pair kernel, the same kernel
// instance as the first such member.  Members of the same network family
// and operand type whose tuned tile differs are first set to the tile most
// of them have (every tile gives bitwise the same fitness, and a generation
// graph a member captured before keeps the kernel and maps it was captured
// with), so that one launch serves them all.
std::vector<int> group_fusable(mgfwa_group* g, const std::vector<int>& live) {
  std::vector<int> cand;
  for (int i : live) {
    const mgfwa_t* h = g->members[(size_t)i];
    if (h->kind == MGFWA_OBJ_MLP_CE && use_tc(h, h->cfg.precision) && h->tc.pair) cand.push_back(i);
  }
  std::vector<int> out;
  if (cand.empty()) return out;
  // the family of the first candidate: the same network layers (h1, h2, logit rows) and operand type
  const mgfwa_t* h0 = g->members[(size_t)cand[0]];
  auto same_family = [&](const mgfwa_t* h) {
    TcPlan a = h0->tc, b = h->tc;
    b.sparks_per_tile = a.sparks_per_tile;
    return tc_pair_same_instance(a, h0->mlp, b, h->mlp);
  };
  std::vector<int> fam;
  for (int i : cand)
    if (same_family(g->members[(size_t)i])) fam.push_back(i);
  // the tile most of the family has (the first member's on a tie), and a member that has it
  int best_s = h0->tc.sparks_per_tile, best_n = 0;
  const mgfwa_t* lead = h0;
  for (int i : fam) {
    const mgfwa_t* h = g->members[(size_t)i];
    int n = 0;
    for (int k : fam) n += g->members[(size_t)k]->tc.sparks_per_tile == h->tc.sparks_per_tile ? 1 : 0;
    if (n > best_n) {
      best_n = n;
      best_s = h->tc.sparks_per_tile;
      lead = h;
    }
  }
  for (int i : fam) {
    mgfwa_t* h = g->members[(size_t)i];
    if (h->tc.sparks_per_tile != best_s) {
      if (tc_pair_configure(h->tc, h->mlp, best_s, lead->tc.stages) != MGFWA_OK) continue;  // keeps its own tile
      h->tc.tuned = 0;
    }
    if (tc_pair_same_instance(lead->tc, lead->mlp, h->tc, h->mlp)) out.push_back(i);
  }
  if (out.size() < 2) out.clear();  // a lone member gains nothing from a grouped launch
  return out;
}

// Capture one generation of every live member into one graph.  Each member's
// kernels run on a branch of their own (the member's stream swapped for the
// branch while capturing).  Members on the same CTA-pair kernel instance
// share two grouped fitness launches: every such member's explosion, then one
// launch for all their explosion sparks, then every member's rank and guide,
// then one launch for all their guiding sparks, then every member's re-score
// and selection.  A grouped launch gives each spark bitwise the fitness of
// the member's own launch (a tile owns whole sparks and writes the member's
// partial sums in its own layout).  Other members run their whole generation
// on their branch.
mgfwa_status group_capture(mgfwa_group* g, const std::vector<int>& live) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  g->live.clear();
  const std::vector<int> fused = group_fusable(g, live);
  std::vector<char> is_fused(g->members.size(), 0);
  for (int i : fused) is_fused[(size_t)i] = 1;
  // the grouped launches' member tables (fixed for the graph's life), written before the capture
  const int32_t nf = (int32_t)fused.size();
  int32_t tiles_e = 0, tiles_g = 0;
  if (nf > 0) {
    std::vector<PairMember> tab((size_t)(2 * nf));
    for (int32_t k = 0; k < nf; ++k) {
      mgfwa_t* h = g->members[(size_t)fused[(size_t)k]];
      const Problem& p = h->p;
      const int64_t n_e = (int64_t)p.B * p.mu * p.lam, n_g = (int64_t)p.B * p.mu * p.m;
      tc_pair_member(h->tc, h->mlp, 0, h->sparks, p.Dp, (int32_t)n_e, h->op_scale, h->partial, h->status,
                     &tab[(size_t)k]);
      tc_pair_member(h->tc, h->mlp, n_e, h->sparks + n_e * p.Dp, p.Dp, (int32_t)n_g, h->op_scale, h->partial,
                     h->status, &tab[(size_t)(nf + k)]);
      tab[(size_t)k].tile_start = tiles_e;
      tiles_e += tab[(size_t)k].tiles;
      tab[(size_t)(nf + k)].tile_start = tiles_g;
      tiles_g += tab[(size_t)(nf + k)].tiles;
    }
    if (g->table_cap < 2 * nf) {
      if (g->table) cudaFree(g->table);
      g->table = nullptr;
      g->table_cap = 0;
      if (cudaMalloc(&g->table, sizeof(PairMember) * (size_t)(2 * nf)) != cudaSuccess)
        return group_fail(g, MGFWA_ENOMEM, "group: grouped launch table");
      g->table_cap = 2 * nf;
    }
    if (cudaMemcpy(g->table, tab.data(), sizeof(PairMember) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return group_fail(g, MGFWA_ECUDA, "group: grouped launch table copy");
  }
  if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return group_fail(g, MGFWA_ECUDA, "group: begin capture");
  mgfwa_status st = MGFWA_OK;
  bool ok = cudaEventRecord(g->fork, g->stream) == cudaSuccess;
  // phases [p0, p1] of member i on its branch after event `wait`, skipping its own fitness launches when it is
  // fused; the branch then records `end`, which the group stream waits on
  auto member_phases = [&](int i, int32_t p0, int32_t p1, cudaEvent_t wait, cudaEvent_t end) -> bool {
    mgfwa_t* h = g->members[(size_t)i];
    cudaStream_t br = g->branch[(size_t)i];
    if (cudaStreamWaitEvent(br, wait, 0) != cudaSuccess) return false;
    cudaStream_t own = h->stream;
    h->stream = br;
    h->capturing = true;
    const int64_t before = h->launches;
    for (int32_t ph = p0; ph <= p1 && st == MGFWA_OK; ++ph) {
      if (is_fused[(size_t)i] && (ph == MGFWA_PHASE_EVAL_E || ph == MGFWA_PHASE_EVAL_G)) continue;
      st = run_phase(h, ph);
      if (st == MGFWA_OK && is_fused[(size_t)i] && ph == MGFWA_PHASE_RESCORE && !finish_in_pick(h)) {
        // the grouped guiding launch left the partial sums, and this member's pick does not finish them
        const Problem& p = h->p;
        const int64_t n_e = (int64_t)p.B * p.mu * p.lam;
        if (launch_fitness_finish(h->partial, h->mtiles, p.B * p.mu * p.m, h->mlp.N, h->fit + n_e, br) < 0)
          st = cuda_fail(h, "group: guiding fitness means");
        else
          h->launches += 1;
      }
    }
    g->kernels[(size_t)i] += h->launches - before;
    h->launches = before;
    h->capturing = false;
    h->stream = own;
    if (st != MGFWA_OK) return false;
    return cudaEventRecord(end, br) == cudaSuccess && cudaStreamWaitEvent(g->stream, end, 0) == cudaSuccess;
  };
  for (int i : live) g->kernels[(size_t)i] = 0;
  g->group_kernels = 0;
  // stage 1: every member's explosion (and the whole generation of a member that is not fused)
  for (int i : live) {
    if (!ok) break;
    ok = is_fused[(size_t)i] ? member_phases(i, MGFWA_PHASE_EXPLODE, MGFWA_PHASE_EXPLODE, g->fork, g->mid_a[(size_t)i])
                             : member_phases(i, MGFWA_PHASE_EXPLODE, MGFWA_PHASE_SELECT, g->fork, g->join[(size_t)i]);
  }
  if (ok && nf > 0) {
    const mgfwa_t* h0 = g->members[(size_t)fused[0]];
    // stage 2: one launch for all fused members' explosion sparks, then each member's rank and guide
    ok = launch_fitness_pair_group(h0->tc, h0->mlp, g->table, nf, h0->status, g->stream, tiles_e) == 1 &&
         cudaEventRecord(g->fit_e, g->stream) == cudaSuccess;
    g->group_kernels += 1;
    for (int i : fused) {
      if (!ok) break;
      ok = member_phases(i, MGFWA_PHASE_EVAL_E, MGFWA_PHASE_EVAL_G, g->fit_e, g->mid_b[(size_t)i]);
    }
    // stage 3: one launch for all fused members' guiding sparks, then each member's re-score and selection
    if (ok)
      ok = launch_fitness_pair_group(h0->tc, h0->mlp, g->table + nf, nf, h0->status, g->stream, tiles_g) == 1 &&
           cudaEventRecord(g->fit_g, g->stream) == cudaSuccess;
    g->group_kernels += 1;
    for (int i : fused) {
      if (!ok) break;
      ok = member_phases(i, MGFWA_PHASE_RESCORE, MGFWA_PHASE_SELECT, g->fit_g, g->join[(size_t)i]);
    }
  }
  cudaGraph_t graph = nullptr;
  const bool ended = cudaStreamEndCapture(g->stream, &graph) == cudaSuccess;
  if (!ok || !ended || !graph || cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    g->exec = nullptr;
    return st != MGFWA_OK ? st : group_fail(g, MGFWA_ECUDA, "group: capture of a generation");
  }
  cudaGraphDestroy(graph);
  g->live = live;
  return MGFWA_OK;
}

}  // namespace

extern "C" {

mgfwa_status mgfwa_group_create(mgfwa_t* const* handles, int32_t count, mgfwa_group_t** out) {
  if (!out || !handles || count < 1) {
    set_thread_error("group: need an output pointer and at least one handle");
    return MGFWA_EINVAL;
  }
  *out = nullptr;
  for (int32_t i = 0; i < count; ++i) {
    mgfwa_t* h = handles[i];
    if (!h || h->broken || h->grouped) {
      set_thread_error("group: a handle is null, unusable or already in a group");
      return MGFWA_EINVAL;
    }
    for (int32_t j = 0; j < i; ++j)
      if (handles[j] == h) {
        set_thread_error("group: a handle appears twice");
        return MGFWA_EINVAL;
      }
    if (h->refine || h->profiling || h->cfg.lagged_guiding || h->next_phase != MGFWA_PHASE_EXPLODE ||
        h->device != handles[0]->device) {
      set_thread_error("group: members must not refine, profile, guide lagged or be inside a debug generation, "
                       "one device");
      return MGFWA_EINVAL;
    }
  }
  mgfwa_group* g = new (std::nothrow) mgfwa_group();
  if (!g) return MGFWA_ENOMEM;
  g->members.assign(handles, handles + count);
  g->branch.assign((size_t)count, nullptr);
  g->join.assign((size_t)count, nullptr);
  g->mid_a.assign((size_t)count, nullptr);
  g->mid_b.assign((size_t)count, nullptr);
  g->kernels.assign((size_t)count, 0);
  bool ok = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fit_e, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fit_g, cudaEventDisableTiming) == cudaSuccess;
  for (int32_t i = 0; i < count && ok; ++i)
    ok = cudaStreamCreateWithFlags(&g->branch[(size_t)i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->join[(size_t)i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->mid_a[(size_t)i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->mid_b[(size_t)i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    group_fail(g, MGFWA_ECUDA, "group: streams and events");
    group_release(g);
    delete g;
    return MGFWA_ECUDA;
  }
  for (mgfwa_t* h : g->members) h->grouped = true;
  *out = g;
  return MGFWA_OK;
}

mgfwa_status mgfwa_group_step(mgfwa_group_t* g, int32_t n_generations) {
  if (!g || n_generations < 0) return MGFWA_EINVAL;
  const size_t M = g->members.size();
  for (mgfwa_t* h : g->members) {
    if (h->broken) return group_fail(g, MGFWA_ECUDA, "group: a member is unusable after a CUDA error");
    if (h->next_phase != MGFWA_PHASE_EXPLODE) return group_fail(g, MGFWA_EINVAL, "group: a member is mid-generation");
  }
  // the group stream starts after everything already enqueued on the members' streams
  for (mgfwa_t* h : g->members)
    if (cudaEventRecord(g->done, h->stream) != cudaSuccess || cudaStreamWaitEvent(g->stream, g->done, 0) != cudaSuccess)
      return group_fail(g, MGFWA_ECUDA, "group: order after the members' streams");
  int32_t ran = 0;
  std::vector<int> live;
  for (int32_t it = 0; it < n_generations; ++it) {
    live.clear();
    for (size_t i = 0; i < M; ++i)
      if (budget_allows(g->members[i])) live.push_back((int)i);
    if (live.empty()) break;
    if (!g->exec || live != g->live) {
      mgfwa_status st = group_capture(g, live);
      if (st != MGFWA_OK) return st;
    }
    if (cudaGraphLaunch(g->exec, g->stream) != cudaSuccess) return group_fail(g, MGFWA_ECUDA, "group: graph launch");
    for (int i : live) {
      mgfwa_t* h = g->members[(size_t)i];
      h->gen += 1;
      h->evals += h->P;
      h->launches += g->kernels[(size_t)i];
    }
    ++ran;
  }
  // later work on a member's own stream runs after the group's
  if (cudaEventRecord(g->done, g->stream) != cudaSuccess) return group_fail(g, MGFWA_ECUDA, "group: record");
  for (mgfwa_t* h : g->members)
    if (cudaStreamWaitEvent(h->stream, g->done, 0) != cudaSuccess)
      return group_fail(g, MGFWA_ECUDA, "group: order before the members' streams");
  if (n_generations > 0 && ran == 0) return group_fail(g, MGFWA_EBUDGET, "group: no member's budget allows a generation");
  return MGFWA_OK;
}

void mgfwa_group_destroy(mgfwa_group_t* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (mgfwa_t* h : g->members) h->grouped = false;
  group_release(g);
  delete g;
}

// ---------------------------------------------------------------------------
// mgfwa_debug.h

mgfwa_status mgfwa_debug_phase(mgfwa_t* h, int32_t phase) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  const bool skip_rescore = phase == MGFWA_PHASE_SELECT && h->next_phase == MGFWA_PHASE_RESCORE;
  if (phase != h->next_phase && !skip_rescore)
    return fail(h, MGFWA_EINVAL, "phase %d out of order (expected %d)", phase, h->next_phase);
  if (phase == MGFWA_PHASE_EXPLODE && !budget_allows(h)) return fail(h, MGFWA_EBUDGET, "budget spent");
  st = run_phase(h, phase);
  if (st != MGFWA_OK) return st;
  // after selection the generation is over unless a refinement is due
  if (phase == MGFWA_PHASE_SELECT)
    h->next_phase = refine_due(h, h->gen) ? MGFWA_PHASE_REFINE : MGFWA_PHASE_EXPLODE;
  else
    h->next_phase = phase == MGFWA_PHASE_REFINE ? MGFWA_PHASE_EXPLODE : phase + 1;
  return MGFWA_OK;
}

namespace {
struct BufView {
  void* dev;
  int64_t rows;      // 0 for flat buffers
  int64_t row_bytes; // packed host bytes per row
  int64_t pitch;     // device bytes per row
  int64_t flat_bytes;
};

bool buffer_view(mgfwa_t* h, int32_t buf, BufView* v) {
  const Problem& p = h->p;
  const int64_t F = (int64_t)p.B * p.mu;
  const int64_t n_e = F * p.lam;
  const int64_t rb = sizeof(float) * p.D, pitch = sizeof(float) * p.Dp;
  *v = BufView{nullptr, 0, 0, 0, 0};
  switch (buf) {
    case MGFWA_BUF_FW_X: *v = {h->fw_x, F, rb, pitch, 0}; return true;
    case MGFWA_BUF_FW_AMP: *v = {h->fw_amp, 0, 0, 0, (int64_t)sizeof(float) * F}; return true;
    case MGFWA_BUF_FW_F: *v = {h->fw_f, 0, 0, 0, (int64_t)sizeof(float) * F}; return true;
    case MGFWA_BUF_SPARKS: *v = {h->sparks, n_e, rb, pitch, 0}; return true;
    case MGFWA_BUF_GUIDES: *v = {h->sparks + n_e * p.Dp, F * p.m, rb, pitch, 0}; return true;
    case MGFWA_BUF_FIT_E: *v = {h->fit, 0, 0, 0, (int64_t)sizeof(float) * n_e}; return true;
    case MGFWA_BUF_FIT_G: *v = {h->fit + n_e, 0, 0, 0, (int64_t)sizeof(float) * F * p.m}; return true;
    case MGFWA_BUF_TOP: *v = {h->top, 0, 0, 0, (int64_t)sizeof(int32_t) * F * p.m * p.k}; return true;
    case MGFWA_BUF_BOTTOM: *v = {h->bottom, 0, 0, 0, (int64_t)sizeof(int32_t) * F * p.m * p.k}; return true;
    case MGFWA_BUF_WINNER: *v = {h->winner, 0, 0, 0, (int64_t)sizeof(int32_t) * F}; return true;
    case MGFWA_BUF_BEST_X: *v = {h->best_x, p.B, rb, pitch, 0}; return true;
    case MGFWA_BUF_BEST_F: *v = {h->best_f, 0, 0, 0, (int64_t)sizeof(float) * p.B}; return true;
    case MGFWA_BUF_REFINE_X:
      if (!h->refine) return false;
      *v = {h->rw, p.B, rb, pitch, 0};
      return true;
    case MGFWA_BUF_REFINE_F:
      if (!h->refine) return false;
      *v = {h->rf, 0, 0, 0, (int64_t)sizeof(float) * p.B};
      return true;
    case MGFWA_BUF_REFINE_ELITE:
      if (!h->refine) return false;
      *v = {h->relite, 0, 0, 0, (int64_t)sizeof(int32_t) * p.B};
      return true;
    case MGFWA_BUF_LOSER: *v = {h->loser, 0, 0, 0, (int64_t)sizeof(int32_t) * F}; return true;
    case MGFWA_BUF_GV:
      if (!h->gv) return false;
      *v = {h->gv, F * p.m, rb, pitch, 0};
      return true;
  }
  return false;
}
}  // namespace

mgfwa_status mgfwa_debug_read(mgfwa_t* h, int32_t buf, void* host, int64_t nbytes) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  BufView v;
  if (!host || !buffer_view(h, buf, &v)) return fail(h, MGFWA_EINVAL, "debug_read: unknown buffer %d", buf);
  const int64_t want = v.rows ? v.rows * v.row_bytes : v.flat_bytes;
  if (nbytes != want) return fail(h, MGFWA_EINVAL, "debug_read: buffer %d holds %lld bytes", buf, (long long)want);
  cudaError_t e = v.rows ? cudaMemcpy2DAsync(host, v.row_bytes, v.dev, v.pitch, v.row_bytes, v.rows,
                                             cudaMemcpyDeviceToHost, h->stream)
                         : cudaMemcpyAsync(host, v.dev, v.flat_bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "debug_read");
  return MGFWA_OK;
}

mgfwa_status mgfwa_debug_write(mgfwa_t* h, int32_t buf, const void* host, int64_t nbytes) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  BufView v;
  if (!host || !buffer_view(h, buf, &v)) return fail(h, MGFWA_EINVAL, "debug_write: unknown buffer %d", buf);
  const int64_t want = v.rows ? v.rows * v.row_bytes : v.flat_bytes;
  if (nbytes != want) return fail(h, MGFWA_EINVAL, "debug_write: buffer %d holds %lld bytes", buf, (long long)want);
  cudaError_t e = v.rows ? cudaMemcpy2DAsync(v.dev, v.pitch, host, v.row_bytes, v.row_bytes, v.rows,
                                             cudaMemcpyHostToDevice, h->stream)
                         : cudaMemcpyAsync(v.dev, host, v.flat_bytes, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "debug_write");
  return MGFWA_OK;
}

mgfwa_status mgfwa_debug_gradient(mgfwa_t* h, const float* xs, int32_t count, float* g_out, float* f_out) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  const Problem& p = h->p;
  if (!h->refine) return fail(h, MGFWA_EINVAL, "debug_gradient: handle made without refinement");
  if (!xs || !g_out || !f_out || count < 1 || count > p.B)
    return fail(h, MGFWA_EINVAL, "debug_gradient: bad arguments (1 <= count <= %d)", p.B);
  if (h->next_phase != MGFWA_PHASE_EXPLODE) return fail(h, MGFWA_EINVAL, "a debug generation is in progress");
  const size_t rb = sizeof(float) * p.D, pitch = sizeof(float) * p.Dp;
  if (cudaMemcpy2DAsync(h->rw, pitch, xs, rb, rb, count, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return cuda_fail(h, "debug_gradient: copy rows");
  MG_LAUNCH(h, launch_grad(h->gp, h->mlp, h->rw, p.Dp, h->gscratch, h->rg, h->rf, h->stream, nullptr,
                           &h->refine_l1, h->status),
            "debug gradient");
  if (cudaMemcpy2DAsync(g_out, rb, h->rg, pitch, rb, count, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(f_out, h->rf, sizeof(float) * count, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return cuda_fail(h, "debug_gradient: read");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "debug_gradient synchronise");
  return MGFWA_OK;
}

mgfwa_status mgfwa_debug_fp32_tc(const mgfwa_t* h, int32_t* rescore, int32_t* refine) {
  if (!h) return MGFWA_EINVAL;
  if (rescore) *rescore = h->rescore_scratch ? (l1_on_tensor_cores(h->rescore_plan, h->mlp, &h->rescore_l1) ? 1 : 0) : -1;
  if (refine) *refine = h->refine ? (l1_on_tensor_cores(h->gp, h->mlp, &h->refine_l1) ? 1 : 0) : -1;
  return MGFWA_OK;
}

mgfwa_status mgfwa_debug_wait_budget(mgfwa_t* h, uint64_t ticks) {
  if (!h) return MGFWA_EINVAL;
  h->tc.wait_budget = ticks;
  return MGFWA_OK;
}

mgfwa_status mgfwa_debug_pair_tile(const mgfwa_t* h, int32_t* sparks_per_tile, int32_t* stages, int32_t* tuned,
                                   int32_t* k_tail) {
  if (!h) return MGFWA_EINVAL;
  const bool on = h->tc.ready && h->tc.pair;
  if (sparks_per_tile) *sparks_per_tile = on ? h->tc.sparks_per_tile : -1;
  if (stages) *stages = on ? h->tc.stages : -1;
  if (tuned) *tuned = on ? h->tc.tuned : -1;
  if (k_tail) *k_tail = on ? h->tc.ktail : -1;
  return MGFWA_OK;
}

mgfwa_status mgfwa_debug_set_pair_tile(mgfwa_t* h, int32_t sparks_per_tile, int32_t stages, int32_t k_tail) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  if (!h->tc.ready || !h->tc.pair) return fail(h, MGFWA_EINVAL, "the handle is not on the CTA-pair fitness kernel");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "set pair tile synchronise");
  st = tc_pair_configure(h->tc, h->mlp, sparks_per_tile, stages, k_tail);
  if (st != MGFWA_OK) return fail(h, st, "%s", tc_last_error());
  h->tc.tuned = 0;
  // the next generation is captured again, with the new shape
  if (h->gen_exec) cudaGraphExecDestroy(h->gen_exec);
  h->gen_exec = nullptr;
  return MGFWA_OK;
}

mgfwa_status mgfwa_debug_profile(mgfwa_t* h, int32_t enable) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "profile synchronise");
  h->ev_marks.clear();
  h->ev_next = 0;
  h->profiling = enable != 0;
  if (h->profiling && h->ev_pool.empty()) {
    h->ev_pool.resize(1 << 14);
    for (auto& e : h->ev_pool)
      if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(h, "event pool");
  }
  return MGFWA_OK;
}

mgfwa_status mgfwa_debug_kernel_times(mgfwa_t* h, double* ms_out, int64_t* launches_out) {
  mgfwa_status st = check_usable(h);
  if (st != MGFWA_OK) return st;
  if (!ms_out || !launches_out) return fail(h, MGFWA_EINVAL, "kernel_times: null output");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "kernel_times synchronise");
  for (int g = 0; g < MGFWA_N_KERNEL_GROUPS; ++g) {
    ms_out[g] = 0.0;
    launches_out[g] = 0;
  }
  for (auto& m : h->ev_marks) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, m.second.first, m.second.second) != cudaSuccess) return cuda_fail(h, "elapsed");
    ms_out[m.first] += ms;
    launches_out[m.first] += 1;
  }
  return MGFWA_OK;
}

}  // extern "C"
