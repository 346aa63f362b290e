/*
 * mgfwa.h -- C ABI of a GB300 (sm_103a) library that runs the Multi-Guiding
 * Spark Fireworks Algorithm (GPU-MGFWA, arXiv 2501.03944) on one GPU.
 *
 * Problem statement (Algorithm 1, Sec. 3; Eq. 1, Sec. 4.1): given a black box
 * f over a D-dimensional box [lb, ub]^D, return the best position found and
 * its fitness.  One generation of Algorithm 1 is: explosion sparks around
 * each firework with random mapping of out-of-bound coordinates, multi-
 * guiding sparks built from the ranked explosion sparks, random mapping,
 * fitness of every spark, and selection of the best individual of each
 * firework's population with the dynamic amplitude update.
 *
 * The black box here is the mean cross-entropy of a small MLP whose
 * flattened parameters (torch nn.Linear order: W1[h1][d_in] row-major, b1,
 * W2[h2][h1], b2, ...) are the search vector, on a fixed labelled batch; a
 * sphere objective (sum of squares) is kept for convergence checks.
 *
 * Conventions for every call:
 *  - Pointers in this header are HOST pointers unless a name says _dev.
 *    The library copies what it needs at create time; the caller keeps
 *    ownership of its buffers.
 *  - The handle owns all device memory it uses (one allocation made at
 *    create time and freed by mgfwa_destroy) and one CUDA stream (the
 *    caller's, if given, else its own).
 *  - Every call returns a status.  After MGFWA_ECUDA the handle can only be
 *    destroyed.  mgfwa_last_error() gives a one-line reason.
 *  - One handle per host thread at a time; several handles may share a GPU.
 */
#ifndef MGFWA_H
#define MGFWA_H

#include <stdint.h>

#if defined(__GNUC__)
#define MGFWA_API __attribute__((visibility("default")))
#else
#define MGFWA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MGFWA_OK = 0,
  MGFWA_EINVAL = 1,   /* an argument or configuration is invalid */
  MGFWA_ENOMEM = 2,   /* device or host allocation failed */
  MGFWA_ECUDA = 3,    /* a CUDA call failed; the handle is unusable */
  MGFWA_ETIMEOUT = 4, /* a bounded device-side wait gave up */
  MGFWA_EBUDGET = 5   /* the evaluation budget does not allow another generation */
} mgfwa_status;

typedef enum {
  MGFWA_FP32 = 0, /* FP32 CUDA-core fitness */
  MGFWA_BF16 = 1, /* tensor cores (tcgen05): BF16 first layer, TF32 later layers, FP32 accumulate; MLPs with
                     d_in % 8 == 0 and two layers (h1 in {32, 64, 128}, <= 32 classes) or three ((h1, h2) in
                     {(128, 64), (64, 32)}, <= 16 classes) */
  MGFWA_FP8 = 2,  /* tensor cores: E4M3 first layer (X scaled by 448 / max|X|, weights by 448 / max(|lb|, |ub|),
                     the product rescaled before the bias), TF32 later layers, FP32 accumulate; the BF16 shapes
                     with d_in % 16 == 0 */
  MGFWA_FP32X3 = 3, /* the testbed network objective at FP32 accuracy on the tensor cores: every FP32 operand
                       split into three BF16 parts, six products per K step into three FP32 accumulators; the
                       layers with fan_in % 8 == 0 and an even fan_out >= 16 (the others, and the final
                       1-output layer, on the CUDA cores) */
} mgfwa_precision;

/* Objectives: the cross-entropy of an MLP whose flattened parameters are the
 * search vector; the sphere; and the paper's own testbed (Sec. 4.1, Eq. 1),
 * the scalar output of a fixed network whose input is the search vector. */
enum { MGFWA_OBJ_MLP_CE = 0, MGFWA_OBJ_SPHERE = 1, MGFWA_OBJ_NET_OUTPUT = 2 };
/* GELU(v) = v (1 + erf(v / sqrt 2)) / 2, the exact form (testbed networks only) */
enum { MGFWA_ACT_TANH = 0, MGFWA_ACT_RELU = 1, MGFWA_ACT_GELU = 2 };

typedef struct {
  int64_t dim;                  /* D; equals the MLP parameter count for MLP objectives */
  float lb, ub;                 /* scalar bounds, lb < ub */
  int32_t n_fireworks;          /* mu >= 1 */
  int32_t sparks_per_firework;  /* lambda, a multiple of m */
  int32_t guiding_per_firework; /* m >= 1; group size g = lambda / m <= 1024 */
  float sigma;                  /* top/bottom fraction: k = round-half-up(sigma g) clamped to [1, g/2] */
  float boost;                  /* beta: guiding spark = x + beta * GV (default 1) */
  float amp_init;               /* A0 (default ub - lb) */
  float c_amplify, c_reduce;    /* amplitude factors on improvement / no improvement (1.2, 0.9) */
  int64_t eval_budget;          /* total evaluations, including the mu initial ones */
  uint64_t seed;                /* Philox key */
  int32_t precision;            /* mgfwa_precision */
  int32_t elite_rescore;        /* E in [0, 8], <= lambda + m: with BF16, each firework's E best candidates (by
                                   BF16 fitness) are re-scored in FP32 before selection (default 2; 0 = off) */
  int32_t n_runs;               /* B >= 1 independent runs of the same problem, stepped together (the
                                   batch dimension of Table 1, Sec. 3); run b uses seed + b */
  /* Hybrid refinement (the gradient reading of the hybrid strategies of
   * Sec. 5; MLP objectives only).  After the selection of every
   * refine_every-th generation (0 = never), each run's elite firework (the
   * first minimum of its fireworks' fitness) takes refine_steps projected
   * gradient steps w <- min(max(fma(-refine_lr, grad f(w), w), lb), ub), FP32
   * backpropagation on the whole batch; the firework (and the run's best)
   * take the result only if its FP32 fitness is strictly lower.  Amplitudes
   * are unchanged.  Each refinement charges 3 * refine_steps + 1
   * evaluations to the budget (a forward and a backward pass cost about
   * three forward passes; one more for the result), and a generation runs
   * only if its sparks and its refinement fit. */
  int32_t refine_every;
  int32_t refine_steps;
  float refine_lr;
  /* Loser-out tournament (Algorithm 1, the step after the selection; 0 =
   * off, 1 = on).  After each selection and the runs' best-so-far update,
   * every firework except its run's best (the first minimum of the run's
   * fireworks' fitness) whose fitness before and after the selection are
   * both finite is projected forward at its last improvement I (fitness
   * before minus after) over the g_rem generations the budget still allows
   * at mu (lambda + m) evaluations each (refinement not counted):
   * fmaf(-I, g_rem, f) in FP32.  If that is above the run's best-so-far the
   * firework loses: it is re-drawn uniformly in [lb, ub]^D (Philox purpose
   * 4), its amplitude set back to A0 and its fitness to +infinity (unknown
   * until its next sparks are evaluated; the next selection takes its best
   * candidate).  Costs no evaluations. */
  int32_t loser_out;
  /* Lagged multi-guiding (a variant of the generation's order; 0 = off,
   * 1 = on).  Generation t >= 2 builds its guiding sparks from the guiding
   * vectors of generation t - 1 at the fireworks' current positions,
   * G = x + beta GV_{t-1} (then the mapping), so that the explosion and
   * guiding sparks are evaluated in one launch; generation 1 runs the method
   * as written.  Handles with it cannot be checkpointed or grouped. */
  int32_t lagged_guiding;
  /* Sharding one run's fireworks over several handles (for example one per
   * GPU): the mu fireworks are split into n_shards contiguous ranges, and
   * this handle holds range shard_id, fireworks [shard_id mu / n_shards,
   * (shard_id + 1) mu / n_shards) of the run (integer division).  Every
   * firework draws from the Philox units of its index in the whole run, so
   * each shard's fireworks evolve bit for bit as in the unsharded run: the
   * selection is per firework, and nothing else crosses fireworks once the
   * loser-out tournament and the refinement (which read the run's best) are
   * off, as they must be with n_shards > 1.  eval_budget stays the whole
   * run's budget: a shard runs a generation exactly when the whole run
   * would.  The run's best is the minimum over the shards' best keys
   * (mgfwa_shard_key, mgfwa_reduce_best_keys).  n_shards 0 or 1 = one
   * handle holds the run. */
  int32_t shard_id;
  int32_t n_shards;
} mgfwa_config;

typedef struct {
  int32_t kind;          /* MGFWA_OBJ_MLP_CE, MGFWA_OBJ_SPHERE or MGFWA_OBJ_NET_OUTPUT */
  int32_t n_layers;      /* linear layers: 2 or 3 (MLP); 1 to 16 (testbed network) */
  const int32_t* widths; /* n_layers + 1 widths.  MLP: d_in, h1, [h2,] C: d_in % 8 == 0, hidden widths
                            <= 192, C in [2, 32]; the tensor-core shapes are listed at mgfwa_precision.
                            Testbed network: d (= dim), hidden widths, 1; every width in [1, 4096] */
  const int32_t* acts;   /* n_layers - 1 hidden activations (MGFWA_ACT_*; GELU for testbed networks only) */
  int64_t n_samples;     /* 1 <= N <= 65535 * 128 (MLP) */
  const float* X;        /* [N][d_in] row-major FP32 (MLP) */
  const int32_t* y;      /* [N] labels in [0, C) (MLP) */
  /* testbed network: its fixed parameters in nn.Linear order (W_1[h][d]
   * row-major, b_1, W_2, b_2, ...), copied at create; the precision is
   * MGFWA_FP32 (CUDA-core products, FP32 accumulation in an order fixed by
   * the layer shape alone) or MGFWA_FP32X3 (tensor-core layers at FP32
   * accuracy, also in an order fixed by the shape) */
  const float* params;
} mgfwa_objective;

typedef struct mgfwa_handle mgfwa_t;

/* Fill *cfg with the defaults (beta 1, A0 = ub - lb once bounds are set,
 * C_a 1.2, C_r 0.9, sigma 0.2, FP32, two elite re-scores, one run).  Fields the caller must still set:
 * dim, lb, ub, n_fireworks, sparks_per_firework, guiding_per_firework,
 * eval_budget, seed.  amp_init <= 0 means ub - lb. */
MGFWA_API mgfwa_status mgfwa_config_init(mgfwa_config* cfg);

/* Validate, allocate device state, copy the objective's batch, initialise
 * the mu fireworks (Algorithm 1, init) and evaluate them.  `cuda_stream`
 * is a cudaStream_t or NULL (the handle then creates its own).  The device
 * state is one allocation from the library's stream-ordered pool (one per
 * device); memory freed by mgfwa_destroy stays in that pool for later
 * handles.  A BF16 or E4M3 handle on the CTA-pair fitness kernel times
 * that kernel's tile shapes and pipeline depths once per device and
 * problem shape in the process (a few launches on the handle's stream) and
 * keeps the fastest; every choice gives bitwise the same fitness, and the
 * environment variable MGFWA_TUNE=0 keeps the default tile instead.  On
 * success *out is a new handle; on failure *out is NULL and nothing is
 * leaked.  Errors: EINVAL (configuration), ENOMEM, ECUDA. */
MGFWA_API mgfwa_status mgfwa_create(const mgfwa_config* cfg, const mgfwa_objective* obj, void* cuda_stream,
                          mgfwa_t** out);

/* Bytes of device memory mgfwa_create would allocate for this problem (the
 * handle's one arena), without allocating.  Same validation as create. */
MGFWA_API mgfwa_status mgfwa_footprint(const mgfwa_config* cfg, const mgfwa_objective* obj, int64_t* bytes_out);

/* Enqueue up to n_generations generations on the handle's stream; stops
 * early (without error) when the budget allows no further generation.
 * Returns EBUDGET if not even one generation fits.  Asynchronous. */
MGFWA_API mgfwa_status mgfwa_step(mgfwa_t* h, int32_t n_generations);

/* Run generations until the budget is spent, then synchronise. */
MGFWA_API mgfwa_status mgfwa_run(mgfwa_t* h);

/* Synchronise; write the best position so far (x_out: D floats, may be
 * NULL), its fitness recomputed in FP64 on the GPU (f_out, may be NULL) and
 * the evaluations used per run (evals_out, may be NULL).  With several runs:
 * the best of the run whose FP32 best-so-far is lowest (the first on ties). */
MGFWA_API mgfwa_status mgfwa_best(mgfwa_t* h, float* x_out, double* f_out, int64_t* evals_out);

/* As mgfwa_best for run `run` in [0, n_runs); EINVAL otherwise. */
MGFWA_API mgfwa_status mgfwa_best_run(mgfwa_t* h, int32_t run, float* x_out, double* f_out, int64_t* evals_out);

/* Evaluate `count` host vectors (each D floats, row-major) with the
 * handle's objective in the given precision; f_out gets count FP32 values.
 * The precision selects the MLP objective's path (BF16 / FP8 need the
 * handle's own tensor-core precision) and the testbed network's (FP32 on
 * the CUDA cores, or FP32X3 on a handle created in FP32X3); the sphere is
 * always FP32.  Uses the handle's device workspace (count <= the sparks
 * of one generation of all runs) and synchronises.  Only between
 * generations. */
MGFWA_API mgfwa_status mgfwa_evaluate(mgfwa_t* h, const float* xs, int64_t count, int32_t precision,
                            float* f_out);

typedef struct {
  int64_t evals;           /* evaluations so far per run, including init */
  int32_t generations;     /* generations run */
  int32_t k;               /* the subset size in use */
  int64_t dim_padded;      /* row stride of sparks and fireworks on the device (floats) */
  int64_t sparks_per_gen;  /* n_runs mu (lambda + m): sparks evaluated per generation, all runs */
  int64_t device_bytes;    /* bytes of the handle's device allocation */
  int64_t kernel_launches; /* kernels enqueued so far by this handle */
  int32_t n_runs;          /* B */
  float fp8_inv_scale_x;   /* FP8: X is stored as E4M3(X * this); 0 otherwise */
  float fp8_inv_scale_w;   /* FP8: first-layer weights stored as E4M3(w * this); 0 otherwise */
} mgfwa_info;

MGFWA_API mgfwa_status mgfwa_get_info(const mgfwa_t* h, mgfwa_info* info);

/* Checkpoint / resume.  A checkpoint (host memory, mgfwa_checkpoint_size
 * bytes) holds what the rest of a run depends on: the fireworks, their
 * amplitudes and fitness, each run's best-so-far, the evaluation and
 * generation counts (the generation is a word of the Philox counter).  It
 * loads only into a handle created with the same configuration (the budget
 * may differ) and objective (a fingerprint of both is checked: EINVAL
 * otherwise), between
 * generations, and the run then continues exactly as the saved one would
 * have.  Both calls synchronise. */
MGFWA_API mgfwa_status mgfwa_checkpoint_size(const mgfwa_t* h, int64_t* bytes);
MGFWA_API mgfwa_status mgfwa_checkpoint_save(mgfwa_t* h, void* host, int64_t bytes);
MGFWA_API mgfwa_status mgfwa_checkpoint_load(mgfwa_t* h, const void* host, int64_t bytes);

/* Release the handle's device memory and stream.  NULL-safe. */
MGFWA_API void mgfwa_destroy(mgfwa_t* h);

/* A one-line description of the handle's last error ("" if none).  With a
 * NULL handle: the last error of a failed mgfwa_create or
 * mgfwa_evaluate_fp32_noalloc in this thread. */
MGFWA_API const char* mgfwa_last_error(const mgfwa_t* h);

/* FP32 fitness (mean MLP cross-entropy, the objective above) of `count`
 * caller-owned spark rows, with NO device allocation.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc -- a
 * process whose device memory is owned and budgeted by another framework's
 * allocator, or a latency-critical loop where cudaMalloc/cudaFree may
 * synchronise the whole device.
 *  - X_dev [n_samples][widths[0]] FP32, y_dev [n_samples] int32 labels in
 *    [0, C), rows_dev [count][ld] FP32 (ld >= D, ld % 4 == 0; X_dev and
 *    rows_dev 16-byte aligned) are DEVICE pointers the caller owns; widths
 *    and acts are host arrays as in mgfwa_objective (d_in % 8 == 0, hidden
 *    widths <= 192, C in [2, 32]).  Labels are not checked on the device.
 *  - fitness_dev [count] FP32 receives the results (device pointer).
 *  - The work is enqueued on cuda_stream (a cudaStream_t, NULL = legacy
 *    default stream); the call does not synchronise.
 *  - 1 <= n_samples <= 65535 * 128.
 *  - Scratch is a fixed array inside the library's device image (1 MiB,
 *    held by every GPU that has loaded the library's device code, until the
 *    process exits): ceil(n_samples / 128) * count must be <= 262,144, else
 *    MGFWA_EINVAL.  The first call on each device looks up that array's
 *    device address (cudaGetSymbolAddress).  Under CUDA's default lazy
 *    module loading that first call (or any earlier use of the library on
 *    that device) is also what loads the device code there, which takes
 *    device memory for the code and this array; make the first call during
 *    set-up, before any stream capture and before the caller's memory is
 *    budgeted.  The address is cached per device ordinal for the device's
 *    primary context (the CUDA runtime's default context).  Calls share the
 *    array: calls that overlap on the GPU (other streams, other threads)
 *    race and give wrong results; serialise them.
 *  - Returns EINVAL on bad arguments (reason in mgfwa_last_error(NULL)),
 *    ECUDA if a launch fails. */
MGFWA_API mgfwa_status mgfwa_evaluate_fp32_noalloc(int32_t n_layers, const int32_t* widths, const int32_t* acts,
                                                   int64_t n_samples, const float* X_dev, const int32_t* y_dev,
                                                   const float* rows_dev, int64_t ld, int32_t count,
                                                   float* fitness_dev, void* cuda_stream);

/* ------------------------------------------------------------------------
 * The run's best over shards (the sharding seam; see mgfwa_config).
 *
 * A shard's key is its run's best-so-far FP32 fitness and its shard index.
 * The run's best is the key with the smallest fitness (NaN ranks last), the
 * smallest shard on ties: the same first minimum the unsharded run takes
 * over its fireworks in index order.  Callers that combine keys across
 * processes (an all-gather, an all-reduce) register that step as a hook;
 * mgfwa_reduce_best_keys is the host reduction such a hook (or a caller
 * holding every shard's key) applies.  Algorithm 1's "find the best
 * individual" over the whole population.
 * ------------------------------------------------------------------------ */
typedef struct {
  float f;          /* best-so-far FP32 fitness of the shard's run (NaN ranks last) */
  int32_t shard;    /* the shard's shard_id */
  int32_t run;      /* run index within the handle (0 .. n_runs - 1) */
  int32_t pad;      /* zero */
} mgfwa_best_key;

/* This handle's key for run `run` (synchronises the handle's stream).
 * Errors: EINVAL (bad handle or run), ECUDA. */
MGFWA_API mgfwa_status mgfwa_shard_key(mgfwa_t* h, int32_t run, mgfwa_best_key* key_out);

/* The reduction of `n` >= 1 keys (host memory) into *out: smallest f (NaN
 * last), then smallest shard, then smallest run.  Pure host code. */
MGFWA_API mgfwa_status mgfwa_reduce_best_keys(const mgfwa_best_key* keys, int32_t n, mgfwa_best_key* out);

/* Hook that combines this shard's key with the other shards' keys in place
 * (on every shard the same result); returns 0 on success.  `ctx` is the
 * caller's. */
typedef int32_t (*mgfwa_reduce_best_fn)(void* ctx, mgfwa_best_key* key);

/* Register (or, with fn NULL, remove) the handle's hook. */
MGFWA_API mgfwa_status mgfwa_set_reduce_best(mgfwa_t* h, mgfwa_reduce_best_fn fn, void* ctx);

/* The run's best key over all shards: this shard's key passed through the
 * hook, or this shard's key when no hook is registered (a handle that holds
 * the whole run).  Errors: as mgfwa_shard_key, ECUDA if the hook fails. */
MGFWA_API mgfwa_status mgfwa_global_best_key(mgfwa_t* h, int32_t run, mgfwa_best_key* key_out);

/* ------------------------------------------------------------------------
 * Serving: many optimisation requests on one GPU with continuous batching.
 *
 * Requests (a configuration and an objective, copied at submit) wait in a
 * FIFO.  mgfwa_server_tick() first admits waiting requests in order while a
 * slot is free and the head's device footprint (mgfwa_footprint) fits in
 * the memory limit beside the live runs; each admitted request becomes a
 * handle with its own stream, and all its state (fireworks, sparks, Philox
 * counters) stays on the device until it finishes.  The tick then enqueues
 * up to `generations` generations of every live run, on their streams, so
 * the runs' kernels overlap on the GPU.  A run whose budget allows no more
 * generations is finished: its best position and FP64 fitness are read
 * back, its memory is freed and its slot is given to the next request.
 * A request's result equals that of the same configuration run alone.
 * Single-threaded: one host thread drives a server.
 * ------------------------------------------------------------------------ */
typedef struct mgfwa_server mgfwa_server_t;

enum { MGFWA_REQ_QUEUED = 0, MGFWA_REQ_RUNNING = 1, MGFWA_REQ_DONE = 2, MGFWA_REQ_FAILED = 3 };

typedef struct {
  int32_t state;           /* MGFWA_REQ_* */
  int32_t status;          /* mgfwa_status of a failed request */
  int64_t evals;           /* evaluations used per run so far */
  double best_f;           /* FP64 best fitness (DONE) */
  double t_submit, t_admit, t_done; /* seconds on the server's steady clock */
  int64_t footprint;       /* device bytes of the request's handle */
} mgfwa_request_info;

typedef struct {
  int64_t submitted, admitted, completed, failed;
  int32_t live, queued;
  int64_t device_bytes_in_use; /* footprints of the live runs */
  int64_t sparks_evaluated;    /* over all generations enqueued so far */
} mgfwa_server_stats;

/* max_live: slots for concurrent runs (>= 1); device_bytes_limit: memory the
 * live runs may hold (> 0). */
MGFWA_API mgfwa_status mgfwa_server_create(int32_t max_live, int64_t device_bytes_limit, mgfwa_server_t** out);
/* Queue a request; *request_id identifies it.  EINVAL if the configuration
 * is invalid or its footprint exceeds the server's whole limit. */
MGFWA_API mgfwa_status mgfwa_server_submit(mgfwa_server_t* s, const mgfwa_config* cfg, const mgfwa_objective* obj,
                                           int64_t* request_id);
/* Admit, step every live run by up to `generations`, retire finished runs. */
MGFWA_API mgfwa_status mgfwa_server_tick(mgfwa_server_t* s, int32_t generations);
/* State and timing of a request; x_out (D floats, may be NULL) gets the best
 * position once DONE. */
MGFWA_API mgfwa_status mgfwa_server_poll(mgfwa_server_t* s, int64_t request_id, mgfwa_request_info* info,
                                         float* x_out);
MGFWA_API mgfwa_status mgfwa_server_stats_get(const mgfwa_server_t* s, mgfwa_server_stats* stats);
/* Seconds on the server's steady clock (the clock of the request times). */
MGFWA_API double mgfwa_server_now(const mgfwa_server_t* s);
/* Finish nothing further: destroy live handles and free everything. NULL-safe. */
MGFWA_API void mgfwa_server_destroy(mgfwa_server_t* s);

/* ------------------------------------------------------------------------
 * Groups: many handles of any shapes (dimension, population, network,
 * batch, precision) stepped together.  mgfwa_group_step() captures one
 * generation of every member whose budget allows one as parallel branches
 * of a single CUDA graph, then launches that graph once per generation; it
 * is captured again only when a member's budget runs out.  Each member's
 * results equal those of the same handle stepped alone (the generation
 * number is read on the device).  Members must not refine (refine_every =
 * 0), profile, or be inside a debug generation, and stay owned by the
 * caller; a handle belongs to at most one group.  Work already enqueued on
 * a member's stream runs before the group's generations, and later work on
 * it after them.  Asynchronous.
 * ------------------------------------------------------------------------ */
typedef struct mgfwa_group mgfwa_group_t;

MGFWA_API mgfwa_status mgfwa_group_create(mgfwa_t* const* handles, int32_t count, mgfwa_group_t** out);
/* Up to n_generations generations of every member (each stops at its
 * budget); EBUDGET if none could run one. */
MGFWA_API mgfwa_status mgfwa_group_step(mgfwa_group_t* g, int32_t n_generations);
/* The members stay valid (and usable alone again). NULL-safe. */
MGFWA_API void mgfwa_group_destroy(mgfwa_group_t* g);

#ifdef __cplusplus
}
#endif
#endif
