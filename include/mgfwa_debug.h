/*
 * mgfwa_debug.h -- step-by-step access to one MGFWA generation, for parity
 * tests and checkpointing.  Same conventions as mgfwa.h (host pointers,
 * status codes, the handle owns its device memory).
 *
 * A generation of Algorithm 1 (Sec. 3) split into the phases below runs
 * exactly what mgfwa_step() runs, one kernel group at a time, so that a
 * test can read every intermediate and inject the oracle's fitness before
 * ranking and selection.
 */
#ifndef MGFWA_DEBUG_H
#define MGFWA_DEBUG_H

#include "mgfwa.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MGFWA_PHASE_EXPLODE = 0, /* generation += 1; explosion sparks + random mapping (Alg. 1, explosion) */
  MGFWA_PHASE_EVAL_E = 1,  /* fitness of the mu*lambda explosion sparks */
  MGFWA_PHASE_RANK = 2,    /* per firework and guiding group: top-k / bottom-k indices */
  MGFWA_PHASE_GUIDE = 3,   /* mu*m guiding sparks + random mapping (Alg. 1, multi-guiding) */
  MGFWA_PHASE_EVAL_G = 4,  /* fitness of the guiding sparks */
  MGFWA_PHASE_RESCORE = 5, /* low precision only: FP32 re-score of each firework's elite candidates */
  MGFWA_PHASE_SELECT = 6,  /* per-firework selection, amplitude update, run best, counters */
  MGFWA_PHASE_REFINE = 7   /* hybrid refinement of each run's elite, in the generations it is due */
} mgfwa_phase;

/* Enqueue one phase.  Phases must come in the order above, starting with
 * EXPLODE; RESCORE may be skipped (selection then uses the fitness as
 * evaluated or injected), and REFINE may be skipped in generations where no
 * refinement is due (it is a no-op there).  EINVAL otherwise, and EBUDGET if EXPLODE would
 * exceed the budget.  Asynchronous. */
MGFWA_API mgfwa_status mgfwa_debug_phase(mgfwa_t* h, int32_t phase);

/* Buffers of all B runs, run-major (B = 1 for a single run): firework
 * z = b*mu + i, explosion row z*lambda + j, guiding row z*m + q. */
typedef enum {
  MGFWA_BUF_FW_X = 0,    /* [B*mu][D] FP32 fireworks */
  MGFWA_BUF_FW_AMP = 1,  /* [B*mu] FP32 amplitudes */
  MGFWA_BUF_FW_F = 2,    /* [B*mu] FP32 firework fitness */
  MGFWA_BUF_SPARKS = 3,  /* [B*mu*lambda][D] FP32 explosion sparks */
  MGFWA_BUF_GUIDES = 4,  /* [B*mu*m][D] FP32 guiding sparks */
  MGFWA_BUF_FIT_E = 5,   /* [B*mu*lambda] FP32 explosion fitness */
  MGFWA_BUF_FIT_G = 6,   /* [B*mu*m] FP32 guiding fitness */
  MGFWA_BUF_TOP = 7,     /* [B*mu][m][k] int32: index within the firework of rank r, best first */
  MGFWA_BUF_BOTTOM = 8,  /* [B*mu][m][k] int32: index of rank g-1-r, worst first */
  MGFWA_BUF_WINNER = 9,  /* [B*mu] int32: -1 kept, j explosion j, lambda+q guiding q */
  MGFWA_BUF_BEST_X = 10, /* [B][D] FP32 best-so-far position per run */
  MGFWA_BUF_BEST_F = 11, /* [B] FP32 best-so-far fitness per run (the precision decisions use) */
  MGFWA_BUF_REFINE_X = 12,     /* [B][D] FP32 each run's vector after its last refinement (refining handles) */
  MGFWA_BUF_REFINE_F = 13,     /* [B] FP32 fitness of that vector */
  MGFWA_BUF_REFINE_ELITE = 14, /* [B] int32 index within the run of the firework it refined */
  MGFWA_BUF_LOSER = 15,        /* [B*mu] int32: 1 where the last selection's loser-out tournament re-drew the firework */
  MGFWA_BUF_GV = 16            /* [B*mu*m][D] FP32 the last recorded guiding vectors (lagged_guiding handles) */
} mgfwa_buffer;

/* Copy a buffer to / from host memory (rows packed D floats apart);
 * nbytes must equal the buffer's size.  Synchronises. */
MGFWA_API mgfwa_status mgfwa_debug_read(mgfwa_t* h, int32_t buf, void* host, int64_t nbytes);
MGFWA_API mgfwa_status mgfwa_debug_write(mgfwa_t* h, int32_t buf, const void* host, int64_t nbytes);

/* Kernel timing on the handle's stream.  While enabled, every kernel group
 * the handle enqueues is bracketed by CUDA events (taken from a pool made
 * here); mgfwa_debug_kernel_times() synchronises and returns, per group, the
 * summed milliseconds and the number of launches since the last enable.
 * Groups: 0 explode, 1 explosion fitness (main kernel), 2 fitness finish,
 * 3 rank, 4 guide, 5 guiding fitness (main kernel), 6 select + run best,
 * 7 elite FP32 re-score (pick + fitness + finish), 8 hybrid refinement. */
#define MGFWA_N_KERNEL_GROUPS 9
/* FP32 objective and gradient (by the refinement's backpropagation
 * kernels) of `count` <= n_runs host vectors of D floats; g_out gets
 * count * D floats, f_out count floats.  Only for handles made with
 * refine_every > 0, between generations.  Synchronises. */
MGFWA_API mgfwa_status mgfwa_debug_gradient(mgfwa_t* h, const float* xs, int32_t count, float* g_out,
                                            float* f_out);
/* Which products serve the handle's FP32 first layer: *rescore (the elite
 * re-score of a BF16 or FP8 handle) and *refine (the hybrid refinement and
 * mgfwa_debug_gradient) are 1 where the FP32-accurate tensor-core layer runs
 * (split TF32 products on tcgen05; a Blackwell GPU, first-layer width 32,
 * 64 or 128, d_in a multiple of 4, and its (128-sample tile, vector)
 * pairs numbering at least half the SMs), 0 where the CUDA-core products
 * run, -1 where the handle has no such phase.  Either pointer may be NULL. */
MGFWA_API mgfwa_status mgfwa_debug_fp32_tc(const mgfwa_t* h, int32_t* rescore, int32_t* refine);
MGFWA_API mgfwa_status mgfwa_debug_profile(mgfwa_t* h, int32_t enable);
MGFWA_API mgfwa_status mgfwa_debug_kernel_times(mgfwa_t* h, double* ms_out, int64_t* launches_out);
/* Budget, in SM clock ticks (clock64), of every bounded mbarrier wait in the
 * handle's tensor-core fitness kernels, for launches made after the call
 * (0 restores the default of about 2 s; a generation graph captured earlier
 * keeps the budget it was captured with).  With a budget of a few ticks an
 * ordinary wait runs out: the kernel raises its abort flag, every role leaves
 * its loop, drains its own copies and MMAs (fixed budgets), frees TMEM and
 * returns, and the call that launched it reports MGFWA_ETIMEOUT.  Failure
 * detection tests use it; nothing faults and no arrival is withheld.
 * Errors: EINVAL (null handle). */
MGFWA_API mgfwa_status mgfwa_debug_wait_budget(mgfwa_t* h, uint64_t ticks);
/* The CTA-pair fitness kernel's tile of a BF16 or FP8 handle (Sec. 3.3's
 * fitness of many sparks at once as one contraction): *sparks_per_tile
 * sparks per 256-sample tile -- 256/h1 when each spark's logits go into its
 * own accumulator columns once its activations are packed, 256/(h1 + 16 or
 * 32 logit rows) when the logits have columns of their own -- *stages
 * shared-memory pipeline stages, and *k_tail the layer-1 MMAs of the
 * partial last K atom (d_in not a multiple of 64 BF16 or 128 E4M3 values)
 * that go through the two K-tail buffers instead of taking a pipeline stage
 * of their own (0: none, or the atom is a stage); *tuned is 1 where
 * mgfwa_create chose the three by timing every shape, depth and K-tail
 * choice that fits (once per device and problem shape in the process), 0
 * where they were set.  All four are -1 for a handle not on the pair
 * kernel.  Any pointer may be NULL.
 * Errors: EINVAL (null handle). */
MGFWA_API mgfwa_status mgfwa_debug_pair_tile(const mgfwa_t* h, int32_t* sparks_per_tile, int32_t* stages,
                                             int32_t* tuned, int32_t* k_tail);
/* Set the pair kernel's tile for the generations that follow (the
 * handle's generation graph is captured again).  k_tail: 1 = the partial
 * last K atom through the K-tail buffers, 0 = as a pipeline stage, -1 = the
 * buffers where the network has such an atom and they fit beside the
 * pipeline.  Every shape, depth and K-tail choice gives every spark bitwise
 * the same fitness.  Synchronises the handle's stream.  Errors: EINVAL
 * (null handle, not on the pair kernel, a tile the kernel has not got for
 * this network, a depth outside 2 .. the deepest that fits, k_tail = 1
 * without a partial atom or with buffers that do not fit beside the
 * pipeline, k_tail outside -1 .. 1), ECUDA. */
MGFWA_API mgfwa_status mgfwa_debug_set_pair_tile(mgfwa_t* h, int32_t sparks_per_tile, int32_t stages,
                                                 int32_t k_tail);

#ifdef __cplusplus
}
#endif
#endif
