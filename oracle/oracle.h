/*
 * MGFWA CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-purpose restatement of one generation of the
 * Multi-Guiding Spark Fireworks Algorithm (GPU-MGFWA, Algorithm 1) used to
 * check the CUDA library.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load it.  It shares no code with the CUDA
 * path: its own Philox4x32-10 (Salmon et al., SC'11), its own MLP forward in
 * FP64, its own ranking, guiding and selection loops.
 *
 * Precision contract:
 *  - fitness (MLP cross-entropy, sphere) is computed in FP64;
 *  - spark positions, amplitudes and guiding vectors use exact FP32
 *    arithmetic in a fixed order (every product-add is an explicit fmaf);
 *  - every decision (rank, argmin, strict improvement) is taken on FP32
 *    fitness, the precision the kernels decide in: callers round the FP64
 *    fitness to FP32 before ranking or selection.
 *
 * Readings of passages the paper leaves open are stated at each function.
 * The build must use -ffp-contract=off so that no a*b+c is fused behind the
 * code's back (gcc contracts by default on aarch64).
 */
#ifndef MGFWA_ORACLE_H
#define MGFWA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox stream purposes (the fourth counter word). */
enum { ORC_INIT = 0, ORC_EXPLODE = 1, ORC_MAP = 2, ORC_GMAP = 3, ORC_LOSER = 4 };

/* Objective kinds and hidden activations. */
enum { ORC_MLP_CE = 0, ORC_SPHERE = 1, ORC_NET_OUTPUT = 2 };
enum { ORC_TANH = 0, ORC_RELU = 1, ORC_GELU = 2 };

typedef struct {
  int64_t dim;      /* D */
  float lb, ub;     /* scalar box bounds */
  int32_t mu;       /* fireworks */
  int32_t lam;      /* explosion sparks per firework */
  int32_t m;        /* guiding sparks per firework; lam % m == 0 */
  int32_t k;        /* top/bottom subset size per guiding group */
  float beta;       /* guiding-vector boost */
  float amp0;       /* initial amplitude */
  float c_a, c_r;   /* amplitude amplification / reduction factors */
  /* hybrid refinement of each run's elite (0 = off); see orc_refine */
  int32_t refine_every;  /* T: after the selection of every T-th generation */
  int32_t refine_steps;  /* T_g projected gradient steps */
  float refine_lr;       /* eta */
  /* loser-out tournament after each selection (0 = off); see orc_loser_out */
  int32_t loser_out;
  /* lagged multi-guiding (0 = off); see orc_guiding_vectors */
  int32_t lagged_guiding;
} orc_params;

typedef struct {
  int32_t kind;            /* ORC_MLP_CE or ORC_SPHERE */
  int64_t dim;             /* D (the sphere's length; the MLP's parameter count) */
  int32_t n_layers;        /* linear layers (MLP) */
  const int32_t* widths;   /* n_layers + 1 widths: d_in, h1, ..., C */
  const int32_t* acts;     /* n_layers - 1 hidden activations */
  int64_t n_samples;       /* N */
  const float* X;          /* [N][d_in] row-major */
  const int32_t* y;        /* [N] labels in [0, C) */
  /* ORC_NET_OUTPUT (the paper's testbed, Sec. 4.1, Eq. 1): the output of a
   * fixed network at the search vector, its input; widths d, h.., 1 and
   * its parameters in nn.Linear order (W_1[h][d] row-major, b_1, ...). */
  const float* params;
} orc_objective;

/* Philox4x32 with 10 rounds: out = bijection(ctr) keyed by key. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Uniform in [0,1) on a 2^-24 grid for coordinate `coord` of unit `unit`. */
float orc_uniform(uint64_t seed, uint32_t purpose, uint32_t gen, uint32_t unit, int64_t coord);

/* Subset size k from sigma and the group size g. */
int32_t orc_subset_size(float sigma, int32_t g);

/* FP64 objective value of one FP32 search vector. */
double orc_fitness(const orc_objective* obj, const float* x);

/* FP64 objective of `count` vectors spaced `stride` floats apart. */
void orc_fitness_many(const orc_objective* obj, const float* xs, int64_t count, int64_t stride,
                      double* out, int32_t n_threads);

/* Gradient of the objective at x (grad[D], FP64) by backpropagation;
 * returns the FP64 objective value. */
double orc_gradient(const orc_objective* obj, const float* x, double* grad);

/* Hybrid refinement of one vector: `steps` projected gradient steps
 *   w <- min(max(fmaf(-lr, (float)grad f(w), w), lb), ub)
 * from x_in, result in x_out; returns the FP64 objective of the result. */
double orc_refine(const orc_objective* obj, int64_t dim, const float* x_in, int32_t steps, float lr, float lb,
                  float ub, float* x_out);

/* Evaluations charged for one refinement: 3 per gradient step (a forward
 * and a backward pass cost about three forward passes) plus 1 for the
 * objective of the result. */
int64_t orc_refine_cost(const orc_params* p);

void orc_init(const orc_params* p, uint64_t seed, float* fw_x, float* fw_amp);
void orc_explode(const orc_params* p, uint64_t seed, uint32_t gen, const float* fw_x,
                 const float* fw_amp, float* sparks);
void orc_rank(const orc_params* p, const float* fit_e, int32_t* top, int32_t* bottom);
void orc_guide(const orc_params* p, uint64_t seed, uint32_t gen, const float* fw_x,
               const float* fw_amp, const float* sparks, const int32_t* top,
               const int32_t* bottom, float* guides);
/*
 * Lagged multi-guiding (a variant of the generation's order, off by
 * default): generation t >= 2 builds its guiding sparks from the guiding
 * vectors of generation t - 1, applied at the fireworks' positions of
 * generation t,
 *   G_t = x_t + beta * GV_{t-1}   (then the random mapping, stream GMAP, generation t),
 * so that a generation's explosion and guiding sparks need no ranking in
 * between and can be evaluated together.  Generation 1 has no earlier ranks
 * and runs the method as written (and records its GV).
 *
 * orc_guiding_vectors: GV of group q of firework i (row i*m + q) from the
 * explosion sparks and the rank lists, (sum top - sum bottom) / k with each
 * sum in list order, as in orc_guide.
 * orc_guide_from: the guiding sparks G = x + beta * GV with the mapping,
 * from given vectors.
 */
void orc_guiding_vectors(const orc_params* p, const float* sparks, const int32_t* top, const int32_t* bottom,
                         float* gv);
void orc_guide_from(const orc_params* p, uint64_t seed, uint32_t gen, const float* fw_x, const float* fw_amp,
                    const float* gv, float* guides);

void orc_select(const orc_params* p, const float* fit_e, const float* fit_g, const float* sparks,
                const float* guides, float* fw_x, float* fw_amp, float* fw_f, int32_t* winner);

/*
 * Loser-out tournament (Algorithm 1, last step of the loop; reading C-R15):
 * after the selection of generation `gen` and the run's best-so-far update
 * (run_best), every firework i except the run's best one (the first
 * minimum of fw_f) whose fitness before the selection, f_old[i], and after
 * it, fw_f[i], are both finite is projected forward at its last
 * improvement I = f_old[i] - fw_f[i] over the g_rem generations the budget
 * still allows: proj = fmaf(-I, g_rem, fw_f[i]).  If proj > run_best it
 * cannot reach the run's best and loses: it is re-initialised uniformly in
 * [lb, ub]^D (purpose ORC_LOSER, generation gen, unit i), its amplitude
 * set back to A0 and its fitness to +infinity (unknown until its sparks
 * are evaluated: the next selection takes its best candidate).
 * loser[i] = 1 for a loser, else 0.
 */
void orc_loser_out(const orc_params* p, uint64_t seed, uint32_t gen, int32_t g_rem, float run_best,
                   const float* f_old, float* fw_x, float* fw_amp, float* fw_f, int32_t* loser);

/* A whole run: init, then generations while the budget allows (and at most
 * max_gens).  Writes the best vector, its FP64 fitness, the evaluations
 * used and the generations run; trace (optional, max_gens entries) gets the
 * run's FP32 best-so-far after each generation.  Returns 0 on success. */
int32_t orc_run(const orc_params* p, const orc_objective* obj, uint64_t seed, int64_t budget,
                int32_t max_gens, int32_t n_threads, float* best_x, double* best_f,
                int64_t* evals_out, int32_t* gens_out, float* trace);

#ifdef __cplusplus
}
#endif
#endif
