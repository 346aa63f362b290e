/*
 * Oracle MGFWA generation, step by step -- TEST INFRASTRUCTURE ONLY (see
 * oracle.h).
 *
 * Follows the paper's Algorithm 1 (Sec. 3): initialise mu fireworks, then
 * repeat { explosion sparks, random mapping, multi-guiding sparks, random
 * mapping, evaluation, selection of the best of each firework's population }
 * until the budget is spent.  The paper names MGFWA's mechanisms (Sec. 2.1:
 * multi-guiding sparks, boosted guiding vector, population-based random
 * mapping, dynamic amplitude) without restating them; each function states
 * the reading it implements.  All fireworks of a generation read the same
 * pre-generation state (the parallel semantics of Sec. 3 and Fig. 1).
 * Explosion sparks are evaluated before the guiding sparks are built, since
 * building them needs the explosion sparks' fitness (Algorithm 1 lists the
 * guiding step before evaluation).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* Subset size: k = round-half-up(sigma * g), clamped to [1, g/2]. */
int32_t orc_subset_size(float sigma, int32_t g) {
  int32_t k = (int32_t)floor((double)sigma * (double)g + 0.5);
  if (k > g / 2) k = g / 2;
  if (k < 1) k = 1;
  return k;
}

/* NaN fitness ranks as +infinity (nothing in the paper ranks a NaN). */
static float key(float f) { return isnan(f) ? INFINITY : f; }

/* Strict "a before b" in the (fitness, index) order. */
static int before(float fa, int32_t ia, float fb, int32_t ib) {
  float ka = key(fa), kb = key(fb);
  return ka < kb || (ka == kb && ia < ib);
}

/*
 * Random mapping of one coordinate (reading of "population-based random
 * mapping"): a coordinate outside [lb, ub] is redrawn uniformly in the
 * firework's amplitude box clipped to the bounds,
 *   lo = max(lb, x - A), hi = min(ub, x + A), v = lo + u (hi - lo).
 */
static float map_coord(const orc_params* p, float v, float x, float amp, float u) {
  if (!(v < p->lb) && !(v > p->ub)) return v;
  float lo = x - amp;
  float hi = x + amp;
  if (lo < p->lb) lo = p->lb;
  if (hi > p->ub) hi = p->ub;
  return fmaf(u, hi - lo, lo);
}

/* Algorithm 1 init: mu fireworks uniform in [lb, ub]^D; amplitude A0. */
void orc_init(const orc_params* p, uint64_t seed, float* fw_x, float* fw_amp) {
  const float width = p->ub - p->lb;
  for (int32_t i = 0; i < p->mu; ++i) {
    for (int64_t d = 0; d < p->dim; ++d) {
      float u = orc_uniform(seed, ORC_INIT, 0, (uint32_t)i, d);
      fw_x[(int64_t)i * p->dim + d] = fmaf(u, width, p->lb);
    }
    fw_amp[i] = p->amp0;
  }
}

/*
 * Explosion (reading: lam sparks per firework, each coordinate uniform in
 * the hypercube x +- A):  s = x + A (2u - 1), then the random mapping.
 * Rows are ordered firework-major: row i*lam + j.
 */
void orc_explode(const orc_params* p, uint64_t seed, uint32_t gen, const float* fw_x,
                 const float* fw_amp, float* sparks) {
  for (int32_t i = 0; i < p->mu; ++i) {
    const float* x = fw_x + (int64_t)i * p->dim;
    const float amp = fw_amp[i];
    for (int32_t j = 0; j < p->lam; ++j) {
      const uint32_t unit = (uint32_t)(i * p->lam + j);
      float* s = sparks + (int64_t)unit * p->dim;
      for (int64_t d = 0; d < p->dim; ++d) {
        float u = orc_uniform(seed, ORC_EXPLODE, gen, unit, d);
        float t = 2.0f * u - 1.0f;
        float v = fmaf(amp, t, x[d]);
        if (v < p->lb || v > p->ub) v = map_coord(p, v, x[d], amp, orc_uniform(seed, ORC_MAP, gen, unit, d));
        s[d] = v;
      }
    }
  }
}

/*
 * Ranking for the multi-guiding sparks (reading): the lam explosion sparks of
 * firework i are split in index order into m groups of g = lam/m; in each
 * group the sparks are ordered by (fitness, index) ascending.
 *   top[(i*m+q)*k + r]    = index (within the firework) of rank r (best first)
 *   bottom[(i*m+q)*k + r] = index of rank g-1-r (worst first)
 * The order is found by counting, for each spark, how many sparks of its
 * group come strictly before it.
 */
void orc_rank(const orc_params* p, const float* fit_e, int32_t* top, int32_t* bottom) {
  const int32_t g = p->lam / p->m, k = p->k;
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)g);
  for (int32_t i = 0; i < p->mu; ++i) {
    for (int32_t q = 0; q < p->m; ++q) {
      const int32_t base = q * g;
      const float* f = fit_e + (int64_t)i * p->lam + base;
      for (int32_t a = 0; a < g; ++a) {
        int32_t r = 0;
        for (int32_t b = 0; b < g; ++b)
          if (before(f[b], b, f[a], a)) ++r;
        order[r] = base + a;
      }
      int32_t* t = top + ((int64_t)i * p->m + q) * k;
      int32_t* bt = bottom + ((int64_t)i * p->m + q) * k;
      for (int32_t r = 0; r < k; ++r) {
        t[r] = order[r];
        bt[r] = order[g - 1 - r];
      }
    }
  }
  free(order);
}

/*
 * Multi-guiding sparks (reading of the guiding vector and its boost): for
 * group q of firework i,
 *   GV = (sum of the k best sparks - sum of the k worst sparks) / k,
 *   G  = x + beta * GV,
 * each sum taken in the order of the index lists (best first, worst first),
 * then the random mapping with its own stream.  Row i*m + q.
 */
void orc_guide(const orc_params* p, uint64_t seed, uint32_t gen, const float* fw_x,
               const float* fw_amp, const float* sparks, const int32_t* top,
               const int32_t* bottom, float* guides) {
  const int32_t k = p->k;
  const float fk = (float)k;
  for (int32_t i = 0; i < p->mu; ++i) {
    const float* x = fw_x + (int64_t)i * p->dim;
    const float amp = fw_amp[i];
    const float* fs = sparks + (int64_t)i * p->lam * p->dim;
    for (int32_t q = 0; q < p->m; ++q) {
      const int32_t* t = top + ((int64_t)i * p->m + q) * k;
      const int32_t* bt = bottom + ((int64_t)i * p->m + q) * k;
      const uint32_t unit = (uint32_t)(i * p->m + q);
      float* G = guides + (int64_t)unit * p->dim;
      for (int64_t d = 0; d < p->dim; ++d) {
        float sum_top = fs[(int64_t)t[0] * p->dim + d];
        float sum_bot = fs[(int64_t)bt[0] * p->dim + d];
        for (int32_t r = 1; r < k; ++r) {
          sum_top = sum_top + fs[(int64_t)t[r] * p->dim + d];
          sum_bot = sum_bot + fs[(int64_t)bt[r] * p->dim + d];
        }
        float gv = (sum_top - sum_bot) / fk;
        float v = fmaf(p->beta, gv, x[d]);
        if (v < p->lb || v > p->ub) v = map_coord(p, v, x[d], amp, orc_uniform(seed, ORC_GMAP, gen, unit, d));
        G[d] = v;
      }
    }
  }
}

/* Lagged multi-guiding: the guiding vectors alone (Sec. 2.1's GV, sums in
 * list order as in orc_guide), and the guiding sparks from given vectors. */
void orc_guiding_vectors(const orc_params* p, const float* sparks, const int32_t* top, const int32_t* bottom,
                         float* gv) {
  const int32_t k = p->k;
  const float fk = (float)k;
  for (int32_t i = 0; i < p->mu; ++i) {
    const float* fs = sparks + (int64_t)i * p->lam * p->dim;
    for (int32_t q = 0; q < p->m; ++q) {
      const int32_t* t = top + ((int64_t)i * p->m + q) * k;
      const int32_t* bt = bottom + ((int64_t)i * p->m + q) * k;
      float* out = gv + ((int64_t)i * p->m + q) * p->dim;
      for (int64_t d = 0; d < p->dim; ++d) {
        float sum_top = fs[(int64_t)t[0] * p->dim + d];
        float sum_bot = fs[(int64_t)bt[0] * p->dim + d];
        for (int32_t r = 1; r < k; ++r) {
          sum_top = sum_top + fs[(int64_t)t[r] * p->dim + d];
          sum_bot = sum_bot + fs[(int64_t)bt[r] * p->dim + d];
        }
        out[d] = (sum_top - sum_bot) / fk;
      }
    }
  }
}

void orc_guide_from(const orc_params* p, uint64_t seed, uint32_t gen, const float* fw_x, const float* fw_amp,
                    const float* gv, float* guides) {
  for (int32_t i = 0; i < p->mu; ++i) {
    const float* x = fw_x + (int64_t)i * p->dim;
    const float amp = fw_amp[i];
    for (int32_t q = 0; q < p->m; ++q) {
      const uint32_t unit = (uint32_t)(i * p->m + q);
      const float* g = gv + (int64_t)unit * p->dim;
      float* G = guides + (int64_t)unit * p->dim;
      for (int64_t d = 0; d < p->dim; ++d) {
        float v = fmaf(p->beta, g[d], x[d]);
        if (v < p->lb || v > p->ub) v = map_coord(p, v, x[d], amp, orc_uniform(seed, ORC_GMAP, gen, unit, d));
        G[d] = v;
      }
    }
  }
}

/*
 * Selection of the best individual of each firework's population with the
 * dynamic amplitude (reading): candidates in the order explosion 0..lam-1,
 * guiding 0..m-1; the first minimum wins ties.  If it is strictly better than
 * the firework, the firework moves there and A <- C_a A; otherwise the
 * firework stays and A <- C_r A.  winner[i] = -1 (kept), j (explosion j) or
 * lam + q (guiding q).
 */
void orc_select(const orc_params* p, const float* fit_e, const float* fit_g, const float* sparks,
                const float* guides, float* fw_x, float* fw_amp, float* fw_f, int32_t* winner) {
  const int32_t n_cand = p->lam + p->m;
  for (int32_t i = 0; i < p->mu; ++i) {
    int32_t best = 0;
    float best_f = fit_e[(int64_t)i * p->lam];
    for (int32_t c = 1; c < n_cand; ++c) {
      float f = c < p->lam ? fit_e[(int64_t)i * p->lam + c] : fit_g[(int64_t)i * p->m + (c - p->lam)];
      if (before(f, c, best_f, best)) {
        best = c;
        best_f = f;
      }
    }
    if (key(best_f) < key(fw_f[i])) {
      const float* src = best < p->lam ? sparks + ((int64_t)i * p->lam + best) * p->dim
                                       : guides + ((int64_t)i * p->m + (best - p->lam)) * p->dim;
      memcpy(fw_x + (int64_t)i * p->dim, src, sizeof(float) * (size_t)p->dim);
      fw_f[i] = best_f;
      fw_amp[i] = fw_amp[i] * p->c_a;
      winner[i] = best;
    } else {
      fw_amp[i] = fw_amp[i] * p->c_r;
      winner[i] = -1;
    }
  }
}

void orc_loser_out(const orc_params* p, uint64_t seed, uint32_t gen, int32_t g_rem, float run_best,
                   const float* f_old, float* fw_x, float* fw_amp, float* fw_f, int32_t* loser) {
  int32_t e = 0;
  for (int32_t i = 1; i < p->mu; ++i)
    if (key(fw_f[i]) < key(fw_f[e])) e = i;
  const float width = p->ub - p->lb;
  for (int32_t i = 0; i < p->mu; ++i) {
    loser[i] = 0;
    if (i == e || !isfinite(f_old[i]) || !isfinite(fw_f[i])) continue;
    const float improvement = f_old[i] - fw_f[i];
    const float proj = fmaf(-improvement, (float)g_rem, fw_f[i]);
    if (!(proj > run_best)) continue;
    loser[i] = 1;
    for (int64_t d = 0; d < p->dim; ++d) {
      const float u = orc_uniform(seed, ORC_LOSER, gen, (uint32_t)i, d);
      fw_x[(int64_t)i * p->dim + d] = fmaf(u, width, p->lb);
    }
    fw_amp[i] = p->amp0;
    fw_f[i] = INFINITY;
  }
}

static void eval_f32(const orc_objective* obj, const float* xs, int64_t count, int64_t stride,
                     float* out, int32_t n_threads) {
  double* tmp = (double*)malloc(sizeof(double) * (size_t)count);
  orc_fitness_many(obj, xs, count, stride, tmp, n_threads);
  for (int64_t i = 0; i < count; ++i) out[i] = (float)tmp[i];
  free(tmp);
}

/*
 * Hybrid refinement (the paper's outlook, Sec. 5, proposes combining MGFWA
 * with other optimisers; this is the gradient reading of it): projected
 * gradient descent on the objective from x_in.  Each step takes the FP64
 * gradient, rounds it to FP32 and moves every coordinate by one fused
 * multiply-add, then clips it to the box.
 */
double orc_refine(const orc_objective* obj, int64_t dim, const float* x_in, int32_t steps, float lr, float lb,
                  float ub, float* x_out) {
  double* g = (double*)malloc(sizeof(double) * (size_t)dim);
  memcpy(x_out, x_in, sizeof(float) * (size_t)dim);
  for (int32_t s = 0; s < steps; ++s) {
    orc_gradient(obj, x_out, g);
    for (int64_t k = 0; k < dim; ++k) x_out[k] = fminf(fmaxf(fmaf(-lr, (float)g[k], x_out[k]), lb), ub);
  }
  free(g);
  return orc_fitness(obj, x_out);
}

int64_t orc_refine_cost(const orc_params* p) { return 3 * (int64_t)p->refine_steps + 1; }

/* Generation `gen` (1-based) ends with a refinement. */
static int refine_due(const orc_params* p, int32_t gen) {
  return p->refine_every > 0 && p->refine_steps > 0 && gen % p->refine_every == 0;
}

int32_t orc_run(const orc_params* p, const orc_objective* obj, uint64_t seed, int64_t budget,
                int32_t max_gens, int32_t n_threads, float* best_x, double* best_f,
                int64_t* evals_out, int32_t* gens_out, float* trace) {
  const int64_t D = p->dim;
  const int32_t g = p->lam / p->m;
  if (p->m <= 0 || p->lam % p->m != 0 || p->k < 1 || p->k > g / 2 || budget < p->mu) return 1;
  float* fw_x = (float*)malloc(sizeof(float) * (size_t)(p->mu * D));
  float* fw_amp = (float*)malloc(sizeof(float) * (size_t)p->mu);
  float* fw_f = (float*)malloc(sizeof(float) * (size_t)p->mu);
  float* sparks = (float*)malloc(sizeof(float) * (size_t)((int64_t)p->mu * p->lam * D));
  float* guides = (float*)malloc(sizeof(float) * (size_t)((int64_t)p->mu * p->m * D));
  float* fit_e = (float*)malloc(sizeof(float) * (size_t)(p->mu * p->lam));
  float* fit_g = (float*)malloc(sizeof(float) * (size_t)(p->mu * p->m));
  int32_t* top = (int32_t*)malloc(sizeof(int32_t) * (size_t)(p->mu * p->m * p->k));
  int32_t* bottom = (int32_t*)malloc(sizeof(int32_t) * (size_t)(p->mu * p->m * p->k));
  int32_t* winner = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->mu);
  float* f_old = (float*)malloc(sizeof(float) * (size_t)p->mu);
  int32_t* loser = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->mu);
  float* gv = p->lagged_guiding ? (float*)malloc(sizeof(float) * (size_t)((int64_t)p->mu * p->m * D)) : NULL;

  orc_init(p, seed, fw_x, fw_amp);
  eval_f32(obj, fw_x, p->mu, D, fw_f, n_threads);
  int64_t evals = p->mu;
  int32_t best_i = 0;
  for (int32_t i = 1; i < p->mu; ++i)
    if (key(fw_f[i]) < key(fw_f[best_i])) best_i = i;
  float run_best = fw_f[best_i];
  memcpy(best_x, fw_x + (int64_t)best_i * D, sizeof(float) * (size_t)D);

  const int64_t per_gen = (int64_t)p->mu * (p->lam + p->m);
  /* the generations the budget allows at per_gen evaluations each (refinement not counted) */
  const int64_t g_max = (budget - p->mu) / per_gen;
  int32_t gen = 0;
  float* refined = (float*)malloc(sizeof(float) * (size_t)D);
  while (gen < max_gens && evals + per_gen + (refine_due(p, gen + 1) ? orc_refine_cost(p) : 0) <= budget) {
    ++gen;
    orc_explode(p, seed, (uint32_t)gen, fw_x, fw_amp, sparks);
    if (p->lagged_guiding && gen > 1) {
      /* lagged: the guiding sparks from generation gen - 1's vectors, then
       * this generation's ranks give the vectors for the next one */
      orc_guide_from(p, seed, (uint32_t)gen, fw_x, fw_amp, gv, guides);
      eval_f32(obj, sparks, (int64_t)p->mu * p->lam, D, fit_e, n_threads);
      eval_f32(obj, guides, (int64_t)p->mu * p->m, D, fit_g, n_threads);
      orc_rank(p, fit_e, top, bottom);
      orc_guiding_vectors(p, sparks, top, bottom, gv);
    } else {
      eval_f32(obj, sparks, (int64_t)p->mu * p->lam, D, fit_e, n_threads);
      orc_rank(p, fit_e, top, bottom);
      orc_guide(p, seed, (uint32_t)gen, fw_x, fw_amp, sparks, top, bottom, guides);
      eval_f32(obj, guides, (int64_t)p->mu * p->m, D, fit_g, n_threads);
      if (p->lagged_guiding) orc_guiding_vectors(p, sparks, top, bottom, gv);
    }
    memcpy(f_old, fw_f, sizeof(float) * (size_t)p->mu);
    orc_select(p, fit_e, fit_g, sparks, guides, fw_x, fw_amp, fw_f, winner);
    evals += per_gen;
    for (int32_t i = 0; i < p->mu; ++i) {
      if (key(fw_f[i]) < key(run_best)) {
        run_best = fw_f[i];
        memcpy(best_x, fw_x + (int64_t)i * D, sizeof(float) * (size_t)D);
      }
    }
    if (p->loser_out) {
      const int64_t g_rem = g_max - gen > 0 ? g_max - gen : 0;
      orc_loser_out(p, seed, (uint32_t)gen, (int32_t)g_rem, run_best, f_old, fw_x, fw_amp, fw_f, loser);
    }
    if (refine_due(p, gen)) {
      /* refine the run's elite firework (first minimum); keep the result
       * only on strict improvement; the amplitude is left as selected */
      int32_t e = 0;
      for (int32_t i = 1; i < p->mu; ++i)
        if (key(fw_f[i]) < key(fw_f[e])) e = i;
      const float fr = (float)orc_refine(obj, D, fw_x + (int64_t)e * D, p->refine_steps, p->refine_lr, p->lb,
                                         p->ub, refined);
      if (key(fr) < key(fw_f[e])) {
        memcpy(fw_x + (int64_t)e * D, refined, sizeof(float) * (size_t)D);
        fw_f[e] = fr;
        if (key(fr) < key(run_best)) {
          run_best = fr;
          memcpy(best_x, refined, sizeof(float) * (size_t)D);
        }
      }
      evals += orc_refine_cost(p);
    }
    if (trace) trace[gen - 1] = run_best;
  }
  *best_f = orc_fitness(obj, best_x);
  *evals_out = evals;
  *gens_out = gen;

  free(fw_x); free(fw_amp); free(fw_f); free(sparks); free(guides);
  free(fit_e); free(fit_g); free(top); free(bottom); free(winner); free(refined); free(f_old); free(loser);
  free(gv);
  return 0;
}
