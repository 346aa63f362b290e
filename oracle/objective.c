/*
 * Oracle objectives in FP64 -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The black box f of Algorithm 1 (the paper's Sec. 4.1, Eq. 1 minimises the
 * output of a fixed network; here the search vector is the network's own
 * flattened parameters and f is its mean cross-entropy on a fixed batch):
 *
 *   a_0 = x_n;  a_l = act(W_l a_{l-1} + b_l) for hidden layers;
 *   z = W_L a_{L-1} + b_L;
 *   f = (1/N) sum_n [ log sum_c exp(z_c) - z_{y_n} ],
 *
 * with parameters laid out in torch nn.Linear order (W_1[h1][d_in]
 * row-major, b_1, W_2[h2][h1], b_2, ...).  log-sum-exp subtracts max_c z_c
 * first.  Every multiply and add is plain double arithmetic in index order.
 *
 * The sphere objective f(x) = sum_k x_k^2 is kept for convergence checks.
 *
 * The paper's own testbed (Sec. 4.1, Eq. 1): the search vector x is the
 * input of a fixed network and f(x) its scalar output,
 *   a_0 = x;  a_l = act(W_l a_{l-1} + b_l) for hidden layers;  f = W_L a_{L-1} + b_L,
 * activations ReLU, tanh or GELU(v) = v (1 + erf(v / sqrt 2)) / 2, the
 * network's parameters in the same nn.Linear order.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static double act(int32_t kind, double v) {
  if (kind == ORC_TANH) return tanh(v);
  if (kind == ORC_GELU) return 0.5 * v * (1.0 + erf(v / sqrt(2.0)));
  return v > 0.0 ? v : 0.0;
}

static double net_output(const orc_objective* obj, const float* x) {
  const int32_t L = obj->n_layers;
  int32_t wmax = 0;
  for (int32_t l = 0; l <= L; ++l)
    if (obj->widths[l] > wmax) wmax = obj->widths[l];
  double* a = (double*)malloc(sizeof(double) * (size_t)wmax);
  double* b = (double*)malloc(sizeof(double) * (size_t)wmax);
  for (int32_t i = 0; i < obj->widths[0]; ++i) a[i] = (double)x[i];
  const float* p = obj->params;
  for (int32_t l = 0; l < L; ++l) {
    const int32_t fan_in = obj->widths[l], fan_out = obj->widths[l + 1];
    const float* W = p;
    const float* bias = p + (int64_t)fan_in * fan_out;
    for (int32_t j = 0; j < fan_out; ++j) {
      double s = (double)bias[j];
      for (int32_t i = 0; i < fan_in; ++i) s += (double)W[(int64_t)j * fan_in + i] * a[i];
      b[j] = (l + 1 < L) ? act(obj->acts[l], s) : s;
    }
    p = bias + fan_out;
    double* t = a; a = b; b = t;
  }
  const double f = a[0];
  free(a);
  free(b);
  return f;
}

static double mlp_ce(const orc_objective* obj, const float* x) {
  const int32_t L = obj->n_layers;
  int32_t wmax = 0;
  for (int32_t l = 0; l <= L; ++l)
    if (obj->widths[l] > wmax) wmax = obj->widths[l];
  double* a = (double*)malloc(sizeof(double) * (size_t)wmax);
  double* b = (double*)malloc(sizeof(double) * (size_t)wmax);
  double total = 0.0;
  for (int64_t n = 0; n < obj->n_samples; ++n) {
    const int32_t d0 = obj->widths[0];
    for (int32_t i = 0; i < d0; ++i) a[i] = (double)obj->X[n * d0 + i];
    const float* p = x;
    for (int32_t l = 0; l < L; ++l) {
      const int32_t fan_in = obj->widths[l], fan_out = obj->widths[l + 1];
      const float* W = p;
      const float* bias = p + (int64_t)fan_in * fan_out;
      for (int32_t j = 0; j < fan_out; ++j) {
        double s = (double)bias[j];
        for (int32_t i = 0; i < fan_in; ++i) s += (double)W[(int64_t)j * fan_in + i] * a[i];
        b[j] = (l + 1 < L) ? act(obj->acts[l], s) : s;
      }
      p = bias + fan_out;
      double* t = a; a = b; b = t;
    }
    const int32_t C = obj->widths[L];
    double zmax = a[0];
    for (int32_t c = 1; c < C; ++c)
      if (a[c] > zmax) zmax = a[c];
    double se = 0.0;
    for (int32_t c = 0; c < C; ++c) se += exp(a[c] - zmax);
    total += (zmax + log(se)) - a[obj->y[n]];
  }
  free(a);
  free(b);
  return total / (double)obj->n_samples;
}

double orc_fitness(const orc_objective* obj, const float* x) {
  if (obj->kind == ORC_SPHERE) {
    double s = 0.0;
    for (int64_t k = 0; k < obj->dim; ++k) s += (double)x[k] * (double)x[k];
    return s;
  }
  if (obj->kind == ORC_NET_OUTPUT) return net_output(obj, x);
  return mlp_ce(obj, x);
}

typedef struct {
  const orc_objective* obj;
  const float* xs;
  int64_t begin, end, stride;
  double* out;
} fit_job;

static void* fit_worker(void* arg) {
  fit_job* j = (fit_job*)arg;
  for (int64_t i = j->begin; i < j->end; ++i) j->out[i] = orc_fitness(j->obj, j->xs + i * j->stride);
  return NULL;
}

void orc_fitness_many(const orc_objective* obj, const float* xs, int64_t count, int64_t stride,
                      double* out, int32_t n_threads) {
  if (n_threads <= 1 || count < 2) {
    for (int64_t i = 0; i < count; ++i) out[i] = orc_fitness(obj, xs + i * stride);
    return;
  }
  if (n_threads > count) n_threads = (int32_t)count;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  fit_job* jobs = (fit_job*)malloc(sizeof(fit_job) * (size_t)n_threads);
  for (int32_t t = 0; t < n_threads; ++t) {
    jobs[t].obj = obj;
    jobs[t].xs = xs;
    jobs[t].stride = stride;
    jobs[t].out = out;
    jobs[t].begin = count * t / n_threads;
    jobs[t].end = count * (t + 1) / n_threads;
    pthread_create(&th[t], NULL, fit_worker, &jobs[t]);
  }
  for (int32_t t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/*
 * Gradient of the MLP cross-entropy above with respect to the flattened
 * parameters, by backpropagation in FP64 (the derivative of the same
 * formula, sample by sample in index order):
 *
 *   delta_L = (softmax(z) - onehot(y_n)) / N,
 *   dW_l += delta_l a_{l-1}^T,  db_l += delta_l,
 *   delta_{l-1} = (W_l^T delta_l) * act'(pre_{l-1}),
 *
 * with tanh' = 1 - tanh^2 and relu'(v) = 1 if v > 0 else 0 (the value 0 is
 * given slope 0).  The sphere's gradient is 2x.  Returns the objective.
 */
double orc_gradient(const orc_objective* obj, const float* x, double* grad) {
  if (obj->kind == ORC_SPHERE) {
    double s = 0.0;
    for (int64_t k = 0; k < obj->dim; ++k) {
      s += (double)x[k] * (double)x[k];
      grad[k] = 2.0 * (double)x[k];
    }
    return s;
  }
  const int32_t L = obj->n_layers;
  if (L < 1 || L > 7) return NAN;
  int64_t w_off[8], b_off[8], total_units = 0, off = 0;
  for (int32_t l = 0; l < L; ++l) {
    w_off[l] = off;
    off += (int64_t)obj->widths[l] * obj->widths[l + 1];
    b_off[l] = off;
    off += obj->widths[l + 1];
  }
  for (int32_t l = 0; l <= L; ++l) total_units += obj->widths[l];
  for (int64_t k = 0; k < off; ++k) grad[k] = 0.0;
  /* a[l] holds layer l's output for the current sample (a[0] = input),
   * pre[l] its pre-activation, delta[l] the loss derivative wrt pre[l] */
  double* a = (double*)malloc(sizeof(double) * (size_t)total_units);
  double* pre = (double*)malloc(sizeof(double) * (size_t)total_units);
  double* delta = (double*)malloc(sizeof(double) * (size_t)total_units);
  int64_t start[9];
  start[0] = 0;
  for (int32_t l = 0; l < L; ++l) start[l + 1] = start[l] + obj->widths[l];
  const double inv_n = 1.0 / (double)obj->n_samples;
  double total = 0.0;
  for (int64_t n = 0; n < obj->n_samples; ++n) {
    const int32_t d0 = obj->widths[0];
    for (int32_t i = 0; i < d0; ++i) a[i] = (double)obj->X[n * d0 + i];
    for (int32_t l = 0; l < L; ++l) {
      const int32_t fan_in = obj->widths[l], fan_out = obj->widths[l + 1];
      const float* W = x + w_off[l];
      const float* bias = x + b_off[l];
      const double* ain = a + start[l];
      double* zout = pre + start[l + 1];
      double* aout = a + start[l + 1];
      for (int32_t j = 0; j < fan_out; ++j) {
        double s = (double)bias[j];
        for (int32_t i = 0; i < fan_in; ++i) s += (double)W[(int64_t)j * fan_in + i] * ain[i];
        zout[j] = s;
        aout[j] = (l + 1 < L) ? act(obj->acts[l], s) : s;
      }
    }
    const int32_t C = obj->widths[L];
    const double* z = a + start[L];
    double zmax = z[0];
    for (int32_t c = 1; c < C; ++c)
      if (z[c] > zmax) zmax = z[c];
    double se = 0.0;
    for (int32_t c = 0; c < C; ++c) se += exp(z[c] - zmax);
    total += (zmax + log(se)) - z[obj->y[n]];
    double* dL = delta + start[L];
    for (int32_t c = 0; c < C; ++c) dL[c] = (exp(z[c] - zmax) / se - (c == obj->y[n] ? 1.0 : 0.0)) * inv_n;
    for (int32_t l = L - 1; l >= 0; --l) {
      const int32_t fan_in = obj->widths[l], fan_out = obj->widths[l + 1];
      const float* W = x + w_off[l];
      const double* dout = delta + start[l + 1];
      const double* ain = a + start[l];
      double* gW = grad + w_off[l];
      double* gb = grad + b_off[l];
      for (int32_t j = 0; j < fan_out; ++j) {
        for (int32_t i = 0; i < fan_in; ++i) gW[(int64_t)j * fan_in + i] += dout[j] * ain[i];
        gb[j] += dout[j];
      }
      if (l == 0) break;
      double* din = delta + start[l];
      const double* zin = pre + start[l];
      for (int32_t i = 0; i < fan_in; ++i) {
        double s = 0.0;
        for (int32_t j = 0; j < fan_out; ++j) s += (double)W[(int64_t)j * fan_in + i] * dout[j];
        double d;
        if (obj->acts[l - 1] == ORC_TANH) {
          const double t = tanh(zin[i]);
          d = 1.0 - t * t;
        } else {
          d = zin[i] > 0.0 ? 1.0 : 0.0;
        }
        din[i] = s * d;
      }
    }
  }
  free(a);
  free(pre);
  free(delta);
  return total * inv_n;
}
