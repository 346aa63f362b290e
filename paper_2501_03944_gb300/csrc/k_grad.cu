// Gradient of the MLP cross-entropy for a few search vectors at once, and
// the hybrid refinement built on it: projected gradient descent on each
// run's elite firework (the gradient reading of the hybrid strategies the
// paper's conclusion, Sec. 5, proposes).
//
// Backpropagation as dense FP32 products over the shared batch X:
//   forward   Z_l = A_{l-1} W_l^T + b_l,  A_l = act(Z_l)
//   loss      dZ_L = (softmax(Z_L) - onehot(y)) / N
//   backward  dW_l = dZ_l^T A_{l-1},  db_l = sum_n dZ_l,
//             dZ_{l-1} = (dZ_l W_l) * act'(A_{l-1})
// One tiled FP32 kernel computes every product.  It writes split-K
// partials and a second kernel sums them in split order and applies the
// epilogue (bias and activation, activation derivative, or the scatter of
// dW_l and db_l into the flattened gradient), so the result does not
// depend on scheduling.  The bias gradient is the product with a column of
// ones appended to A_{l-1}.
#include <cuda_runtime.h>

#include "grad.cuh"
#include "mgfwa_internal.cuh"

namespace mgfwa {
namespace {

constexpr int kTile = 64;
constexpr int kBK = 16;

struct GemmArgs {
  const float* A;
  int64_t sam, sak, sar;  // element (m, k) of vector r: A[r*sar + m*sam + k*sak]
  const float* B;
  int64_t sbk, sbn, sbr;  // element (k, n) of vector r: B[r*sbr + k*sbk + n*sbn]
  int32_t b_ones;         // column of B that reads 1.0 (the bias column), or -1
  float* P;               // partials [S][R][M][Nc]
  int32_t M, Nc, K, S, kchunk, R;
};

// A_K / B_K: the operand is contiguous along k (else along m / n); the
// loaders let consecutive threads walk the contiguous dimension.
template <bool A_K, bool B_K>
__global__ void __launch_bounds__(256) k_gemm_f32(GemmArgs g) {
  __shared__ __align__(16) float As[kBK][kTile + 4];
  __shared__ __align__(16) float Bs[kBK][kTile + 4];
  const int tid = threadIdx.x;
  const int r = blockIdx.z / g.S, s = blockIdx.z % g.S;
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  const int kb = s * g.kchunk;
  const int ke = min(g.K, kb + g.kchunk);
  const float* A = g.A + (int64_t)r * g.sar;
  const float* B = g.B + (int64_t)r * g.sbr;
  const int ty = tid >> 4, tx = tid & 15;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int k0 = kb; k0 < ke; k0 += kBK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + 256 * i;
      int mm, kk;
      if (A_K) {
        kk = idx & 15;
        mm = idx >> 4;
      } else {
        mm = idx & 63;
        kk = idx >> 6;
      }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < g.M && k < ke) ? A[(int64_t)m * g.sam + (int64_t)k * g.sak] : 0.f;
      int nn;
      if (B_K) {
        kk = idx & 15;
        nn = idx >> 4;
      } else {
        nn = idx & 63;
        kk = idx >> 6;
      }
      const int n = n0 + nn, k2 = k0 + kk;
      float v = 0.f;
      if (k2 < ke && n < g.Nc) v = n == g.b_ones ? 1.f : B[(int64_t)k2 * g.sbk + (int64_t)n * g.sbn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* P = g.P + ((int64_t)s * g.R + r) * (int64_t)g.M * g.Nc;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n < g.Nc) P[(int64_t)m * g.Nc + n] = acc[i][j];
    }
  }
}

enum { kRedBiasAct = 0, kRedBias = 1, kRedDact = 2, kRedGrad = 3 };

struct RedArgs {
  const float* P;
  int32_t S, R, M, Nc;
  int32_t mode, act;
  const float* bias;  // kRedBiasAct / kRedBias: bias[r*ldv + n]
  int64_t ldv;
  float* out;          // [R][M][Nc] (modes 0-2)
  const float* aprev;  // kRedDact: [R][M][Nc] activations whose derivative multiplies
  float* grad;         // kRedGrad: grad[r*ldv + w_off + m*(Nc-1) + n], bias column to b_off + m
  int64_t w_off, b_off;
};

__device__ __forceinline__ float act_f(int act, float v) { return act == kActTanh ? tanhf(v) : fmaxf(v, 0.f); }
// derivative from the activation's output a: tanh' = 1 - a^2, relu' = [a > 0]
__device__ __forceinline__ float dact_f(int act, float a) {
  return act == kActTanh ? fmaf(-a, a, 1.f) : (a > 0.f ? 1.f : 0.f);
}

__global__ void k_reduce_epi(RedArgs a) {
  const int64_t per = (int64_t)a.M * a.Nc;
  const int64_t total = per * a.R;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / per);
    const int64_t rem = idx - (int64_t)r * per;
    const int m = (int)(rem / a.Nc), n = (int)(rem - (int64_t)m * a.Nc);
    float v = 0.f;
    for (int s = 0; s < a.S; ++s) v += a.P[((int64_t)s * a.R + r) * per + rem];
    switch (a.mode) {
      case kRedBiasAct:
        a.out[idx] = act_f(a.act, v + a.bias[(int64_t)r * a.ldv + n]);
        break;
      case kRedBias:
        a.out[idx] = v + a.bias[(int64_t)r * a.ldv + n];
        break;
      case kRedDact:
        a.out[idx] = v * dact_f(a.act, a.aprev[idx]);
        break;
      default: {
        float* g = a.grad + (int64_t)r * a.ldv;
        if (n < a.Nc - 1)
          g[a.w_off + (int64_t)m * (a.Nc - 1) + n] = v;
        else
          g[a.b_off + m] = v;
      }
    }
  }
}

// Per sample: loss = logsumexp(z) - z_y; with want_grad, z is overwritten
// by dZ = (softmax(z) - onehot(y)) / N.
__global__ void k_ce_grad(float* z, const int32_t* y, int64_t N, int32_t C, int32_t R, float* loss,
                          int32_t want_grad) {
  const int64_t total = (int64_t)R * N;
  const float inv_n = 1.0f / (float)N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    float* row = z + idx * C;
    const int64_t n = idx % N;
    const int yn = y[n];
    float zmax = row[0];
    for (int c = 1; c < C; ++c) zmax = fmaxf(zmax, row[c]);
    float se = 0.f;
    for (int c = 0; c < C; ++c) se += expf(row[c] - zmax);
    loss[idx] = (zmax + logf(se)) - row[yn];
    if (want_grad) {
      for (int c = 0; c < C; ++c) {
        const float p = expf(row[c] - zmax) / se;
        row[c] = (p - (c == yn ? 1.f : 0.f)) * inv_n;
      }
    }
  }
}

// f[r] = mean of loss[r][0..N): per-thread sums in sample order, then a
// fixed tree, so the value does not depend on scheduling.
__global__ void __launch_bounds__(256) k_loss_mean(const float* loss, int64_t N, float* f) {
  __shared__ float part[256];
  const float* l = loss + (int64_t)blockIdx.x * N;
  float s = 0.f;
  for (int64_t n = threadIdx.x; n < N; n += 256) s += l[n];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) f[blockIdx.x] = part[0] / (float)N;
}

// w <- min(max(fma(-lr, g, w), lb), ub) on the D real coordinates.
__global__ void k_sgd(float* w, const float* g, int32_t R, int64_t D, int64_t Dp, float lr, float lb, float ub) {
  const int64_t total = (int64_t)R * D;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / D, k = idx - r * D;
    const int64_t o = r * Dp + k;
    w[o] = fminf(fmaxf(__fmaf_rn(-lr, g[o], w[o]), lb), ub);
  }
}

// Per run: its elite firework (first minimum of the fireworks' fitness),
// copied into the refinement buffer.
__global__ void __launch_bounds__(256) k_refine_pick(const float* fw_x, const float* fw_f, int32_t mu, int64_t Dp,
                                                     float* w, int32_t* elite) {
  __shared__ int e_s;
  const int r = blockIdx.x;
  if (threadIdx.x == 0) {
    int e = 0;
    for (int i = 1; i < mu; ++i)
      if (rank_key(fw_f[(int64_t)r * mu + i]) < rank_key(fw_f[(int64_t)r * mu + e])) e = i;
    e_s = e;
    elite[r] = e;
  }
  __syncthreads();
  const float4* src = reinterpret_cast<const float4*>(fw_x + ((int64_t)r * mu + e_s) * Dp);
  float4* dst = reinterpret_cast<float4*>(w + (int64_t)r * Dp);
  for (int64_t k = threadIdx.x; k < Dp / 4; k += 256) dst[k] = src[k];
}

// Per run: keep the refined vector if its fitness is strictly better than
// the elite firework's; then update the run's best-so-far the same way.
__global__ void __launch_bounds__(256) k_refine_accept(const float* w, const float* fr, const int32_t* elite,
                                                       float* fw_x, float* fw_f, float* best_x, float* best_f,
                                                       int32_t mu, int64_t Dp) {
  const int r = blockIdx.x;
  const int64_t z = (int64_t)r * mu + elite[r];
  const float f = fr[r];
  const bool take = rank_key(f) < rank_key(fw_f[z]);
  const bool best = take && rank_key(f) < rank_key(best_f[r]);
  __syncthreads();  // every thread has read fw_f[z] and best_f[r] before they change
  if (!take) return;
  const float4* src = reinterpret_cast<const float4*>(w + (int64_t)r * Dp);
  float4* dx = reinterpret_cast<float4*>(fw_x + z * Dp);
  float4* db = reinterpret_cast<float4*>(best_x + (int64_t)r * Dp);
  for (int64_t k = threadIdx.x; k < Dp / 4; k += 256) {
    const float4 v = src[k];
    dx[k] = v;
    if (best) db[k] = v;
  }
  if (threadIdx.x == 0) {
    fw_f[z] = f;
    if (best) best_f[r] = f;
  }
}

int grid_for(int64_t total, int threads = 256) {
  const int64_t b = (total + threads - 1) / threads;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

// Split count for an M x Nc product with reduction length K over R vectors:
// enough blocks to cover the SMs about three times, at least 64 of K per split.
int splits_for(int64_t M, int64_t Nc, int64_t K, int R, int num_sms) {
  const int64_t tiles = ((M + kTile - 1) / kTile) * ((Nc + kTile - 1) / kTile) * R;
  int64_t s = (3 * (int64_t)num_sms + tiles - 1) / tiles;
  const int64_t kmax = (K + 63) / 64;
  if (s > kmax) s = kmax;
  if (s > 32) s = 32;
  return (int)(s < 1 ? 1 : s);
}

int64_t round_floats(int64_t n) { return (n + 63) / 64 * 64; }

struct Gemm {
  int64_t M, Nc, K;
  int S;
};

// The products of one gradient evaluation, in launch order, with their
// split counts: forward l = 1..L, then per layer L..1 the weight gradient
// and (l > 1) the back-propagated derivative.
int gemm_list(const Mlp& mlp, int R, int num_sms, Gemm* out) {
  const int L = mlp.n_layers;
  const int64_t N = mlp.N;
  int n = 0;
  for (int l = 1; l <= L; ++l) {
    const int64_t fi = mlp.widths[l - 1], fo = mlp.widths[l];
    out[n++] = {N, fo, fi, splits_for(N, fo, fi, R, num_sms)};
  }
  for (int l = L; l >= 1; --l) {
    const int64_t fi = mlp.widths[l - 1], fo = mlp.widths[l];
    out[n++] = {fo, fi + 1, N, splits_for(fo, fi + 1, N, R, num_sms)};
    if (l > 1) out[n++] = {N, fi, fo, splits_for(N, fi, fo, R, num_sms)};
  }
  return n;
}

}  // namespace

GradPlan grad_plan(const Mlp& mlp, int32_t R, int32_t num_sms) {
  GradPlan gp{};
  gp.R = R;
  gp.num_sms = num_sms;
  const int L = mlp.n_layers;
  const int64_t N = mlp.N;
  int64_t off = 0;
  for (int l = 1; l <= L; ++l) {
    gp.act_off[l] = off;  // act[l] (hidden) or, for l = L, the logits / dZ_L
    off += round_floats((int64_t)R * N * mlp.widths[l]);
  }
  for (int l = 1; l < L; ++l) {
    gp.dz_off[l] = off;
    off += round_floats((int64_t)R * N * mlp.widths[l]);
  }
  gp.loss_off = off;
  off += round_floats((int64_t)R * N);
  Gemm gl[8];
  const int ng = gemm_list(mlp, R, num_sms, gl);
  int64_t pmax = 0;
  for (int i = 0; i < ng; ++i) {
    const int64_t v = (int64_t)gl[i].S * R * gl[i].M * gl[i].Nc;
    if (v > pmax) pmax = v;
  }
  gp.partial_off = off;
  off += round_floats(pmax);
  gp.floats = off;
  return gp;
}

namespace {

struct Enq {
  cudaStream_t s;
  int n = 0;
  bool ok = true;
  void gemm(const GemmArgs& g) {
    const dim3 grid((unsigned)((g.Nc + kTile - 1) / kTile), (unsigned)((g.M + kTile - 1) / kTile),
                    (unsigned)(g.R * g.S));
    const bool ak = g.sak == 1, bk = g.sbk == 1;
    if (ak && bk)
      k_gemm_f32<true, true><<<grid, 256, 0, s>>>(g);
    else if (ak)
      k_gemm_f32<true, false><<<grid, 256, 0, s>>>(g);
    else if (bk)
      k_gemm_f32<false, true><<<grid, 256, 0, s>>>(g);
    else
      k_gemm_f32<false, false><<<grid, 256, 0, s>>>(g);
    note();
  }
  void reduce(const RedArgs& a) {
    k_reduce_epi<<<grid_for((int64_t)a.R * a.M * a.Nc), 256, 0, s>>>(a);
    note();
  }
  void note() {
    if (cudaPeekAtLastError() != cudaSuccess) ok = false;
    ++n;
  }
};

GemmArgs make_gemm(const Gemm& sh, int R, float* P) {
  GemmArgs g{};
  g.M = (int32_t)sh.M;
  g.Nc = (int32_t)sh.Nc;
  g.K = (int32_t)sh.K;
  g.S = sh.S;
  g.kchunk = (int32_t)((sh.K + sh.S - 1) / sh.S + kBK - 1) / kBK * kBK;
  g.R = R;
  g.P = P;
  g.b_ones = -1;
  return g;
}

}  // namespace

int launch_grad(const GradPlan& gp, const Mlp& mlp, const float* W, int64_t ld, float* scratch, float* G,
                float* f_out, cudaStream_t s) {
  const int L = mlp.n_layers;
  const int R = gp.R;
  const int64_t N = mlp.N;
  Gemm gl[8];
  gemm_list(mlp, R, gp.num_sms, gl);
  float* P = scratch + gp.partial_off;
  float* loss = scratch + gp.loss_off;
  auto act = [&](int l) { return scratch + gp.act_off[l]; };
  auto dz = [&](int l) { return l == L ? scratch + gp.act_off[L] : scratch + gp.dz_off[l]; };
  Enq q{s};
  int gi = 0;
  // forward
  for (int l = 1; l <= L; ++l) {
    const int64_t fi = mlp.widths[l - 1];
    GemmArgs g = make_gemm(gl[gi++], R, P);
    if (l == 1) {
      g.A = mlp.X, g.sam = fi, g.sak = 1, g.sar = 0;
    } else {
      g.A = act(l - 1), g.sam = fi, g.sak = 1, g.sar = N * fi;
    }
    g.B = W + mlp.w_off[l - 1], g.sbk = 1, g.sbn = fi, g.sbr = ld;
    q.gemm(g);
    RedArgs a{};
    a.P = P, a.S = g.S, a.R = R, a.M = g.M, a.Nc = g.Nc;
    a.mode = l < L ? kRedBiasAct : kRedBias;
    a.act = l < L ? mlp.acts[l - 1] : 0;
    a.bias = W + mlp.b_off[l - 1], a.ldv = ld;
    a.out = act(l);
    q.reduce(a);
  }
  const int want_grad = G != nullptr;
  k_ce_grad<<<grid_for((int64_t)R * N), 256, 0, s>>>(act(L), mlp.y, N, mlp.widths[L], R, loss, want_grad);
  q.note();
  if (f_out) {
    k_loss_mean<<<R, 256, 0, s>>>(loss, N, f_out);
    q.note();
  }
  if (want_grad) {
    for (int l = L; l >= 1; --l) {
      const int64_t fi = mlp.widths[l - 1], fo = mlp.widths[l];
      // dW_l, db_l = dZ_l^T [A_{l-1} | 1]
      GemmArgs g = make_gemm(gl[gi++], R, P);
      g.A = dz(l), g.sam = 1, g.sak = fo, g.sar = N * fo;
      if (l == 1) {
        g.B = mlp.X, g.sbk = fi, g.sbn = 1, g.sbr = 0;
      } else {
        g.B = act(l - 1), g.sbk = fi, g.sbn = 1, g.sbr = N * fi;
      }
      g.b_ones = (int32_t)fi;
      q.gemm(g);
      RedArgs a{};
      a.P = P, a.S = g.S, a.R = R, a.M = g.M, a.Nc = g.Nc;
      a.mode = kRedGrad;
      a.grad = G, a.ldv = ld, a.w_off = mlp.w_off[l - 1], a.b_off = mlp.b_off[l - 1];
      q.reduce(a);
      if (l > 1) {
        // dZ_{l-1} = (dZ_l W_l) * act'(A_{l-1})
        GemmArgs h = make_gemm(gl[gi++], R, P);
        h.A = dz(l), h.sam = fo, h.sak = 1, h.sar = N * fo;
        h.B = W + mlp.w_off[l - 1], h.sbk = fi, h.sbn = 1, h.sbr = ld;
        q.gemm(h);
        RedArgs b{};
        b.P = P, b.S = h.S, b.R = R, b.M = h.M, b.Nc = h.Nc;
        b.mode = kRedDact;
        b.act = mlp.acts[l - 2];
        b.aprev = act(l - 1);
        b.out = dz(l - 1);
        q.reduce(b);
      }
    }
  }
  return q.ok ? q.n : -1;
}

int launch_sgd(float* w, const float* g, int32_t R, int64_t D, int64_t Dp, float lr, float lb, float ub,
               cudaStream_t s) {
  k_sgd<<<grid_for((int64_t)R * D), 256, 0, s>>>(w, g, R, D, Dp, lr, lb, ub);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_refine_pick(const float* fw_x, const float* fw_f, int32_t R, int32_t mu, int64_t Dp, float* w,
                       int32_t* elite, cudaStream_t s) {
  k_refine_pick<<<R, 256, 0, s>>>(fw_x, fw_f, mu, Dp, w, elite);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_refine_accept(const float* w, const float* fr, const int32_t* elite, float* fw_x, float* fw_f,
                         float* best_x, float* best_f, int32_t R, int32_t mu, int64_t Dp, cudaStream_t s) {
  k_refine_accept<<<R, 256, 0, s>>>(w, fr, elite, fw_x, fw_f, best_x, best_f, mu, Dp);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mgfwa
