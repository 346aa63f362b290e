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

constexpr int kBK = 8;

__device__ __forceinline__ float act_f(int act, float v) { return act == kActTanh ? tanhf(v) : fmaxf(v, 0.f); }
// derivative from the activation's output a: tanh' = 1 - a^2, relu' = [a > 0]
__device__ __forceinline__ float dact_f(int act, float a) {
  return act == kActTanh ? fmaf(-a, a, 1.f) : (a > 0.f ? 1.f : 0.f);
}

enum { kEpiPartial = 0, kEpiBias = 1, kEpiBiasAct = 2 };

struct GemmArgs {
  const float* A;
  int64_t sam, sak, sar;  // element (m, k) of vector r: A[r*sar + m*sam + k*sak]
  const float* B;
  int64_t sbk, sbn, sbr;  // element (k, n) of vector r: B[vb*sbr + k*sbk + n*sbn], vb = idx ? idx[r] : r
  const int32_t* idx;     // optional gather of B's vector
  int32_t a_ones;         // row of A that reads 1.0 (the bias row), or -1
  int32_t b_ones;         // column of B that reads 1.0 (the bias column), or -1
  float* P;               // kEpiPartial: partials [S][R][M][Nc]
  int32_t M, Nc, K, S, kchunk, R;
  // fused epilogue (one split): out[r][m][n] = [act](acc + bias[vb*ldv + n])
  int32_t epi, act;
  const float* bias;
  int64_t ldv;
  float* out;
};

// C[m][n] = sum_k A[m][k] B[k][n] over one k-chunk, for a BM x BN tile:
// 256 threads, each BM/16 rows x BN/16 columns in 4-wide groups (rows
// ty*4 + i [and 64 + ty*4 + i], columns tx*4 + j [and 64 + tx*4 + j]), the
// operands staged through two shared-memory buffers of 8 k-steps so that the
// next chunk's global loads overlap the current chunk's FMAs.  Every output
// accumulates its products in k order, whatever the tile shape.  A_K / B_K:
// the operand is contiguous along k (else along m / n); VEC: 16-byte loads
// along the contiguous dimension (its extent and the other strides multiples
// of 4).
template <int BM, int BN, bool A_K, bool B_K, bool VEC>
__global__ void __launch_bounds__(256, 2) k_gemm_f32(GemmArgs g) {
  griddep_wait();
  griddep_launch_dependents();
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int EA = BM * kBK / 256, EB = BN * kBK / 256;  // scalar loads per thread
  constexpr int PADM = BM + 4, PADN = BN + 4;
  __shared__ __align__(16) float As[2][kBK][PADM];
  __shared__ __align__(16) float Bs[2][kBK][PADN];
  const int tid = threadIdx.x;
  const int r = blockIdx.z / g.S, s = blockIdx.z % g.S;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = s * g.kchunk;
  const int ke = min(g.K, kb + g.kchunk);
  const int vb = g.idx ? g.idx[r] : r;
  const float* A = g.A + (int64_t)r * g.sar;
  const float* B = g.B + (int64_t)vb * g.sbr;
  const int n_real = g.b_ones >= 0 ? g.b_ones : g.Nc;  // columns read from B
  const int m_real = g.a_ones >= 0 ? g.a_ones : g.M;   // rows read from A
  const int ty = tid >> 4, tx = tid & 15;

  float ra[4], rb[4];  // one chunk's loads in flight
  auto load = [&](int k0) {
    if (VEC) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < 2 * BM) {
        int m, k;
        if (A_K) {
          m = m0 + (tid >> 1), k = k0 + (tid & 1) * 4;
        } else {
          m = m0 + (tid % (BM / 4)) * 4, k = k0 + tid / (BM / 4);
        }
        if (k < ke) {
          if (m < m_real)
            v = A_K ? *reinterpret_cast<const float4*>(A + (int64_t)m * g.sam + k)
                    : *reinterpret_cast<const float4*>(A + m + (int64_t)k * g.sak);
          else if (m == g.a_ones)
            v = A_K ? make_float4(1.f, 1.f, 1.f, 1.f) : make_float4(1.f, 0.f, 0.f, 0.f);
        }
      }
      ra[0] = v.x, ra[1] = v.y, ra[2] = v.z, ra[3] = v.w;
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < 2 * BN) {
        int n, k;
        if (B_K) {
          n = n0 + (tid >> 1), k = k0 + (tid & 1) * 4;
        } else {
          n = n0 + (tid % (BN / 4)) * 4, k = k0 + tid / (BN / 4);
        }
        if (k < ke) {
          if (n < n_real)
            w = B_K ? *reinterpret_cast<const float4*>(B + (int64_t)n * g.sbn + k)
                    : *reinterpret_cast<const float4*>(B + (int64_t)k * g.sbk + n);
          else if (n == g.b_ones)
            w = B_K ? make_float4(1.f, 1.f, 1.f, 1.f) : make_float4(1.f, 0.f, 0.f, 0.f);
        }
      }
      rb[0] = w.x, rb[1] = w.y, rb[2] = w.z, rb[3] = w.w;
    } else {
#pragma unroll
      for (int i = 0; i < EA; ++i) {
        const int e = tid + 256 * i;
        const int mm = A_K ? e >> 3 : e % BM, kk = A_K ? e & 7 : e / BM;
        const int m = m0 + mm, k = k0 + kk;
        float va = 0.f;
        if (k < ke) {
          if (m < m_real)
            va = A[(int64_t)m * g.sam + (int64_t)k * g.sak];
          else if (m == g.a_ones)
            va = 1.f;
        }
        ra[i] = va;
      }
#pragma unroll
      for (int i = 0; i < EB; ++i) {
        const int e = tid + 256 * i;
        const int nn = B_K ? e >> 3 : e % BN, kk = B_K ? e & 7 : e / BN;
        const int n = n0 + nn, k = k0 + kk;
        float vb2 = 0.f;
        if (k < ke) {
          if (n < n_real)
            vb2 = B[(int64_t)k * g.sbk + (int64_t)n * g.sbn];
          else if (n == g.b_ones)
            vb2 = 1.f;
        }
        rb[i] = vb2;
      }
    }
  };
  auto stash = [&](int buf) {
    if (VEC) {
      if (tid < 2 * BM) {
        if (A_K) {
          const int mm = tid >> 1, kq = (tid & 1) * 4;
#pragma unroll
          for (int i = 0; i < 4; ++i) As[buf][kq + i][mm] = ra[i];
        } else {
          *reinterpret_cast<float4*>(&As[buf][tid / (BM / 4)][(tid % (BM / 4)) * 4]) =
              make_float4(ra[0], ra[1], ra[2], ra[3]);
        }
      }
      if (tid < 2 * BN) {
        if (B_K) {
          const int nn = tid >> 1, kq = (tid & 1) * 4;
#pragma unroll
          for (int i = 0; i < 4; ++i) Bs[buf][kq + i][nn] = rb[i];
        } else {
          *reinterpret_cast<float4*>(&Bs[buf][tid / (BN / 4)][(tid % (BN / 4)) * 4]) =
              make_float4(rb[0], rb[1], rb[2], rb[3]);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < EA; ++i) {
        const int e = tid + 256 * i;
        if (A_K)
          As[buf][e & 7][e >> 3] = ra[i];
        else
          As[buf][e / BM][e % BM] = ra[i];
      }
#pragma unroll
      for (int i = 0; i < EB; ++i) {
        const int e = tid + 256 * i;
        if (B_K)
          Bs[buf][e & 7][e >> 3] = rb[i];
        else
          Bs[buf][e / BN][e % BN] = rb[i];
      }
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  if (kb < ke) {
    load(kb);
    stash(0);
  }
  __syncthreads();
  int buf = 0;
  for (int k0 = kb; k0 < ke; k0 += kBK) {
    const bool more = k0 + kBK < ke;
    if (more) load(k0 + kBK);
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float av[TM], bv[TN];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      av[0] = a0.x, av[1] = a0.y, av[2] = a0.z, av[3] = a0.w;
      if (TM == 8) {
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
        av[TM - 4] = a1.x, av[TM - 3] = a1.y, av[TM - 2] = a1.z, av[TM - 1] = a1.w;
      }
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      bv[0] = b0.x, bv[1] = b0.y, bv[2] = b0.z, bv[3] = b0.w;
      if (TN == 8) {
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
        bv[TN - 4] = b1.x, bv[TN - 3] = b1.y, bv[TN - 2] = b1.z, bv[TN - 1] = b1.w;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* P = g.P + ((int64_t)s * g.R + r) * (int64_t)g.M * g.Nc;
  float* O = g.out + (int64_t)r * g.M * g.Nc;
  const float* bias = g.bias + (int64_t)vb * g.ldv;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (n >= g.Nc) continue;
      if (g.epi == kEpiPartial) {
        P[(int64_t)m * g.Nc + n] = acc[i][j];
      } else {
        const float v = acc[i][j] + bias[n];
        O[(int64_t)m * g.Nc + n] = g.epi == kEpiBiasAct ? act_f(g.act, v) : v;
      }
    }
  }
}

enum { kRedBiasAct = 0, kRedBias = 1, kRedDact = 2, kRedGrad = 3, kRedGradT = 4 };

struct RedArgs {
  const float* P;
  int32_t S, R, M, Nc;
  int32_t mode, act;
  const float* bias;  // kRedBiasAct / kRedBias: bias[vb*ldv + n], vb = idx ? idx[r] : r
  const int32_t* idx;
  int64_t ldv;
  float* out;          // [R][M][Nc] (modes 0-2)
  const float* aprev;  // kRedDact: [R][M][Nc] activations whose derivative multiplies
  float* grad;         // kRedGrad: grad[r*ldv + w_off + m*(Nc-1) + n], bias column to b_off + m;
                       // kRedGradT: grad[r*ldv + w_off + n*(M-1) + m], bias row to b_off + n
  int64_t w_off, b_off;
};


__global__ void k_reduce_epi(RedArgs a) {
  griddep_wait();
  griddep_launch_dependents();
  const int64_t per = (int64_t)a.M * a.Nc;
  const int64_t total = per * a.R;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / per);
    const int64_t rem = idx - (int64_t)r * per;
    const int m = (int)(rem / a.Nc), n = (int)(rem - (int64_t)m * a.Nc);
    // in split order; eight loads in flight at a time
    float v = 0.f;
    int s = 0;
    for (; s + 8 <= a.S; s += 8) {
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = a.P[((int64_t)(s + u) * a.R + r) * per + rem];
#pragma unroll
      for (int u = 0; u < 8; ++u) v += t[u];
    }
    for (; s < a.S; ++s) v += a.P[((int64_t)s * a.R + r) * per + rem];
    switch (a.mode) {
      case kRedBiasAct:
        a.out[idx] = act_f(a.act, v + a.bias[(int64_t)(a.idx ? a.idx[r] : r) * a.ldv + n]);
        break;
      case kRedBias:
        a.out[idx] = v + a.bias[(int64_t)(a.idx ? a.idx[r] : r) * a.ldv + n];
        break;
      case kRedDact:
        a.out[idx] = v * dact_f(a.act, a.aprev[idx]);
        break;
      case kRedGrad: {
        float* g = a.grad + (int64_t)r * a.ldv;
        if (n < a.Nc - 1)
          g[a.w_off + (int64_t)m * (a.Nc - 1) + n] = v;
        else
          g[a.b_off + m] = v;
        break;
      }
      default: {  // kRedGradT: the transposed product [A | 1]^T dZ, rows i, columns j
        float* g = a.grad + (int64_t)r * a.ldv;
        if (m < a.M - 1)
          g[a.w_off + (int64_t)n * (a.M - 1) + m] = v;
        else
          g[a.b_off + n] = v;
      }
    }
  }
}

// f[r] = mean of loss[r][0..N): per-thread sums in sample order, then a
// fixed tree, so the value does not depend on scheduling.
__global__ void __launch_bounds__(256) k_loss_mean(const float* loss, int64_t N, float* f, const int32_t* idx) {
  griddep_wait();
  griddep_launch_dependents();
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
  if (threadIdx.x == 0) f[idx ? idx[blockIdx.x] : (int)blockIdx.x] = part[0] / (float)N;
}

// w <- min(max(fma(-lr, g, w), lb), ub) on the D real coordinates.
__global__ void k_sgd(float* w, const float* g, int32_t R, int64_t D, int64_t Dp, float lr, float lb, float ub) {
  griddep_wait();
  griddep_launch_dependents();
  const int64_t total = (int64_t)R * D;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / D, k = idx - r * D;
    const int64_t o = r * Dp + k;
    w[o] = fminf(fmaxf(__fmaf_rn(-lr, g[o], w[o]), lb), ub);
  }
}

// Per run r (blockIdx.y): its elite firework, the first minimum of the
// fireworks' fitness (every block finds the same one), copied into the
// refinement buffer by all blocks of the run, each a slice of the row.
__global__ void __launch_bounds__(256) k_refine_pick(const float* fw_x, const float* fw_f, int32_t mu, int64_t Dp,
                                                     float* w, int32_t* elite) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ int e_s;
  const int r = blockIdx.y;
  if (threadIdx.x == 0) {
    int e = 0;
    for (int i = 1; i < mu; ++i)
      if (rank_key(fw_f[(int64_t)r * mu + i]) < rank_key(fw_f[(int64_t)r * mu + e])) e = i;
    e_s = e;
    if (blockIdx.x == 0) elite[r] = e;
  }
  __syncthreads();
  const float4* src = reinterpret_cast<const float4*>(fw_x + ((int64_t)r * mu + e_s) * Dp);
  float4* dst = reinterpret_cast<float4*>(w + (int64_t)r * Dp);
  for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < Dp / 4; k += (int64_t)gridDim.x * 256)
    dst[k] = src[k];
}

// Per run (one thread each): keep the refined vector if its fitness is
// strictly better than the elite firework's, and likewise for the run's
// best-so-far.  flags[r]: bit 0 take, bit 1 new best; the rows are copied
// by k_refine_copy.
__global__ void k_refine_decide(const float* fr, const int32_t* elite, float* fw_f, float* best_f, int32_t mu,
                                int32_t R, int32_t* flags) {
  griddep_wait();
  griddep_launch_dependents();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int64_t z = (int64_t)r * mu + elite[r];
  const float f = fr[r];
  const bool take = rank_key(f) < rank_key(fw_f[z]);
  const bool best = take && rank_key(f) < rank_key(best_f[r]);
  if (take) fw_f[z] = f;
  if (best) best_f[r] = f;
  flags[r] = (take ? 1 : 0) | (best ? 2 : 0);
}

__global__ void __launch_bounds__(256) k_refine_copy(const float* w, const int32_t* elite, const int32_t* flags,
                                                     float* fw_x, float* best_x, int32_t mu, int64_t Dp) {
  griddep_wait();
  griddep_launch_dependents();
  const int r = blockIdx.y;
  const int fl = flags[r];
  if (!(fl & 1)) return;
  const int64_t z = (int64_t)r * mu + elite[r];
  const float4* src = reinterpret_cast<const float4*>(w + (int64_t)r * Dp);
  float4* dx = reinterpret_cast<float4*>(fw_x + z * Dp);
  float4* db = reinterpret_cast<float4*>(best_x + (int64_t)r * Dp);
  for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < Dp / 4; k += (int64_t)gridDim.x * 256) {
    const float4 v = src[k];
    dx[k] = v;
    if (fl & 2) db[k] = v;
  }
}

// The output layer of one 32-sample tile of vector r, fused: logits
// z = W_L a + b_L from the tile's last hidden activations, the per-sample
// loss, and with want_grad dZ_L = (softmax(z) - onehot(y)) / N, the
// back-propagated dZ_{L-1} = (dZ_L W_L) * act'(a) and the tile's share of
// [dW_L | db_L] = dZ_L^T [a | 1] into P[tile][r][C][h + 1] (summed over tiles
// in order afterwards).  Shared memory: a [32][h+1], W_L [C][h+1], b_L [C],
// z / dZ [32][C+1] (rows padded against bank conflicts).
constexpr int kTailM = 32;

struct TailArgs {
  const float* A;      // [R][N][h] activations of layer L-1
  const float* W;      // search vectors (row vb = idx ? idx[r] : r, stride ld)
  const int32_t* idx;
  int64_t ld, w_off, b_off;
  const int32_t* y;
  int64_t N;
  int32_t h, C, act, want_grad;
  float* loss;         // [R][N]
  float* dz_prev;      // [R][N][h]
  float* P;            // [mtiles][R][C][h+1]
  int32_t R;
};

size_t tail_smem_bytes(int h, int C) {
  return sizeof(float) * ((size_t)kTailM * (h + 1) + (size_t)C * (h + 1) + C + (size_t)kTailM * (C + 1));
}

__global__ void __launch_bounds__(256) k_out_layer(TailArgs t) {
  griddep_wait();
  griddep_launch_dependents();
  extern __shared__ float sm[];
  const int h = t.h, C = t.C, hp = h + 1, cp = C + 1;
  float* As = sm;                       // [128][hp]
  float* Ws = As + kTailM * hp;         // [C][hp]
  float* bs = Ws + C * hp;              // [C]
  float* Zs = bs + C;                   // [128][cp]
  const int tile = blockIdx.x, r = blockIdx.y;
  const int64_t n0 = (int64_t)tile * kTailM;
  const int rows = t.N - n0 < kTailM ? (int)(t.N - n0) : kTailM;
  const float* W = t.W + (int64_t)(t.idx ? t.idx[r] : r) * t.ld;
  const float* A = t.A + ((int64_t)r * t.N + n0) * h;
  for (int e = threadIdx.x; e < kTailM * h; e += 256) {
    const int sI = e / h, j = e - sI * h;
    As[sI * hp + j] = sI < rows ? A[(int64_t)sI * h + j] : 0.f;
  }
  for (int e = threadIdx.x; e < C * h; e += 256) {
    const int c = e / h, j = e - c * h;
    Ws[c * hp + j] = W[t.w_off + e];
  }
  for (int c = threadIdx.x; c < C; c += 256) bs[c] = W[t.b_off + c];
  __syncthreads();
  for (int e = threadIdx.x; e < kTailM * C; e += 256) {
    const int sI = e / C, c = e - sI * C;
    float z = bs[c];
    const float* a = As + sI * hp;
    const float* wc = Ws + c * hp;
    for (int j = 0; j < h; ++j) z = fmaf(a[j], wc[j], z);
    Zs[sI * cp + c] = z;
  }
  __syncthreads();
  const float inv_n = 1.0f / (float)t.N;
  if (threadIdx.x < kTailM) {
    const int sI = threadIdx.x;
    float* z = Zs + sI * cp;
    if (sI < rows) {
      const int yn = t.y[n0 + sI];
      float zmax = z[0];
      for (int c = 1; c < C; ++c) zmax = fmaxf(zmax, z[c]);
      float se = 0.f;
      for (int c = 0; c < C; ++c) se += expf(z[c] - zmax);
      t.loss[(int64_t)r * t.N + n0 + sI] = (zmax + logf(se)) - z[yn];
      if (t.want_grad)
        for (int c = 0; c < C; ++c) z[c] = (expf(z[c] - zmax) / se - (c == yn ? 1.f : 0.f)) * inv_n;
    } else {
      for (int c = 0; c < C; ++c) z[c] = 0.f;
    }
  }
  if (!t.want_grad) return;
  __syncthreads();
  // dZ_{L-1} for the tile's valid rows
  float* dzp = t.dz_prev + ((int64_t)r * t.N + n0) * h;
  for (int e = threadIdx.x; e < rows * h; e += 256) {
    const int sI = e / h, j = e - sI * h;
    const float* dz = Zs + sI * cp;
    float v = 0.f;
    for (int c = 0; c < C; ++c) v = fmaf(dz[c], Ws[c * hp + j], v);
    dzp[e] = v * dact_f(t.act, As[sI * hp + j]);
  }
  // the tile's [dW_L | db_L]
  float* P = t.P + ((int64_t)tile * t.R + r) * C * hp;
  for (int e = threadIdx.x; e < C * hp; e += 256) {
    const int c = e / hp, j = e - c * hp;
    float v = 0.f;
    if (j < h) {
      for (int sI = 0; sI < kTailM; ++sI) v = fmaf(Zs[sI * cp + c], As[sI * hp + j], v);
    } else {
      for (int sI = 0; sI < kTailM; ++sI) v += Zs[sI * cp + c];
    }
    P[e] = v;
  }
}

int grid_for(int64_t total, int threads = 256) {
  const int64_t b = (total + threads - 1) / threads;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

// Output tile width: 64 for narrow products, else 128.
int tile_n(int64_t Nc) { return Nc <= 64 ? 64 : 128; }

// K per split of an M x Nc product with reduction length K: enough splits
// for two blocks per SM for ONE vector, at least kmin of K each, at most 32.
// It depends on the product's shape (and the device) only, never on how many
// vectors share the launch, so a vector's sums -- chunk by chunk, then the
// chunks in order -- are the same alone or batched.
int kchunk_for(int64_t M, int64_t Nc, int64_t K, int num_sms, int64_t kmin) {
  const int bn = tile_n(Nc);
  const int64_t tiles = ((M + 127) / 128) * ((Nc + bn - 1) / bn);
  int64_t s = (2 * (int64_t)num_sms + tiles - 1) / tiles;
  const int64_t kmax = (K + kmin - 1) / kmin;
  if (s > kmax) s = kmax;
  if (s > 32) s = 32;
  if (s < 1) s = 1;
  return (int)(((K + s - 1) / s + kBK - 1) / kBK * kBK);
}

int64_t round_floats(int64_t n) { return (n + 63) / 64 * 64; }

struct Gemm {
  int64_t M, Nc, K;
  int kchunk, S;
};

Gemm shape(int64_t M, int64_t Nc, int64_t K, int num_sms, int64_t kmin = 64) {
  const int kc = kchunk_for(M, Nc, K, num_sms, kmin);
  return {M, Nc, K, kc, (int)((K + kc - 1) / kc)};
}

// The products of one gradient evaluation, in launch order, with their
// split counts: forward l = 1..L-1, then per layer L-1..1 the weight
// gradient and (l > 1) the back-propagated derivative (the output layer is
// the fused k_out_layer).
int gemm_list(const Mlp& mlp, int num_sms, bool forward_only, Gemm* out) {
  const int L = mlp.n_layers;
  const int64_t N = mlp.N;
  int n = 0;
  for (int l = 1; l < L; ++l) {
    const int64_t fi = mlp.widths[l - 1], fo = mlp.widths[l];
    // objective-only plans serve many vectors at once: longer chunks, fewer partials
    out[n++] = shape(N, fo, fi, num_sms, forward_only ? 128 : 64);
  }
  if (forward_only) return n;
  for (int l = L - 1; l >= 1; --l) {
    const int64_t fi = mlp.widths[l - 1], fo = mlp.widths[l];
    out[n++] = shape(fi + 1, fo, N, num_sms);
    if (l > 1) out[n++] = shape(N, fi, fo, num_sms);
  }
  return n;
}

}  // namespace

GradPlan grad_plan(const Mlp& mlp, int32_t R, int32_t num_sms, bool forward_only) {
  GradPlan gp{};
  gp.R = R;
  gp.num_sms = num_sms;
  gp.forward_only = forward_only;
  const int L = mlp.n_layers;
  const int64_t N = mlp.N;
  int64_t off = 0;
  for (int l = 1; l < L; ++l) {
    gp.act_off[l] = off;  // activations of hidden layer l
    off += round_floats((int64_t)R * N * mlp.widths[l]);
  }
  for (int l = 1; l < L && !forward_only; ++l) {
    gp.dz_off[l] = off;
    off += round_floats((int64_t)R * N * mlp.widths[l]);
  }
  gp.loss_off = off;
  off += round_floats((int64_t)R * N);
  Gemm gl[8];
  const int ng = gemm_list(mlp, num_sms, forward_only, gl);
  // the output layer's per-tile [dW_L | db_L]
  int64_t pmax = forward_only ? 0
                              : ((N + kTailM - 1) / kTailM) * R * mlp.widths[L] * (int64_t)(mlp.widths[L - 1] + 1);
  for (int i = 0; i < ng; ++i) {
    if (i < L - 1 && gl[i].S == 1) continue;  // forward products with one chunk write no partials
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
  int num_sms;
  int n = 0;
  bool ok = true;
  template <int BM, int BN, bool AK, bool BK>
  void go(const GemmArgs& g, bool vec) {
    const dim3 grid((unsigned)((g.Nc + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM), (unsigned)(g.R * g.S));
    const cudaError_t e = vec ? launch_pdl(k_gemm_f32<BM, BN, AK, BK, true>, grid, dim3(256), 0, s, g)
                              : launch_pdl(k_gemm_f32<BM, BN, AK, BK, false>, grid, dim3(256), 0, s, g);
    if (e != cudaSuccess) ok = false;
  }
  template <int BM, int BN>
  void go_tile(const GemmArgs& g, bool vec) {
    const bool ak = g.sak == 1, bk = g.sbk == 1;
    if (ak && bk)
      go<BM, BN, true, true>(g, vec);
    else if (ak)
      go<BM, BN, true, false>(g, vec);
    else if (bk)
      go<BM, BN, false, true>(g, vec);
    else
      go<BM, BN, false, false>(g, vec);
  }
  // The tile shape does not change any sum (each output accumulates in k
  // order): 64-row tiles when 128-row tiles would leave SMs without two blocks.
  void gemm(const GemmArgs& g) {
    const int bn = tile_n(g.Nc);
    const int64_t blocks128 = (int64_t)((g.M + 127) / 128) * ((g.Nc + bn - 1) / bn) * g.R * g.S;
    const bool small = g.M <= 64 || blocks128 < 2 * (int64_t)num_sms;
    const bool vec = vec_ok(g);
    if (bn == 64) {
      if (small)
        go_tile<64, 64>(g, vec);
      else
        go_tile<128, 64>(g, vec);
    } else {
      if (small)
        go_tile<64, 128>(g, vec);
      else
        go_tile<128, 128>(g, vec);
    }
    note();
  }
  // 16-byte loads need both operands contiguous in one dimension with that
  // extent and the other strides multiples of four floats, and aligned bases.
  static bool vec_ok(const GemmArgs& g) {
    auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const int n_real = g.b_ones >= 0 ? g.b_ones : g.Nc;
    const int m_real = g.a_ones >= 0 ? g.a_ones : g.M;
    if (g.sak == 1) {
      if (g.K % 4 || g.sam % 4) return false;
    } else if (g.sam == 1) {
      if (m_real % 4 || g.sak % 4) return false;
    } else {
      return false;
    }
    if (g.sbk == 1) {
      if (g.K % 4 || g.sbn % 4) return false;
    } else if (g.sbn == 1) {
      if (n_real % 4 || g.sbk % 4) return false;
    } else {
      return false;
    }
    return aligned(g.A) && aligned(g.B) && g.sar % 4 == 0 && g.sbr % 4 == 0;
  }
  void reduce(const RedArgs& a) {
    if (launch_pdl(k_reduce_epi, dim3(grid_for((int64_t)a.R * a.M * a.Nc)), dim3(256), 0, s, a) != cudaSuccess)
      ok = false;
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
  g.kchunk = sh.kchunk;
  g.R = R;
  g.P = P;
  g.a_ones = -1;
  g.b_ones = -1;
  g.epi = kEpiPartial;
  return g;
}

}  // namespace

bool l1_on_tensor_cores(const GradPlan& gp, const Mlp& mlp, const L1Plan* l1) {
  const int64_t l1_ctas = (int64_t)gp.R * ((mlp.N + 127) / 128);
  return l1 && l1->ready && 2 * l1_ctas >= gp.num_sms;
}

int launch_grad(const GradPlan& gp, const Mlp& mlp, const float* W, int64_t ld, float* scratch, float* G,
                float* f_out, cudaStream_t s, const int32_t* idx, const L1Plan* l1, uint32_t* status) {
  const int L = mlp.n_layers;
  const int R = gp.R;
  const int64_t N = mlp.N;
  const bool want_grad = G != nullptr;
  if ((want_grad && (gp.forward_only || idx)) || L < 2) return -1;
  Gemm gl[8];
  gemm_list(mlp, gp.num_sms, gp.forward_only, gl);
  float* P = scratch + gp.partial_off;
  float* loss = scratch + gp.loss_off;
  auto act = [&](int l) { return scratch + gp.act_off[l]; };
  auto dz = [&](int l) { return scratch + gp.dz_off[l]; };
  Enq q{s, gp.num_sms};
  int gi = 0;
  // hidden layers: Z_l = A_{l-1} W_l^T, then bias and activation
  // objective only on a two-layer net with the tensor-core first layer: the output layer and the
  // per-sample losses come out of that kernel's epilogue
  const bool fused_out = !want_grad && status && l1_on_tensor_cores(gp, mlp, l1) && l1_fp32x3_fuses_output(mlp);
  for (int l = 1; l < L; ++l) {
    const int64_t fi = mlp.widths[l - 1];
    if (l == 1 && status && l1_on_tensor_cores(gp, mlp, l1)) {
      // the first layer on the tensor cores at FP32 accuracy
      ++gi;
      const int k = launch_l1_fp32x3(*l1, mlp, idx, R, act(1), status, s, fused_out ? loss : nullptr);
      if (k < 0) return -1;
      q.n += k;
      continue;
    }
    GemmArgs g = make_gemm(gl[gi++], R, P);
    if (l == 1) {
      g.A = mlp.X, g.sam = fi, g.sak = 1, g.sar = 0;
    } else {
      g.A = act(l - 1), g.sam = fi, g.sak = 1, g.sar = N * fi;
    }
    g.B = W + mlp.w_off[l - 1], g.sbk = 1, g.sbn = fi, g.sbr = ld;
    g.idx = idx;
    if (g.S == 1) {
      // one chunk: bias and activation in the product's epilogue
      g.epi = kEpiBiasAct, g.act = mlp.acts[l - 1];
      g.bias = W + mlp.b_off[l - 1], g.ldv = ld;
      g.out = act(l);
      q.gemm(g);
      continue;
    }
    q.gemm(g);
    RedArgs a{};
    a.P = P, a.S = g.S, a.R = R, a.M = g.M, a.Nc = g.Nc;
    a.mode = kRedBiasAct;
    a.act = mlp.acts[l - 1];
    a.bias = W + mlp.b_off[l - 1], a.ldv = ld;
    a.idx = idx;
    a.out = act(l);
    q.reduce(a);
  }
  // output layer, loss and (with a gradient) its derivatives, per sample tile
  if (!fused_out) {
    TailArgs t{};
    t.A = act(L - 1);
    t.W = W, t.idx = idx, t.ld = ld, t.w_off = mlp.w_off[L - 1], t.b_off = mlp.b_off[L - 1];
    t.y = mlp.y, t.N = N;
    t.h = mlp.widths[L - 1], t.C = mlp.widths[L], t.act = mlp.acts[L - 2], t.want_grad = want_grad;
    t.loss = loss;
    t.dz_prev = want_grad ? dz(L - 1) : nullptr;
    t.P = P;
    t.R = R;
    const size_t smem = tail_smem_bytes(t.h, t.C);
    if (smem > 48 * 1024 && ensure_smem_limit<k_out_layer>(smem) != cudaSuccess) return -1;
    const dim3 grid((unsigned)((N + kTailM - 1) / kTailM), (unsigned)R);
    if (launch_pdl(k_out_layer, grid, dim3(256), smem, s, t) != cudaSuccess) return -1;
    q.note();
  }
  if (f_out) {
    if (launch_pdl(k_loss_mean, dim3(R), dim3(256), 0, s, (const float*)loss, N, f_out, idx) != cudaSuccess)
      return -1;
    q.note();
  }
  if (!want_grad) return q.ok ? q.n : -1;
  {
    // [dW_L | db_L]: the tiles' shares summed in tile order
    RedArgs a{};
    a.P = P, a.S = (int32_t)((N + kTailM - 1) / kTailM), a.R = R, a.M = mlp.widths[L],
    a.Nc = mlp.widths[L - 1] + 1;
    a.mode = kRedGrad;
    a.grad = G, a.ldv = ld, a.w_off = mlp.w_off[L - 1], a.b_off = mlp.b_off[L - 1];
    q.reduce(a);
  }
  for (int l = L - 1; l >= 1; --l) {
    const int64_t fi = mlp.widths[l - 1], fo = mlp.widths[l];
    // [dW_l | db_l]^T = [A_{l-1} | 1]^T dZ_l: fi + 1 rows (the input units and
    // the bias) by fo columns, so the tiles are full for narrow layers
    GemmArgs g = make_gemm(gl[gi++], R, P);
    if (l == 1) {
      g.A = mlp.X, g.sam = 1, g.sak = fi, g.sar = 0;
    } else {
      g.A = act(l - 1), g.sam = 1, g.sak = fi, g.sar = N * fi;
    }
    g.a_ones = (int32_t)fi;
    g.B = dz(l), g.sbk = fo, g.sbn = 1, g.sbr = N * fo;
    q.gemm(g);
    RedArgs a{};
    a.P = P, a.S = g.S, a.R = R, a.M = g.M, a.Nc = g.Nc;
    a.mode = kRedGradT;
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
  return q.ok ? q.n : -1;
}

int launch_sgd(float* w, const float* g, int32_t R, int64_t D, int64_t Dp, float lr, float lb, float ub,
               cudaStream_t s) {
  return launch_pdl(k_sgd, dim3(grid_for((int64_t)R * D)), dim3(256), 0, s, w, g, R, D, Dp, lr, lb, ub) ==
                 cudaSuccess
             ? 1
             : -1;
}

namespace {
// Blocks per row copy: about 2 KB of the row per thread block, at most 64.
unsigned copy_blocks(int64_t Dp) {
  const int64_t b = (Dp / 4 + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 64 ? 64 : b));
}
}  // namespace

int launch_refine_pick(const float* fw_x, const float* fw_f, int32_t R, int32_t mu, int64_t Dp, float* w,
                       int32_t* elite, cudaStream_t s) {
  return launch_pdl(k_refine_pick, dim3(copy_blocks(Dp), (unsigned)R), dim3(256), 0, s, fw_x, fw_f, mu, Dp, w,
                    elite) == cudaSuccess
             ? 1
             : -1;
}

int launch_refine_accept(const float* w, const float* fr, const int32_t* elite, int32_t* flags, float* fw_x,
                         float* fw_f, float* best_x, float* best_f, int32_t R, int32_t mu, int64_t Dp,
                         cudaStream_t s) {
  if (launch_pdl(k_refine_decide, dim3((R + 127) / 128), dim3(128), 0, s, fr, elite, fw_f, best_f, mu, R, flags) !=
      cudaSuccess)
    return -1;
  return launch_pdl(k_refine_copy, dim3(copy_blocks(Dp), (unsigned)R), dim3(256), 0, s, w, elite,
                    (const int32_t*)flags, fw_x, best_x, mu, Dp) == cudaSuccess
             ? 2
             : -1;
}

}  // namespace mgfwa
