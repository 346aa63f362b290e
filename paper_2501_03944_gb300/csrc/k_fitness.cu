// Fitness kernels on CUDA cores: the FP32 path (GPU-MGFWA, Algorithm 1:
// "evaluate all the fitness of the sparks"), the fixed-order reduction of
// per-tile partial sums shared with the tensor-core path, the sphere, and
// the FP64 re-computation of the reported best loss.
//
// The objective is the mean cross-entropy of an MLP whose flattened
// parameters are the spark (nn.Linear order), on the shared batch X:
//   h_1 = act(W_1 x_n + b_1), ..., z = W_L h_{L-1} + b_L,
//   f = (1/N) sum_n [max_c z_c + log sum_c exp(z_c - max_c z_c) - z_{y_n}].
#include "mgfwa_internal.cuh"

namespace mgfwa {

namespace {

constexpr int kMT = 128;      // samples per tile (one per thread of the tail)
constexpr int kHC = 64;       // hidden units per first-layer chunk
constexpr int kKT = 16;       // K per shared-memory stage
constexpr int kThreads = 256;

__device__ __forceinline__ float act_f(int a, float v) { return a == kActTanh ? tanhf(v) : fmaxf(v, 0.0f); }

__host__ __device__ __forceinline__ int odd_ld(int w) { return w + ((w & 1) == 0 ? 1 : 0); }

// One block = one spark row x 128 samples.  Layer 1 is a register-tiled
// SIMT GEMM (each thread 8 samples x 4 hidden units); the activated hidden
// tile stays in shared memory, later layers run one sample per thread, and
// the block's cross-entropy sum goes to partial[mt][row].
__global__ void __launch_bounds__(kThreads) k_fitness_simt(Mlp mlp, const float* __restrict__ rows, int64_t ld,
                                                           int32_t count, const int32_t* __restrict__ idx,
                                                           float* __restrict__ partial) {
  griddep_wait();
  griddep_launch_dependents();
  extern __shared__ __align__(16) float smem[];
  const int row = blockIdx.x, mt = blockIdx.y;
  const float* w = rows + (int64_t)(idx != nullptr ? idx[row] : row) * ld;
  const int L = mlp.n_layers;
  const int d_in = mlp.widths[0], h1 = mlp.widths[1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int ldmax = 0;
  for (int l = 1; l <= L; ++l) ldmax = max(ldmax, odd_ld(mlp.widths[l]));
  float* Xs = smem;                 // [kKT][kMT]
  float* Ws = Xs + kKT * kMT;       // [kKT][kHC]
  float* bufA = Ws + kKT * kHC;     // [kMT][ldmax]
  float* bufB = bufA + kMT * ldmax; // [kMT][ldmax]
  const int64_t n0 = (int64_t)mt * kMT;
  const float* b1 = w + mlp.b_off[0];
  const int ldh = odd_ld(h1);

  for (int hc = 0; hc < h1; hc += kHC) {
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    for (int k0 = 0; k0 < d_in; k0 += kKT) {
      {
        const int nl = tid >> 1, kk = (tid & 1) * 8;
        const int64_t n = n0 + nl;
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
        if (n < mlp.N) {
          const float* xr = mlp.X + n * d_in + k0 + kk;
          if (k0 + kk < d_in) a0 = *reinterpret_cast<const float4*>(xr);
          if (k0 + kk + 4 < d_in) a1 = *reinterpret_cast<const float4*>(xr + 4);
        }
        Xs[(kk + 0) * kMT + nl] = a0.x; Xs[(kk + 1) * kMT + nl] = a0.y;
        Xs[(kk + 2) * kMT + nl] = a0.z; Xs[(kk + 3) * kMT + nl] = a0.w;
        Xs[(kk + 4) * kMT + nl] = a1.x; Xs[(kk + 5) * kMT + nl] = a1.y;
        Xs[(kk + 6) * kMT + nl] = a1.z; Xs[(kk + 7) * kMT + nl] = a1.w;
      }
      {
        const int j = tid >> 2, kq = (tid & 3) * 4;
        float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (hc + j < h1 && k0 + kq < d_in) b = *reinterpret_cast<const float4*>(w + (int64_t)(hc + j) * d_in + k0 + kq);
        Ws[(kq + 0) * kHC + j] = b.x; Ws[(kq + 1) * kHC + j] = b.y;
        Ws[(kq + 2) * kHC + j] = b.z; Ws[(kq + 3) * kHC + j] = b.w;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kKT; ++kk) {
        const float4 xa = *reinterpret_cast<const float4*>(Xs + kk * kMT + ty * 8);
        const float4 xb = *reinterpret_cast<const float4*>(Xs + kk * kMT + ty * 8 + 4);
        const float4 wv = *reinterpret_cast<const float4*>(Ws + kk * kHC + tx * 4);
        const float xr[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
        const float wr[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xr[a], wr[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int jj = hc + tx * 4 + b;
      if (jj < h1) {
        const float bias = b1[jj];
#pragma unroll
        for (int a = 0; a < 8; ++a) bufA[(ty * 8 + a) * ldh + jj] = act_f(mlp.acts[0], acc[a][b] + bias);
      }
    }
  }
  __syncthreads();

  float* in = bufA;
  int ldin = ldh;
  float* out = bufB;
  const int nl = tid & (kMT - 1), half = tid >> 7;
  for (int l = 1; l < L; ++l) {
    const int fi = mlp.widths[l], fo = mlp.widths[l + 1];
    const float* Wl = w + mlp.w_off[l];
    const float* bl = w + mlp.b_off[l];
    const int ldo = odd_ld(fo);
    const bool hidden = l + 1 < L;
    const float* a = in + nl * ldin;
    for (int j = half; j < fo; j += 2) {
      const float* wr = Wl + (int64_t)j * fi;
      float s = bl[j];
      for (int i = 0; i < fi; ++i) s = fmaf(wr[i], a[i], s);
      out[nl * ldo + j] = hidden ? act_f(mlp.acts[l], s) : s;
    }
    __syncthreads();
    float* t = in; in = out; out = t;
    ldin = ldo;
  }

  __shared__ float red[kThreads / 32];
  float ce = 0.0f;
  const int64_t n = n0 + tid;
  if (tid < kMT && n < mlp.N) {
    const float* z = in + tid * ldin;
    const int C = mlp.widths[L];
    float zmax = z[0];
    for (int c = 1; c < C; ++c) zmax = fmaxf(zmax, z[c]);
    float se = 0.0f;
    for (int c = 0; c < C; ++c) se += expf(z[c] - zmax);
    ce = (zmax + logf(se)) - z[mlp.y[n]];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ce += __shfl_xor_sync(0xffffffffu, ce, off);
  if ((tid & 31) == 0) red[tid >> 5] = ce;
  __syncthreads();
  if (tid == 0) {
    float s = red[0];
    for (int wi = 1; wi < kMT / 32; ++wi) s += red[wi];
    partial[(int64_t)mt * count + row] = s;
  }
}

// Small two-layer networks (d_in = DI, h1 = H1, C classes, all compile-time):
// one block = 128 samples (one per thread, its inputs in registers) x up to
// kSmallSparks sparks, whose rows are staged in shared memory and read as
// broadcasts.  Each hidden unit is accumulated over the inputs in ascending
// order from zero, then the bias is added and the activation applied, and
// each logit starts from its bias and accumulates the hidden units in
// ascending order: the same operations in the same order as k_fitness_simt,
// so both kernels give bitwise the same fitness.  The block's cross-entropy
// sum per spark goes to partial[mt][row] (warp sums added in warp order, as
// there).
constexpr int kSmallSparks = 8;

template <int DI, int H1, int C>
__global__ void __launch_bounds__(kMT) k_fitness_small(Mlp mlp, const float* __restrict__ rows, int64_t ld,
                                                       int32_t count, const int32_t* __restrict__ idx,
                                                       float* __restrict__ partial) {
  constexpr int D = DI * H1 + H1 + C * H1 + C;   // parameters per spark (nn.Linear order)
  constexpr int kB1 = DI * H1, kW2 = kB1 + H1, kB2 = kW2 + C * H1;
  __shared__ float ws[kSmallSparks][D];
  __shared__ float red[kSmallSparks][kMT / 32];
  griddep_wait();
  griddep_launch_dependents();
  const int s0 = blockIdx.x * kSmallSparks, mt = blockIdx.y;
  const int gs = min(kSmallSparks, count - s0);
  for (int e = threadIdx.x; e < gs * D; e += kMT) {
    const int g = e / D, k = e - g * D;
    const int r = s0 + g;
    ws[g][k] = rows[(int64_t)(idx != nullptr ? idx[r] : r) * ld + k];
  }
  const int64_t n = (int64_t)mt * kMT + threadIdx.x;
  const bool valid = n < mlp.N;
  float x[DI];
#pragma unroll
  for (int i = 0; i < DI; ++i) x[i] = valid ? mlp.X[n * DI + i] : 0.0f;
  const int label = valid ? mlp.y[n] : 0;
  const int act = mlp.acts[0];
  __syncthreads();
  for (int g = 0; g < gs; ++g) {
    const float* W = ws[g];
    float z[C];
#pragma unroll
    for (int c = 0; c < C; ++c) z[c] = W[kB2 + c];
#pragma unroll
    for (int j = 0; j < H1; ++j) {
      float a = 0.0f;
#pragma unroll
      for (int i = 0; i < DI; ++i) a = fmaf(x[i], W[j * DI + i], a);
      a = act_f(act, a + W[kB1 + j]);
#pragma unroll
      for (int c = 0; c < C; ++c) z[c] = fmaf(W[kW2 + c * H1 + j], a, z[c]);
    }
    float ce = 0.0f;
    if (valid) {
      float zmax = z[0];
#pragma unroll
      for (int c = 1; c < C; ++c) zmax = fmaxf(zmax, z[c]);
      float se = 0.0f;
#pragma unroll
      for (int c = 0; c < C; ++c) se += expf(z[c] - zmax);
      float zy = z[0];
#pragma unroll
      for (int c = 1; c < C; ++c) zy = label == c ? z[c] : zy;
      ce = (zmax + logf(se)) - zy;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ce += __shfl_xor_sync(0xffffffffu, ce, off);
    if ((threadIdx.x & 31) == 0) red[g][threadIdx.x >> 5] = ce;
  }
  __syncthreads();
  if ((int)threadIdx.x < gs) {
    float v = red[threadIdx.x][0];
#pragma unroll
    for (int wi = 1; wi < kMT / 32; ++wi) v += red[threadIdx.x][wi];
    partial[(int64_t)mt * count + s0 + threadIdx.x] = v;
  }
}

// True if the network is one that k_fitness_small is instantiated for, with
// the parameter layout it assumes.
bool small_net(const Mlp& mlp, int di, int h1, int c) {
  return mlp.n_layers == 2 && mlp.widths[0] == di && mlp.widths[1] == h1 && mlp.widths[2] == c &&
         mlp.w_off[0] == 0 && mlp.b_off[0] == (int64_t)di * h1 && mlp.w_off[1] == mlp.b_off[0] + h1 &&
         mlp.b_off[1] == mlp.w_off[1] + (int64_t)c * h1;
}

__global__ void k_fitness_finish(const float* __restrict__ partial, int32_t mtiles, int32_t count, float n_f,
                                 const int32_t* __restrict__ idx, float* __restrict__ fit) {
  griddep_wait();
  griddep_launch_dependents();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= count) return;
  fit[idx != nullptr ? idx[r] : r] = __fdiv_rn(tile_sum(partial, r, count, mtiles), n_f);
}

__global__ void __launch_bounds__(256) k_sphere(const float* __restrict__ rows, int64_t ld, int64_t D,
                                                float* __restrict__ fit) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ float red[8];
  const float* x = rows + (int64_t)blockIdx.x * ld;
  float s = 0.0f;
  for (int64_t d = threadIdx.x; d < D; d += blockDim.x) s = fmaf(x[d], x[d], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = red[0];
    for (int w = 1; w < 8; ++w) t += red[w];
    fit[blockIdx.x] = t;
  }
}

// FP64 forward of kF64Samples samples per block (so that every weight read
// feeds that many FMAs); one warp per output unit, lanes striding over the
// inputs in index order, then a fixed xor tree per sample.
constexpr int kF64Samples = 4;

__global__ void __launch_bounds__(256) k_fitness_f64(Mlp mlp, const float* __restrict__ x, int wmax,
                                                     double* __restrict__ ce64) {
  griddep_wait();
  griddep_launch_dependents();
  extern __shared__ double sd[];
  double* a = sd;                          // [kF64Samples][wmax]
  double* b = sd + (size_t)kF64Samples * wmax;
  const int64_t n0 = (int64_t)blockIdx.x * kF64Samples;
  const int ns = (int)(mlp.N - n0 < kF64Samples ? mlp.N - n0 : kF64Samples);
  const int d_in = mlp.widths[0];
  for (int e = threadIdx.x; e < kF64Samples * d_in; e += blockDim.x) {
    const int q = e / d_in, i = e - q * d_in;
    a[q * wmax + i] = q < ns ? (double)mlp.X[(n0 + q) * d_in + i] : 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int L = mlp.n_layers;
  for (int l = 0; l < L; ++l) {
    const int fi = mlp.widths[l], fo = mlp.widths[l + 1];
    const float* W = x + mlp.w_off[l];
    const float* bias = x + mlp.b_off[l];
    for (int j = warp; j < fo; j += nwarps) {
      double s[kF64Samples];
#pragma unroll
      for (int q = 0; q < kF64Samples; ++q) s[q] = 0.0;
      for (int i = lane; i < fi; i += 32) {
        const double wv = (double)W[(int64_t)j * fi + i];
#pragma unroll
        for (int q = 0; q < kF64Samples; ++q) s[q] += wv * a[q * wmax + i];
      }
#pragma unroll
      for (int q = 0; q < kF64Samples; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
      }
      if (lane < kF64Samples) {
        double v = s[0];
#pragma unroll
        for (int q = 1; q < kF64Samples; ++q) v = lane == q ? s[q] : v;
        v += (double)bias[j];
        if (l + 1 < L) v = mlp.acts[l] == kActTanh ? tanh(v) : (v > 0.0 ? v : 0.0);
        b[lane * wmax + j] = v;
      }
    }
    __syncthreads();
    double* t = a; a = b; b = t;
  }
  if (threadIdx.x < ns) {
    const int q = threadIdx.x;
    const double* z = a + q * wmax;
    const int C = mlp.widths[L];
    double zmax = z[0];
    for (int c = 1; c < C; ++c) zmax = z[c] > zmax ? z[c] : zmax;
    double se = 0.0;
    for (int c = 0; c < C; ++c) se += exp(z[c] - zmax);
    ce64[n0 + q] = (zmax + log(se)) - z[mlp.y[n0 + q]];
  }
}

// Fixed-order mean (or sum of squares) in FP64 by one block.
__global__ void __launch_bounds__(256) k_reduce_f64(const double* __restrict__ v, const float* __restrict__ xf,
                                                    int64_t n, double scale, double* __restrict__ out) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    if (xf != nullptr) {
      const double t = (double)xf[e];
      s += t * t;
    } else {
      s += v[e];
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

size_t smem_for(const Mlp& mlp) {
  int ldmax = 0;
  for (int l = 1; l <= mlp.n_layers; ++l) ldmax = ldmax > odd_ld(mlp.widths[l]) ? ldmax : odd_ld(mlp.widths[l]);
  return sizeof(float) * ((size_t)kKT * kMT + (size_t)kKT * kHC + 2 * (size_t)kMT * ldmax);
}

}  // namespace

size_t fitness_simt_smem_bytes(const Mlp& mlp) { return smem_for(mlp); }

int launch_fitness_finish(const float* partial, int32_t mtiles, int32_t count, int64_t N, float* fit,
                          cudaStream_t s, const int32_t* idx) {
  if (count <= 0) return 0;
  return launch_pdl(k_fitness_finish, dim3((count + 255) / 256), dim3(256), 0, s, partial, mtiles, count, (float)N,
                    idx, fit) == cudaSuccess
             ? 1
             : -1;
}

int launch_fitness_simt_main(const Mlp& mlp, const float* rows, int64_t ld, int32_t count, float* partial,
                             cudaStream_t s, const int32_t* idx) {
  if (count <= 0) return 0;
  const int mtiles = (int)((mlp.N + kMT - 1) / kMT);
  if (small_net(mlp, 8, 16, 3)) {
    dim3 grid((count + kSmallSparks - 1) / kSmallSparks, mtiles);
    return launch_pdl(k_fitness_small<8, 16, 3>, grid, dim3(kMT), 0, s, mlp, rows, ld, count, idx, partial) ==
                   cudaSuccess
               ? 1
               : -1;
  }
  const size_t smem = smem_for(mlp);
  if (ensure_smem_limit<k_fitness_simt>(smem) != cudaSuccess) return -1;
  dim3 grid(count, mtiles);
  return launch_pdl(k_fitness_simt, grid, dim3(kThreads), smem, s, mlp, rows, ld, count, idx, partial) == cudaSuccess
             ? 1
             : -1;
}

int launch_fitness_sphere(const float* rows, int64_t ld, int64_t D, int32_t count, float* fit, cudaStream_t s) {
  if (count <= 0) return 0;
  return launch_pdl(k_sphere, dim3(count), dim3(256), 0, s, rows, ld, D, fit) == cudaSuccess ? 1 : -1;
}

int launch_fitness_f64(const Mlp& mlp, const float* x, double* ce64, double* out, cudaStream_t s) {
  int wmax = 0;
  for (int l = 0; l <= mlp.n_layers; ++l) wmax = wmax > mlp.widths[l] ? wmax : mlp.widths[l];
  const size_t smem = 2 * sizeof(double) * (size_t)kF64Samples * wmax;
  if (smem > 48 * 1024 && ensure_smem_limit<k_fitness_f64>(smem) != cudaSuccess) return -1;
  k_fitness_f64<<<(unsigned)((mlp.N + kF64Samples - 1) / kF64Samples), 256, smem, s>>>(mlp, x, wmax, ce64);
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  k_reduce_f64<<<1, 256, 0, s>>>(ce64, nullptr, mlp.N, 1.0 / (double)mlp.N, out);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int launch_sphere_f64(const float* x, int64_t D, double* out, cudaStream_t s) {
  k_reduce_f64<<<1, 256, 0, s>>>(nullptr, x, D, 1.0, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mgfwa
