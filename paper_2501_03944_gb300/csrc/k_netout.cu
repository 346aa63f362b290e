// The paper's own testbed objective (Sec. 4.1, Eq. 1): the scalar output of
// a fixed network whose input is the search vector,
//   a_0 = x;  a_l = act(W_l a_{l-1} + b_l) for hidden layers;  f = W_L a_{L-1} + b_L.
// Here the sparks are the rows of a batch and the weights are shared, so each
// layer is one dense product [rows x fan_in] x [fan_in x fan_out] with the
// bias and the activation in its epilogue (FP32 on the CUDA cores; every
// output accumulates its products in index order, so a spark's fitness does
// not depend on which sparks share the launch).  The last layer writes the
// fitness.  An FP64 forward of one vector gives the reported best fitness.
#include "mgfwa_internal.cuh"

namespace mgfwa {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

__device__ __forceinline__ float act32(int a, float v) {
  if (a == kActTanh) return tanhf(v);
  if (a == kActGelu) return 0.5f * v * (1.0f + erff(v * 0.70710678118654752f));
  return fmaxf(v, 0.0f);
}

// out[r][j] = act(sum_i A[r][i] W[j][i] + b[j]) (no activation when act < 0)
// for r < rows, j < n; A row stride lda, out row stride ldo.  256 threads,
// 4 x 4 outputs each.
__global__ void __launch_bounds__(256) k_net_layer(const float* __restrict__ A, int64_t lda, int32_t rows,
                                                   const float* __restrict__ W, const float* __restrict__ bias,
                                                   int32_t k, int32_t n, int32_t act, float* __restrict__ out,
                                                   int64_t ldo) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Ws[kBK][kBN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * kBM, j0 = blockIdx.x * kBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < k; k0 += kBK) {
    for (int e = threadIdx.x; e < kBM * kBK; e += 256) {
      const int rr = e / kBK, kk = e - rr * kBK;
      const int r = r0 + rr, kc = k0 + kk;
      As[kk][rr] = (r < rows && kc < k) ? A[(int64_t)r * lda + kc] : 0.0f;
      const int j = j0 + rr;
      Ws[kk][rr] = (j < n && kc < k) ? W[(int64_t)j * k + kc] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        w[i] = Ws[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty * 4 + i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = j0 + tx * 4 + j;
      if (c >= n) continue;
      const float z = acc[i][j] + bias[c];
      out[(int64_t)r * ldo + c] = act >= 0 ? act32(act, z) : z;
    }
  }
}

// FP64 forward of one vector (one block): each layer's outputs in parallel,
// each a dot product in index order, activations in shared memory.
__global__ void __launch_bounds__(256) k_net_f64(NetOut net, const float* __restrict__ x, double* __restrict__ out) {
  griddep_wait();
  griddep_launch_dependents();
  extern __shared__ double sh[];
  double* a = sh;
  double* b = sh + net.wmax;
  for (int i = threadIdx.x; i < net.widths[0]; i += blockDim.x) a[i] = (double)x[i];
  __syncthreads();
  for (int l = 0; l < net.n_layers; ++l) {
    const int fi = net.widths[l], fo = net.widths[l + 1];
    const float* W = net.params + net.w_off[l];
    const float* bias = net.params + net.b_off[l];
    for (int j = threadIdx.x; j < fo; j += blockDim.x) {
      double s = (double)bias[j];
      for (int i = 0; i < fi; ++i) s += (double)W[(int64_t)j * fi + i] * a[i];
      if (l + 1 < net.n_layers) {
        const int ak = net.acts[l];
        s = ak == kActTanh ? tanh(s) : (ak == kActGelu ? 0.5 * s * (1.0 + erf(s * 0.70710678118654752440)) : fmax(s, 0.0));
      }
      b[j] = s;
    }
    __syncthreads();
    double* t = a;
    a = b;
    b = t;
  }
  if (threadIdx.x == 0) *out = a[0];
}

}  // namespace

int launch_net_output(const NetOut& net, const float* rows, int64_t ld, int32_t count, float* fit, float* scratch,
                      int64_t scratch_ld, cudaStream_t s) {
  if (count <= 0) return 0;
  const float* a = rows;
  int64_t lda = ld;
  int n = 0;
  for (int l = 0; l < net.n_layers; ++l) {
    const int fi = net.widths[l], fo = net.widths[l + 1];
    const bool last = l + 1 == net.n_layers;
    float* o = last ? fit : scratch + (int64_t)(l & 1) * scratch_ld * count;
    const int64_t ldo = last ? 1 : scratch_ld;
    const dim3 grid((unsigned)((fo + kBN - 1) / kBN), (unsigned)((count + kBM - 1) / kBM));
    if (launch_pdl(k_net_layer, grid, dim3(256), 0, s, a, lda, count, (const float*)(net.params + net.w_off[l]),
                   (const float*)(net.params + net.b_off[l]), (int32_t)fi, (int32_t)fo,
                   (int32_t)(last ? -1 : net.acts[l]), o, ldo) != cudaSuccess)
      return -1;
    ++n;
    a = o;
    lda = ldo;
  }
  return n;
}

int launch_net_output_f64(const NetOut& net, const float* x, double* out, cudaStream_t s) {
  const size_t smem = sizeof(double) * 2 * (size_t)net.wmax;
  if (smem > 48 * 1024 && ensure_smem_limit<k_net_f64>(smem) != cudaSuccess) return -1;
  return launch_pdl(k_net_f64, dim3(1), dim3(256), smem, s, net, x, out) == cudaSuccess ? 1 : -1;
}

}  // namespace mgfwa
