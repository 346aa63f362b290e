// The paper's own testbed objective (Sec. 4.1, Eq. 1): the scalar output of
// a fixed network whose input is the search vector,
//   a_0 = x;  a_l = act(W_l a_{l-1} + b_l) for hidden layers;  f = W_L a_{L-1} + b_L.
// Here the sparks are the rows of a batch and the weights are shared, so each
// layer is one dense product [rows x fan_in] x [fan_in x fan_out] with the
// bias and the activation in its epilogue (FP32 on the CUDA cores).  The
// summation order of every output is fixed by the layer's fan-in alone (four
// contiguous chunks of i, each a chain of fmaf in index order, the chunk sums
// added in chunk order, then the bias), so a spark's fitness does not depend
// on which sparks share the launch.  The last layer writes the fitness.  An
// FP64 forward of one vector gives the reported best fitness.
#include "mgfwa_internal.cuh"

namespace mgfwa {

namespace {

constexpr int kBK = 16;      // k-slab depth
constexpr int kStages = 3;   // slabs in flight per group (cp.async ring)
constexpr int kTN = 32;      // output tile columns per block
constexpr int kGroups = 4;   // fan-in chunks, one per 64-thread group
constexpr int kPadW = kTN + 4;

// Tile geometry for TR output rows per thread: 8 TR rows x 32 columns per block.
template <int TR>
struct NetTile {
  static constexpr int kTM = 8 * TR;
  static constexpr int kPadA = kTM + 4;
  static constexpr int kGroupFloats = kStages * kBK * (kPadA + kPadW);  // the ring of A and W slabs per group
  static constexpr size_t kSmem = sizeof(float) * kGroups * kGroupFloats;
  static_assert(kTM * kPadW <= kGroupFloats, "partial tiles must fit in the slab space");
};

__device__ __forceinline__ float act32(int a, float v) {
  if (a == kActTanh) return tanhf(v);
  if (a == kActGelu) return 0.5f * v * (1.0f + erff(v * 0.70710678118654752f));
  return fmaxf(v, 0.0f);
}

// 4-byte asynchronous global -> shared copy; src_bytes = 0 writes a zero
// without reading (the source address must still be a valid one).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, uint32_t src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The fan-in chunk of group g: [g c, min((g + 1) c, k)) with c = 16 ceil(k / 64).
__host__ __device__ __forceinline__ int chunk_len(int k) { return kBK * ((k + kBK * kGroups - 1) / (kBK * kGroups)); }

// out[r][j] = act(sum_i A[r][i] W[j][i] + b[j]) (no activation when act < 0)
// for r < rows, j < n; A row stride lda, out row stride ldo.  One 256-thread
// block per (8 TR) x 32 output tile.  Group g (threads 64 g ..) multiplies
// the tile over its fan-in chunk, TR x 4 outputs per thread:
// k-slabs of A and W are copied asynchronously (4-byte cp.async, transposed
// to k-major so a thread's rows and columns are contiguous) into the group's
// ring of kStages slabs, two slabs in flight while one is multiplied, one
// group barrier per slab.  The four partial tiles then meet in shared memory
// and every thread adds them in group order for TR of the tile's outputs,
// adds the bias and applies the activation.  A quarter of the fan-in per group cuts each
// block's serial slab chain to a quarter, which is what bounds the small-row
// launches (the guiding sparks).  TR = 8 takes three 16-byte shared loads per
// 32 FMAs (for launches that fill the SMs), TR = 4 two per 16 with twice the
// blocks.  Both compute every output with the same operations in the same
// order, so the choice never changes a result.
template <int TR>
__global__ void __launch_bounds__(256, TR == 4 ? 4 : 2) k_net_layer(const float* __restrict__ A, int64_t lda, int32_t rows,
                                                   const float* __restrict__ W, const float* __restrict__ bias,
                                                   int32_t k, int32_t n, int32_t act, float* __restrict__ out,
                                                   int64_t ldo) {
  constexpr int kTM = NetTile<TR>::kTM, kPadA = NetTile<TR>::kPadA, kGroupFloats = NetTile<TR>::kGroupFloats;
  griddep_wait();
  griddep_launch_dependents();
  // slabs [group][stage]{A [kBK][kPadA], W [kBK][kPadW]}; afterwards the partial tiles [group][kTM][kPadW]
  extern __shared__ __align__(16) float sm[];
  const int g = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int tx = t & 7, ty = t >> 3;
  const int r0 = blockIdx.x * kTM, j0 = blockIdx.y * kTN;  // row tiles on x: up to 2^24 rows
  const int c = chunk_len(k);
  const int kbeg = g * c, kend = min(kbeg + c, k);
  const int slabs = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;
  float* const base = sm + g * kGroupFloats;
  auto As = [&](int stage) { return base + stage * kBK * (kPadA + kPadW); };
  auto Ws = [&](int stage) { return base + stage * kBK * (kPadA + kPadW) + kBK * kPadA; };
  constexpr int LA = kTM * kBK / 64, LW = kTN * kBK / 64;  // slab elements each thread copies
  // element q of a thread is (row rq + 4 q, column kq) of the slab: 16
  // neighbouring threads read 16 consecutive floats of one row
  const int kq = t % kBK, rq = t / kBK;
  const float* pa = A + (int64_t)(r0 + rq) * lda + kq;  // dereferenced only where in range
  const float* pw = W + (int64_t)(j0 + rq) * k + kq;
  const int64_t sa = 4 * lda, sw = 4 * (int64_t)k;
  unsigned va = 0, vw = 0;
#pragma unroll
  for (int q = 0; q < LA; ++q) va |= (r0 + rq + 4 * q < rows ? 1u : 0u) << q;
#pragma unroll
  for (int q = 0; q < LW; ++q) vw |= (j0 + rq + 4 * q < n ? 1u : 0u) << q;
  auto fetch = [&](int slab, int stage) {
    const int k0 = kbeg + slab * kBK;
    const bool kin = k0 + kq < kend;
    float* a = As(stage) + kq * kPadA + rq;
    float* w = Ws(stage) + kq * kPadW + rq;
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const bool in = kin && (va >> q & 1u);
      cp_async4(a + 4 * q, in ? pa + q * sa + k0 : A, in ? 4u : 0u);
    }
#pragma unroll
    for (int q = 0; q < LW; ++q) {
      const bool in = kin && (vw >> q & 1u);
      cp_async4(w + 4 * q, in ? pw + q * sw + k0 : W, in ? 4u : 0u);
    }
  };
  auto group_sync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(g + 1) : "memory"); };
  float acc[TR][4];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll
  for (int i = 0; i < kStages - 1; ++i) {
    if (i < slabs) fetch(i, i);
    cp_async_commit();
  }
  for (int s = 0; s < slabs; ++s) {
    const int cur = s % kStages;
    cp_async_wait<kStages - 2>();  // this thread's copies of slab s have landed
    group_sync();                  // everyone's have; everyone is done with slab s - 1
    const float* a = As(cur);
    const float* w = Ws(cur);
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float ai[TR];
#pragma unroll
      for (int h = 0; h < TR / 4; ++h) {
        const float4 av = *reinterpret_cast<const float4*>(a + kk * kPadA + ty * TR + 4 * h);
        ai[4 * h] = av.x; ai[4 * h + 1] = av.y; ai[4 * h + 2] = av.z; ai[4 * h + 3] = av.w;
      }
      const float4 wv = *reinterpret_cast<const float4*>(w + kk * kPadW + tx * 4);
      const float wj[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ai[i], wj[j], acc[i][j]);
    }
    // the ring slot of slab s + kStages - 1 last held slab s - 1, which every
    // thread of the group finished before the barrier above
    if (s + kStages - 1 < slabs) fetch(s + kStages - 1, (s + kStages - 1) % kStages);
    cp_async_commit();
  }
  cp_async_wait<0>();
  __syncthreads();  // every group done with its slabs: the space holds the partial tiles now
  float* part = sm + g * (kTM * kPadW);
#pragma unroll
  for (int i = 0; i < TR; ++i)
    *reinterpret_cast<float4*>(part + (ty * TR + i) * kPadW + tx * 4) =
        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kTM * kTN / 256; ++q) {
    const int o = threadIdx.x + 256 * q, rr = o / kTN, cc = o % kTN;
    const int r = r0 + rr, j = j0 + cc;
    if (r >= rows || j >= n) continue;
    float z = sm[rr * kPadW + cc];
#pragma unroll
    for (int h = 1; h < kGroups; ++h) z += sm[h * (kTM * kPadW) + rr * kPadW + cc];
    z += bias[j];
    out[(int64_t)r * ldo + j] = act >= 0 ? act32(act, z) : z;
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

int launch_net_layer(const float* a, int64_t lda, int32_t count, const float* W, const float* b, int32_t fi,
                     int32_t fo, int32_t ak, float* o, int64_t ldo, cudaStream_t s) {
  if (ensure_smem_limit<k_net_layer<8>>(NetTile<8>::kSmem) != cudaSuccess ||
      ensure_smem_limit<k_net_layer<4>>(NetTile<4>::kSmem) != cudaSuccess)
    return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return -1;
  // 64-row tiles where they fill the SMs, else 32-row tiles (twice the blocks)
  const bool wide = (int64_t)((count + 63) / 64) * ((fo + kTN - 1) / kTN) >= sms;
  cudaError_t e;
  if (wide)
    e = launch_pdl(k_net_layer<8>, dim3((unsigned)((count + 63) / 64), (unsigned)((fo + kTN - 1) / kTN)), dim3(256),
                   NetTile<8>::kSmem, s, a, lda, count, W, b, fi, fo, ak, o, ldo);
  else
    e = launch_pdl(k_net_layer<4>, dim3((unsigned)((count + 31) / 32), (unsigned)((fo + kTN - 1) / kTN)), dim3(256),
                   NetTile<4>::kSmem, s, a, lda, count, W, b, fi, fo, ak, o, ldo);
  return e == cudaSuccess ? 1 : -1;
}

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
    if (launch_net_layer(a, lda, count, net.params + net.w_off[l], net.params + net.b_off[l], fi, fo,
                         last ? -1 : net.acts[l], o, ldo, s) < 0)
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
