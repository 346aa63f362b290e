// Internal declarations shared by the library's translation units: the
// device-side problem description, the Philox4x32-10 generator and the
// kernel launchers.  Nothing here is part of the C ABI (include/mgfwa.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace mgfwa {

// Philox stream purposes: the fourth counter word.
constexpr uint32_t kInit = 0, kExplode = 1, kMap = 2, kGmap = 3, kLoser = 4;

// Scalar parameters of one run, passed by value to the kernels.
// Fireworks of all runs are numbered globally, z = b * mu + i (run b,
// firework i); explosion rows are z * lam + j, guiding rows z * m + q.
struct Problem {
  int64_t D;       // search dimension
  int64_t Dp;      // padded row stride (floats), a multiple of 64
  float lb, ub;
  int32_t mu, lam, m, g, k;
  int32_t B;       // independent runs
  float beta, amp0, c_a, c_r;
  uint64_t seed;   // run b draws from Philox keyed by seed + b
  int32_t lo_gmax; // loser-out tournament: the generations the budget allows (0 = tournament off)
  int32_t fw_off;  // index in the run of this handle's first firework (a shard of the run), 0 otherwise;
                   // Philox units number fireworks by their index in the run
};

// Philox key of run b: low and high words of seed + b.
__host__ __device__ __forceinline__ void run_key(const Problem& p, int b, uint32_t& k0, uint32_t& k1) {
  const uint64_t s = p.seed + (uint64_t)b;
  k0 = (uint32_t)(s & 0xffffffffu);
  k1 = (uint32_t)(s >> 32);
}

// The MLP objective as the kernels see it.
struct Mlp {
  int32_t n_layers;    // linear layers (2 or 3)
  int32_t widths[4];   // d_in, h1, [h2,] C
  int32_t acts[3];     // hidden activations
  int64_t N;
  const float* X;             // [N][d_in] FP32
  const void* Xop;            // [N][d_in] tensor-core copy of X (BF16 or FP8) or null
  const int32_t* y;           // [N]
  int64_t w_off[3], b_off[3]; // offsets of W_l and b_l in the search vector
  int64_t w1_elems;           // h1 * d_in
};

enum { kActTanh = 0, kActRelu = 1, kActGelu = 2 };

// The testbed network of Sec. 4.1 (Eq. 1) as the kernels see it: fixed
// parameters (nn.Linear order) in device memory, the search vector is its input.
constexpr int kNetMaxLayers = 16;
struct NetOut {
  int32_t n_layers;                        // linear layers, 1 to kNetMaxLayers
  int32_t widths[kNetMaxLayers + 1];       // d, hidden widths, 1
  int32_t acts[kNetMaxLayers];             // hidden activations
  int64_t w_off[kNetMaxLayers], b_off[kNetMaxLayers];  // offsets of W_l and b_l in params
  int32_t wmax;                            // largest width
  int32_t hmax;                            // largest hidden width (1 without hidden layers)
  const float* params;                     // device copy
};

// The first-layer GEMM operand the samplers write beside the FP32 rows:
// row r holds the spark's first w1_elems coordinates ([h1][d_in] row-major)
// as BF16, or as E4M3 of (coordinate * inv_scale) with saturation.
// With w2 set (the CTA-pair kernel's networks) the samplers also store each
// spark's second-layer weights W2 [classes][h1] as BF16, row r at
// w2 + r * w2_rows * h1 ([w2_rows][h1], rows classes..w2_rows-1 kept zero;
// classes = C for two layers, h2 for three), and with w3 set (three layers)
// W3 [C][h2] the same way at w3 + r * w3_rows * h2.
enum { kOpNone = 0, kOpBf16 = 1, kOpFp8 = 2 };
struct OpDesc {
  void* base = nullptr;  // row 0
  int32_t kind = kOpNone;
  float inv_scale = 1.0f;
  int64_t w1_elems = 0;
  void* w2 = nullptr;     // BF16 W2 of row 0, or null
  int64_t w2_off = 0;     // coordinate of W2[0][0] in a spark row
  int32_t w2_h1 = 0;      // h1 (elements per W2 row)
  int32_t w2_classes = 0; // W2 rows the samplers write (C, or h2 with three layers)
  int32_t w2_rows = 0;    // W2 rows per spark in the buffer
  void* w3 = nullptr;     // BF16 W3 of row 0, or null
  int64_t w3_off = 0;     // coordinate of W3[0][0] in a spark row
  int32_t w3_k = 0;       // h2 (elements per W3 row)
  int32_t w3_classes = 0; // C
  int32_t w3_rows = 0;    // W3 rows per spark in the buffer (16)
  __host__ __device__ int64_t row_bytes() const { return w1_elems * (kind == kOpFp8 ? 1 : 2); }
  __host__ __device__ int64_t w2_row_elems() const { return (int64_t)w2_rows * w2_h1; }
  __host__ __device__ int64_t w3_row_elems() const { return (int64_t)w3_rows * w3_k; }
  // the descriptor of rows [first, ...)
  OpDesc from(int64_t first) const {
    OpDesc d = *this;
    if (base) d.base = static_cast<uint8_t*>(base) + first * row_bytes();
    if (w2) d.w2 = static_cast<uint16_t*>(w2) + first * w2_row_elems();
    if (w3) d.w3 = static_cast<uint16_t*>(w3) + first * w3_row_elems();
    return d;
  }
};

// Programmatic dependent launch.  A kernel started by launch_pdl may be
// scheduled while its predecessor on the stream is still running, so every
// kernel of the library calls griddep_wait(), which returns once the
// predecessor grid has completed and its memory writes are visible (at once
// when the launch was an ordinary one), before it touches any memory
// another kernel writes -- most at their first line, the tensor-core
// kernels after setting up their barriers and TMEM -- and then calls
// griddep_launch_dependents(), which lets the next such launch be scheduled
// as soon as every CTA of this grid has started.  What overlaps is the next
// kernel's launch, CTA dispatch and that set-up with this kernel's last
// wave, never a memory access that depends on it.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Raise kernel K's dynamic shared-memory limit on the current device once.
// The attribute belongs to one kernel on one device, so the cache is per
// kernel (one template instance per kernel, not per kernel type) and per
// device.  Host threads may launch concurrently, so the cached limit is
// updated under a lock.
template <auto K>
inline cudaError_t ensure_smem_limit(size_t bytes) {
  constexpr int kMaxDevices = 64;
  static size_t configured[kMaxDevices] = {};
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < kMaxDevices && bytes <= configured[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) configured[dev] = bytes;
  return e;
}

// Largest batch the FP32 fitness kernels accept: their grid carries the
// 128-sample tiles in its y dimension, which is limited to 65535 blocks.
constexpr int64_t kMaxSamples = 65535LL * 128;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// on words 0 and 2, xor/permute with words 1, 3 and the round key, key bumped
// by the Weyl constants between rounds.

__device__ __forceinline__ uint64_t mul_wide_u32(uint32_t a, uint32_t b) {
  uint64_t r;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(a), "r"(b));
  return r;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = mul_wide_u32(0xD2511F53u, c.x);
    const uint64_t p1 = mul_wide_u32(0xCD9E8D57u, c.z);
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The ten round keys of one Philox key, for a thread that draws several
// blocks under the same key (the same values the loop above steps through).
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};
__device__ __forceinline__ PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys rk;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
    rk.k1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  return rk;
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = mul_wide_u32(0xD2511F53u, c.x);
    const uint64_t p1 = mul_wide_u32(0xCD9E8D57u, c.z);
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk.k1[r],
                   (uint32_t)p0);
  }
  return c;
}

// Uniform on the 2^-24 grid of [0, 1).
__device__ __forceinline__ float u24(uint32_t r) { return __uint2float_rn(r >> 8) * 0x1p-24f; }

__device__ __forceinline__ float lane_of(const float4& v, int l) {
  return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w;
}
__device__ __forceinline__ uint32_t lane_of(const uint4& v, int l) {
  return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w;
}

// NaN fitness ranks as +infinity; order is (fitness, index) ascending.
__device__ __forceinline__ float rank_key(float f) { return isnan(f) ? __int_as_float(0x7f800000) : f; }
__device__ __forceinline__ bool before(float fa, int ia, float fb, int ib) {
  const float a = rank_key(fa), b = rank_key(fb);
  return a < b || (a == b && ia < ib);
}

// The fitness sum of spark r from the per-sample-tile loss sums partial[mt *
// count + r]: the tiles added in tile order (the fitness-finish arithmetic
// every kernel that finishes a mean shares), loads issued eight at a time so
// that a tile's latency is paid once per eight tiles.
__device__ __forceinline__ float tile_sum(const float* __restrict__ partial, int64_t r, int32_t count,
                                          int32_t mtiles) {
  float s = partial[r];
  int mt = 1;
  for (; mt + 8 <= mtiles; mt += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = partial[(int64_t)(mt + u) * count + r];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; mt < mtiles; ++mt) s += partial[(int64_t)mt * count + r];
  return s;
}

// Sets the calling thread's error text (what mgfwa_last_error(NULL) returns).
void set_thread_error(const char* msg);

// ---------------------------------------------------------------------------
// Launchers (each returns the number of kernels it enqueued, or -1 after a
// launch error; the caller reads cudaGetLastError()).

int launch_init(const Problem& p, float* fw_x, float* fw_amp, cudaStream_t s);

// Explosion sparks rows [0, mu*lam) of `sparks` (row stride Dp); if `op` is
// non-null also the BF16 first-layer operand (w1_elems per spark row).
// The generation number is read on the device: gens_done[0] + 1, where
// gens_done counts completed generations (launch_select advances it), so a
// captured generation replays with the right Philox counters.
int launch_explode(const Problem& p, const uint32_t* gens_done, const float* fw_x, const float* fw_amp,
                   float* sparks, const OpDesc& op, cudaStream_t s);

// With `partial` ([mtiles][stride] per-sample-tile loss sums, the explosion
// rows first, N samples; stride 0 means B*mu*lam), the rank kernel also
// finishes the explosion fitness into fit_e, exactly as
// launch_fitness_finish would.
int launch_rank(const Problem& p, float* fit_e, int32_t* top, int32_t* bottom, cudaStream_t s,
                const float* partial = nullptr, int32_t mtiles = 0, int64_t N = 0, int64_t stride = 0);

// Guiding sparks written to `guides` (mu*m rows of stride Dp) and, if non-
// null, their operand rows `op_guides`.
int launch_guide(const Problem& p, const uint32_t* gens_done, const float* fw_x, const float* fw_amp,
                 const float* sparks, const int32_t* top, const int32_t* bottom, float* guides,
                 const OpDesc& op_guides, cudaStream_t s, const float* gv_in = nullptr, float* gv_out = nullptr);

// Per run: best-so-far over its fireworks (init: the first minimum).
int launch_run_best_init(const Problem& p, const float* fw_x, const float* fw_f, float* best_x, float* best_f,
                         cudaStream_t s);

// Selection of every firework (winner[z]: its winning candidate or -1) and
// each run's best-so-far (winner[B*mu + b]: the run's improving firework or
// -1; winner[B*mu + B]: the generation; winner holds B*mu + B + 1
// entries), the loser-out tournament when p.lo_gmax > 0 (f_old [B*mu]:
// scratch for the fitness before the selection; loser [B*mu]: 1 where a
// firework lost), then the copies of the winning rows into fw_x and best_x
// and the losers' new rows; advances gens_done[0] by one (the generation is
// complete).
int launch_select(const Problem& p, const float* fit_e, const float* fit_g, const float* sparks,
                  const float* guides, float* fw_x, float* fw_amp, float* fw_f, int32_t* winner,
                  float* best_x, float* best_f, uint32_t* gens_done, float* f_old, int32_t* loser, cudaStream_t s);

// FP32 CUDA-core fitness of `count` rows (stride `ld` floats; row r is
// rows[idx[r]] when idx is given): per-(m-tile, r) partial cross-entropy
// sums into `partial` [mtiles][count] (the mean is taken by
// launch_fitness_finish).
int launch_fitness_simt_main(const Mlp& mlp, const float* rows, int64_t ld, int32_t count, float* partial,
                             cudaStream_t s, const int32_t* idx = nullptr);
size_t fitness_simt_smem_bytes(const Mlp& mlp);

// fit[r] (fit[idx[r]] when idx is given) = mean over m-tiles of partial:
// fixed-order FP32 sum / N.
int launch_fitness_finish(const float* partial, int32_t mtiles, int32_t count, int64_t N, float* fit,
                          cudaStream_t s, const int32_t* idx = nullptr);

// Elite candidates for the FP32 re-score: per firework (all runs) the
// `E` best of its lam explosion and m guiding sparks by the current
// fitness, as rows of the spark buffer (explosion z*lam + c, guiding
// n_e + z*m + q) into elite[z*E + e].
// With `partial` ([mtiles][stride] per-sample-tile loss sums whose columns
// start at the guiding rows, N samples; stride 0 means B*mu*m), the pick
// also finishes the guiding fitness into fit_g first, exactly as
// launch_fitness_finish would.
int launch_elite_pick(const Problem& p, const float* fit_e, float* fit_g, int32_t E, int32_t* elite,
                      cudaStream_t s, const float* partial = nullptr, int32_t mtiles = 0, int64_t N = 0,
                      int64_t stride = 0);

int launch_fitness_sphere(const float* rows, int64_t ld, int64_t D, int32_t count, float* fit, cudaStream_t s);

// FP64 objective of one FP32 vector: per-sample CE into ce64[N], then the
// fixed-order mean into *out.
int launch_fitness_f64(const Mlp& mlp, const float* x, double* ce64, double* out, cudaStream_t s);
int launch_sphere_f64(const float* x, int64_t D, double* out, cudaStream_t s);
// The testbed network's output for `count` rows (row stride ld) into fit, one
// launch per layer; scratch holds 2 * count * scratch_ld floats of hidden
// activations.  Returns the launch count or -1.
int launch_net_output(const NetOut& net, const float* rows, int64_t ld, int32_t count, float* fit, float* scratch,
                      int64_t scratch_ld, cudaStream_t s);
// Its FP64 output for one vector into *out (one launch).
int launch_net_output_f64(const NetOut& net, const float* x, double* out, cudaStream_t s);
// One CUDA-core layer of the testbed network: out[r][j] = act(A[r] . W[j] + b[j]) (no activation for act < 0).
int launch_net_layer(const float* A, int64_t lda, int32_t rows, const float* W, const float* b, int32_t k, int32_t n,
                     int32_t act, float* out, int64_t ldo, cudaStream_t s);

// BF16 copy of the first-layer weights of `count` rows (stride ld) into op.
int launch_to_operand(const float* rows, int64_t ld, int32_t count, const OpDesc& op, cudaStream_t s);
// dst[e] = BF16(src[e]) or E4M3(src[e] * inv_scale), e < n.
int launch_f32_to_op(const float* src, int64_t n, int32_t kind, float inv_scale, void* dst, cudaStream_t s);

}  // namespace mgfwa
