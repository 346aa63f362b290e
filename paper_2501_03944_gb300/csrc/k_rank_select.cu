// Ranking and selection kernels (GPU-MGFWA, Algorithm 1: the ranking that
// feeds the multi-guiding sparks, and "select the best individual of each
// population").
//
// Both are decided on FP32 fitness in the total order (fitness, index)
// with NaN ranked as +infinity, so that the outcome is unique and does not
// depend on thread scheduling.
#include "mgfwa_internal.cuh"

namespace mgfwa {

namespace {

// One block per (firework, guiding group), fireworks of all runs numbered
// globally.  Each thread ranks its sparks by
// counting the sparks of the group that come strictly before them; the
// counts are a permutation because the order is total.  With `partial`
// (per-sample-tile loss sums [mtiles][count] of the explosion rows), the
// block first finishes its sparks' fitness as the fitness-finish kernel
// does (tile sums in tile order, then / N) and stores it in fit_e.
__global__ void k_rank(Problem p, float* __restrict__ fit_e, int32_t* __restrict__ top,
                       int32_t* __restrict__ bottom, const float* __restrict__ partial, int32_t mtiles,
                       int32_t count, float n_f) {
  griddep_wait();
  griddep_launch_dependents();
  extern __shared__ float sh[];
  const int g = p.g, k = p.k;
  float* f = sh;
  int* order = reinterpret_cast<int*>(sh + g);
  const int grp = blockIdx.x;  // i * m + q
  const int i = grp / p.m, q = grp % p.m;
  const int base = q * g;
  float* fe = fit_e + (int64_t)i * p.lam + base;
  for (int a = threadIdx.x; a < g; a += blockDim.x) {
    if (partial) {
      const int64_t r = (int64_t)i * p.lam + base + a;
      const float v = __fdiv_rn(tile_sum(partial, r, count, mtiles), n_f);
      fe[a] = v;
      f[a] = v;
    } else {
      f[a] = fe[a];
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < g; a += blockDim.x) {
    const float fa = f[a];
    int r = 0;
    for (int b = 0; b < g; ++b) r += before(f[b], b, fa, a) ? 1 : 0;
    order[r] = a;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    top[(int64_t)grp * k + r] = base + order[r];
    bottom[(int64_t)grp * k + r] = base + order[g - 1 - r];
  }
}

constexpr int kSelThreads = 256;
constexpr int kSelStage = 1024;  // fireworks per run whose fitness the selection's serial part reads from shared memory
constexpr int kSelChunk = 8;     // candidates per lane loaded before they are compared
constexpr int kPickStage = 2048; // candidates per firework the elite pick stages in shared memory

__device__ __forceinline__ void take_if_before(float& bf, int& bc, float of, int oc) {
  if (oc >= 0 && (bc < 0 || before(of, oc, bf, bc))) {
    bf = of;
    bc = oc;
  }
}

// Selection decisions, one block per run and one warp per firework of the
// run (fireworks in turn when mu exceeds the warps): argmin over the
// firework's lam explosion and m guiding sparks (candidate order: explosion
// 0..lam-1, guiding 0..m-1), the strict improvement test and the dynamic
// amplitude update (x C_a on improvement, x C_r otherwise); winner[z] is
// the winning candidate or -1.  Then the run's best-so-far: strict
// improvement over its new fireworks in index order; winner[B*mu + b] is
// that firework or -1, winner[B*mu + B] this generation's number.  Then,
// with p.lo_gmax > 0, the loser-out tournament: every firework but the
// run's first minimum whose fitness before (f_old) and after the selection
// are finite, and whose last improvement I extrapolated over the g_rem =
// lo_gmax - gen generations left, fmaf(-I, g_rem, f), stays above the run's
// best-so-far, loses: fitness +infinity, amplitude A0, loser[z] = 1 (its
// row is re-drawn by k_select_copy).  gens_done is only read here.
__global__ void __launch_bounds__(kSelThreads) k_select_decide(Problem p, const float* __restrict__ fit_e,
                                                               const float* __restrict__ fit_g,
                                                               float* __restrict__ fw_amp, float* __restrict__ fw_f,
                                                               int32_t* __restrict__ winner,
                                                               float* __restrict__ best_f,
                                                               const uint32_t* __restrict__ gens_done,
                                                               float* __restrict__ f_old, int32_t* __restrict__ loser) {
  griddep_wait();
  griddep_launch_dependents();
  const int b = blockIdx.x;
  const uint32_t gen = *gens_done + 1u;  // this generation
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n_cand = p.lam + p.m;
  // the run's fireworks' fitness before and after this selection, for the serial part below
  __shared__ float sh_f[kSelStage], sh_old[kSelStage];
  const bool staged = p.mu <= kSelStage;
  for (int il = warp; il < p.mu; il += kSelThreads / 32) {
    const int i = b * p.mu + il;  // global firework
    float bf = 0.0f;
    int bc = -1;
    // the candidates in chunks of kSelChunk per lane, every load of a chunk issued before its compares
    for (int c = lane; c < n_cand; c += 32 * kSelChunk) {
      float v[kSelChunk];
#pragma unroll
      for (int u = 0; u < kSelChunk; ++u) {
        const int cu = c + 32 * u;
        v[u] = cu >= n_cand ? 0.0f
               : cu < p.lam ? fit_e[(int64_t)i * p.lam + cu]
                            : fit_g[(int64_t)i * p.m + (cu - p.lam)];
      }
#pragma unroll
      for (int u = 0; u < kSelChunk; ++u)
        if (c + 32 * u < n_cand) take_if_before(bf, bc, v[u], c + 32 * u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float of = __shfl_xor_sync(0xffffffffu, bf, off);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
      take_if_before(bf, bc, of, oc);
    }
    if (lane == 0) {
      const float amp = fw_amp[i];
      const float fo = fw_f[i];
      f_old[i] = fo;
      float fn = fo;
      if (rank_key(bf) < rank_key(fo)) {
        fn = bf;
        fw_f[i] = bf;
        fw_amp[i] = __fmul_rn(amp, p.c_a);
        winner[i] = bc;
      } else {
        fw_amp[i] = __fmul_rn(amp, p.c_r);
        winner[i] = -1;
      }
      if (staged) {
        sh_f[il] = fn;
        sh_old[il] = fo;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float* f = staged ? sh_f : fw_f + (int64_t)b * p.mu;
    const float* fold = staged ? sh_old : f_old + (int64_t)b * p.mu;
    int bi = -1;
    float bfv = best_f[b];
    for (int i = 0; i < p.mu; ++i) {
      if (rank_key(f[i]) < rank_key(bfv)) {
        bfv = f[i];
        bi = i;
      }
    }
    if (bi >= 0) best_f[b] = bfv;
    winner[(int64_t)p.B * p.mu + b] = bi;
    if (b == 0) winner[(int64_t)p.B * p.mu + p.B] = (int32_t)gen;
    int e = 0;  // the run's best firework: never a loser
    for (int i = 1; i < p.mu; ++i)
      if (rank_key(f[i]) < rank_key(f[e])) e = i;
    const int64_t left = (int64_t)p.lo_gmax - (int64_t)gen;
    const float g_rem = (float)(left > 0 ? left : 0);
    const float rb = best_f[b];
    for (int il = 0; il < p.mu; ++il) {
      const int64_t z = (int64_t)b * p.mu + il;
      int32_t lo = 0;
      const float fo = fold[il], fn = f[il];
      if (p.lo_gmax > 0 && il != e && isfinite(fo) && isfinite(fn)) {
        const float proj = __fmaf_rn(-__fsub_rn(fo, fn), g_rem, fn);
        if (proj > rb) {
          lo = 1;
          fw_f[z] = __int_as_float(0x7f800000);
          fw_amp[z] = p.amp0;
        }
      }
      loser[z] = lo;
    }
  }
}

// Blocks per row copy: about 1 KB of the row per thread block, at most 64.
__host__ __device__ inline int copy_blocks(int64_t Dp) {
  const int64_t b = (Dp / 4 + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 64 ? 64 : b));
}

// The rows of the selection, grid (row chunks, B*mu + B): row y < B*mu is
// firework y's winning candidate copied into fw_x (when one won), or, for a
// loser of the tournament, a uniform draw in [lb, ub] (purpose kLoser,
// generation winner[B*mu + B], unit = the firework's index in its run);
// row B*mu + b is run b's best firework copied into best_x, read from where
// that firework's new position comes from (its winning candidate, or its
// own row, which no block writes then; the best firework never loses).
// Advances gens_done (nothing else in this launch reads it).
__global__ void __launch_bounds__(256) k_select_copy(Problem p, const float* __restrict__ sparks,
                                                     const float* __restrict__ guides, float* __restrict__ fw_x,
                                                     const int32_t* __restrict__ winner,
                                                     float* __restrict__ best_x, const int32_t* __restrict__ loser,
                                                     uint32_t* __restrict__ gens_done) {
  griddep_wait();
  griddep_launch_dependents();
  const int nz = p.B * p.mu;
  const int y = blockIdx.y;
  if (blockIdx.x == 0 && y == 0 && threadIdx.x == 0) *gens_done += 1u;  // the generation is complete
  const int64_t n4 = p.Dp / 4;
  const int64_t chunk = (n4 + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = (int64_t)blockIdx.x * chunk;
  const int64_t e1 = e0 + chunk < n4 ? e0 + chunk : n4;
  int z, c;
  float* dst;
  if (y < nz && loser[y]) {
    const int b = y / p.mu, il = y - b * p.mu;
    const uint32_t gen = (uint32_t)winner[(int64_t)nz + p.B];
    uint32_t k0, k1;
    run_key(p, b, k0, k1);
    const float width = __fsub_rn(p.ub, p.lb);
    float4* d4 = reinterpret_cast<float4*>(fw_x + (int64_t)y * p.Dp);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const uint4 r = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)(il + p.fw_off), gen, kLoser), k0, k1);
      float v[4];
#pragma unroll
      for (int l = 0; l < 4; ++l) v[l] = (4 * e + l < p.D) ? __fmaf_rn(u24(lane_of(r, l)), width, p.lb) : 0.0f;
      d4[e] = make_float4(v[0], v[1], v[2], v[3]);
    }
    return;
  }
  if (y < nz) {
    z = y;
    c = winner[z];
    if (c < 0) return;
    dst = fw_x + (int64_t)z * p.Dp;
  } else {
    const int b = y - nz;
    const int bi = winner[nz + b];
    if (bi < 0) return;
    z = b * p.mu + bi;
    c = winner[z];
    dst = best_x + (int64_t)b * p.Dp;
  }
  const float* src = c < 0 ? fw_x + (int64_t)z * p.Dp
                     : c < p.lam ? sparks + ((int64_t)z * p.lam + c) * p.Dp
                                 : guides + ((int64_t)z * p.m + (c - p.lam)) * p.Dp;
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) d4[e] = s4[e];
}

// Each run's best-so-far (one block per run): strict improvement over its
// fireworks in index order (init: the first minimum of the initial
// fireworks).
__global__ void __launch_bounds__(kSelThreads) k_run_best(Problem p, int init, const float* __restrict__ fw_x,
                                                          const float* __restrict__ fw_f,
                                                          float* __restrict__ best_x, float* __restrict__ best_f,
                                                          uint32_t* __restrict__ gens_done) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ int s_bi;
  const int b = blockIdx.x;
  const float* f = fw_f + (int64_t)b * p.mu;
  if (threadIdx.x == 0) {
    int bi = init ? 0 : -1;
    float bf = init ? f[0] : best_f[b];
    for (int i = init ? 1 : 0; i < p.mu; ++i) {
      if (rank_key(f[i]) < rank_key(bf)) {
        bf = f[i];
        bi = i;
      }
    }
    if (bi >= 0) best_f[b] = bf;
    s_bi = bi;
    if (gens_done && b == 0) *gens_done += 1u;  // the generation is complete
  }
  __syncthreads();
  const int bi = s_bi;
  if (bi < 0) return;
  const float4* src = reinterpret_cast<const float4*>(fw_x + ((int64_t)b * p.mu + bi) * p.Dp);
  float4* dst = reinterpret_cast<float4*>(best_x + (int64_t)b * p.Dp);
  for (int64_t e = threadIdx.x; e < p.Dp / 4; e += blockDim.x) dst[e] = src[e];
}

// One warp per firework: the E best candidates in the (fitness, index)
// order, picked one at a time (E is small), each pick excluding the
// previous ones.  With `partial` (per-sample-tile loss sums [mtiles][count]
// of the guiding rows), the warp first finishes its firework's guiding
// fitness as the fitness-finish kernel does and stores it in fit_g.
__global__ void k_elite_pick(Problem p, const float* __restrict__ fit_e, float* __restrict__ fit_g,
                             int32_t E, int32_t* __restrict__ elite, const float* __restrict__ partial,
                             int32_t mtiles, int32_t count, float n_f) {
  griddep_wait();
  griddep_launch_dependents();
  const int z = blockIdx.x;
  const int lane = threadIdx.x;
  const int n_cand = p.lam + p.m;
  // the firework's candidates' fitness (explosion 0..lam-1, then guiding), staged once for the E passes
  __shared__ float cand[kPickStage];
  const bool staged = n_cand <= kPickStage;
  if (partial) {
    for (int q = lane; q < p.m; q += 32) {
      const int64_t r = (int64_t)z * p.m + q;
      const float v = __fdiv_rn(tile_sum(partial, r, count, mtiles), n_f);
      fit_g[r] = v;
      if (staged) cand[p.lam + q] = v;
    }
  } else if (staged) {
    for (int q = lane; q < p.m; q += 32) cand[p.lam + q] = fit_g[(int64_t)z * p.m + q];
  }
  if (staged) {
    for (int c = lane; c < p.lam; c += 32 * kSelChunk) {
      float v[kSelChunk];
#pragma unroll
      for (int u = 0; u < kSelChunk; ++u)
        v[u] = c + 32 * u < p.lam ? fit_e[(int64_t)z * p.lam + c + 32 * u] : 0.0f;
#pragma unroll
      for (int u = 0; u < kSelChunk; ++u)
        if (c + 32 * u < p.lam) cand[c + 32 * u] = v[u];
    }
  }
  __syncwarp();
  const int64_t n_e = (int64_t)p.B * p.mu * p.lam;
  float prev_f = 0.0f;
  int prev_c = -1;
  for (int e = 0; e < E; ++e) {
    float bf = 0.0f;
    int bc = -1;
    for (int c = lane; c < n_cand; c += 32) {
      const float f = staged ? cand[c]
                      : c < p.lam ? fit_e[(int64_t)z * p.lam + c]
                                  : fit_g[(int64_t)z * p.m + (c - p.lam)];
      if (prev_c >= 0 && !before(prev_f, prev_c, f, c)) continue;  // already picked
      take_if_before(bf, bc, f, c);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float of = __shfl_xor_sync(0xffffffffu, bf, off);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
      take_if_before(bf, bc, of, oc);
    }
    if (lane == 0) {
      int32_t row = -1;
      if (bc >= 0) row = bc < p.lam ? (int32_t)((int64_t)z * p.lam + bc) : (int32_t)(n_e + (int64_t)z * p.m + (bc - p.lam));
      elite[(int64_t)z * E + e] = row;
    }
    prev_f = bf;
    prev_c = bc;
  }
}

}  // namespace

int launch_elite_pick(const Problem& p, const float* fit_e, float* fit_g, int32_t E, int32_t* elite,
                      cudaStream_t s, const float* partial, int32_t mtiles, int64_t N, int64_t stride) {
  if (E <= 0) return 0;
  if (launch_pdl(k_elite_pick, dim3(p.B * p.mu), dim3(32), 0, s, p, fit_e, fit_g, E, elite, partial, mtiles,
                 (int32_t)(stride > 0 ? stride : (int64_t)p.B * p.mu * p.m), (float)N) != cudaSuccess)
    return -1;
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_rank(const Problem& p, float* fit_e, int32_t* top, int32_t* bottom, cudaStream_t s, const float* partial,
                int32_t mtiles, int64_t N, int64_t stride) {
  const int threads = p.g >= 256 ? 256 : ((p.g + 31) / 32) * 32;
  const size_t smem = (size_t)p.g * (sizeof(float) + sizeof(int));
  if (launch_pdl(k_rank, dim3(p.B * p.mu * p.m), dim3(threads), smem, s, p, fit_e, top, bottom, partial, mtiles,
                 (int32_t)(stride > 0 ? stride : (int64_t)p.B * p.mu * p.lam), (float)N) != cudaSuccess)
    return -1;
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_select(const Problem& p, const float* fit_e, const float* fit_g, const float* sparks,
                  const float* guides, float* fw_x, float* fw_amp, float* fw_f, int32_t* winner, float* best_x,
                  float* best_f, uint32_t* gens_done, float* f_old, int32_t* loser, cudaStream_t s) {
  if (launch_pdl(k_select_decide, dim3(p.B), dim3(kSelThreads), 0, s, p, fit_e, fit_g, fw_amp, fw_f, winner, best_f,
                 (const uint32_t*)gens_done, f_old, loser) != cudaSuccess)
    return -1;
  if (launch_pdl(k_select_copy, dim3(copy_blocks(p.Dp), p.B * p.mu + p.B), dim3(256), 0, s, p, sparks, guides, fw_x,
                 (const int32_t*)winner, best_x, (const int32_t*)loser, gens_done) != cudaSuccess)
    return -1;
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int launch_run_best_init(const Problem& p, const float* fw_x, const float* fw_f, float* best_x, float* best_f,
                         cudaStream_t s) {
  k_run_best<<<p.B, kSelThreads, 0, s>>>(p, 1, fw_x, fw_f, best_x, best_f, nullptr);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mgfwa
