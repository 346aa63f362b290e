// Tensor-core fitness of many sparks at once (GPU-MGFWA, Algorithm 1:
// "parallel evaluate all the fitness of the sparks"), written for sm_103a
// with tcgen05 MMAs, TMEM accumulators and TMA loads.
//
// Layer 1 of every spark's network is one dense GEMM of the shared batch
// X [N x d_in] against all sparks' stacked first-layer weights
// [count*h1 x d_in] (BF16 operands, or E4M3 operands with the scales applied
// in the epilogue; FP32 accumulation).  A tile is 128
// samples x S whole sparks (S*h1 accumulator columns), so that the tile owns
// complete hidden vectors.  Layer 2 also runs on the tensor cores: the
// epilogue adds b1 and applies the activation in place in TMEM, then one
// TF32 MMA per 8 hidden units multiplies that TMEM operand (A) by the
// spark's W2 (B, TMA-loaded from the FP32 spark row) into S*N2 logit
// columns.  The epilogue then reads only the logits, adds b2 and reduces the
// per-sample cross-entropy into one partial sum per (sample tile, spark).
// Nothing of the hidden layer is written to memory.
//
// The (b1, b2, W2) tail of a tile sits in one of three shared buffers, so the
// producer can stage tile t+1 while layer 2 of tile t-1 still reads W2.
//
// TMEM (512 columns) holds two halves of 256 columns; half b carries the
// layer-1 accumulator of tile b (S*h1 columns) and, beside it, that tile's
// logits (S*N2 columns): S = floor(256 / (h1 + N2)).
//
// One persistent CTA per SM; warp roles:
//   warp 0  TMA producer: per tile, b1 and b2 of the S sparks (bulk copies)
//           and their W2 (3-D tiled TMA, 128B swizzle) into one of two tail
//           buffers; then the X tile (128 x 64) and W1 tile (S*h1 x 64) of
//           every K block into a ring of shared-memory stages;
//   warp 1  TMEM allocator and single-thread MMA issuer: layer 1 of tile t
//           (M=128, N=S*h1, K=16, kind::f16), then layer 2 of tile t-1
//           (M=128, N=N2, K=8, kind::tf32, A from TMEM);
//   warps 2..  epilogue, two (BF16) or three (E4M3) warps per TMEM lane
//           quadrant, each taking every second or third spark of the tile.
// Every mbarrier wait is bounded: on timeout the CTA raises a flag in
// shared memory and a bit in the status word, every role leaves its loop,
// and the CTA waits (bounded) for its own copies and MMAs, frees its TMEM
// and returns.
#include <cuda.h>

#include <cstdio>
#include <array>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "fitness_tc.cuh"
#include "tc_ptx.cuh"

namespace mgfwa {

namespace {

using namespace tc;

constexpr int kBM = 128;         // samples per tile
constexpr int kRowBytes = 128;   // bytes of K per stage row: one 128-byte swizzle row
constexpr int kUmmaKBytes = 32;  // bytes of K per layer-1 MMA (16 BF16 or 32 E4M3)
constexpr int kUmmaK2 = 8;       // K per tcgen05.mma kind::tf32
constexpr int kAtomK2 = 32;      // FP32 elements per 128-byte swizzle row of W2
// Epilogue warps: 8 (two per TMEM lane quadrant) with BF16 operands, where layer 1's
// MMAs set the pace; 12 (three per quadrant) with E4M3, whose MMAs take half as long
// and leave the epilogue as the limit.
__host__ __device__ constexpr int epi_warps(bool f8) { return f8 ? 12 : 8; }
__host__ __device__ constexpr int threads_for(bool f8) { return 64 + 32 * epi_warps(f8); }
constexpr int kMaxStages = 6;
constexpr int kTmemCols = 512;   // two halves of 256 columns
constexpr int kTailBufs = 3;     // tail buffers (biases, W2[, W3]): the producer runs a tile ahead of layer 2

struct Smem {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t tmem_full[2];   // layer 1 of the half's tile is complete
  uint64_t tmem_empty[2];  // layer 2 of the half's tile consumed its TMEM operand
  uint64_t a2_full[2];     // the epilogue wrote act(h + b1) into TMEM
  uint64_t l2_full[2];     // layer 2 of the half's tile is complete (logits, or z2 for three layers)
  uint64_t l2_empty[2];    // the epilogue read the half's logits
  uint64_t a3_full[2];     // three layers: the epilogue wrote act(z2 + b2) into TMEM
  uint64_t l3_full[2];     // three layers: the half's logits are complete
  uint64_t tail_full[kTailBufs];
  uint64_t tail_empty[kTailBufs];
  uint64_t mma_done;
  uint32_t tmem_base;
  volatile int abort_flag;
};

__device__ __forceinline__ float act_f(int a, float v) { return a == kActTanh ? tanhf(v) : fmaxf(v, 0.0f); }

struct TcArgs {
  int32_t count;        // sparks in this launch
  int32_t first_spark;  // first spark row of the launch (operand and W2 tensor maps)
  int32_t m_tiles, n_tiles;
  int32_t k_blocks;
  int32_t k_last;       // layer-1 MMAs in the last K block (the rest of it is past d_in: zero fill)
  int32_t stages;
  int32_t S;            // sparks per tile
  int32_t C;            // classes (<= N2)
  int32_t act;
  int32_t c_pad;        // C rounded up to 4 (floats of b2 copied)
  float scale;          // layer-1 accumulator multiplier (1 for BF16; 1 / (inv_x inv_w) for E4M3)
  int64_t N;
  int64_t ld;           // FP32 row stride of the sparks
  int64_t b1_off, b2_off, bl_off;  // biases: layer 1, layer 2 (three layers), last layer
  int32_t act2;                     // three layers: the second hidden activation
  const float* rows;    // FP32 spark rows of this launch
  const int32_t* y;
  float* partial;       // [m_tiles][count]
  uint32_t* status;
  uint64_t wait_budget; // clock64 ticks before a wait gives up (0 = the default)
};

// H2 = 0: two layers, logits (NL columns per spark) = act(h + b1) W2^T.
// H2 > 0: three layers, z2 (H2 columns) = act(h + b1) W2^T, then logits =
// act(z2 + b2) W3^T, both TF32 MMAs with A from TMEM.
template <int H1, int H2, int NL, bool F8>
__global__ void __launch_bounds__(threads_for(F8), 1)
    k_fitness_tc(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_w,
                 const __grid_constant__ CUtensorMap tmap_w2, const __grid_constant__ CUtensorMap tmap_w3, TcArgs a) {
  griddep_wait();
  griddep_launch_dependents();
  constexpr int kBK = F8 ? 128 : 64;  // K elements per stage (one 128-byte row)
  constexpr int kEpiWarps = epi_warps(F8);
  constexpr int kGroups = kEpiWarps / 4;  // epilogue warps per TMEM lane quadrant
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  constexpr bool kL3 = H2 > 0;
  constexpr int kR2 = kL3 ? H2 : NL;                  // rows of layer 2's B operand
  constexpr int kAtoms = H1 / kAtomK2;                // W2 K-atoms per spark
  constexpr uint32_t kAtomBytes = kR2 * 128;          // one W2 K-atom: kR2 rows x 128 B
  constexpr int kAtoms3 = kL3 ? H2 / kAtomK2 : 0;     // W3 K-atoms per spark
  constexpr uint32_t kAtomBytes3 = NL * 128;
  constexpr uint32_t kW2Bytes = kAtoms * kAtomBytes + kAtoms3 * kAtomBytes3;  // W2 [and W3] of one spark
  constexpr int kTB = kL3 ? 2 : kTailBufs;            // tail buffers in use
  constexpr int kTailFloats = H1 + H2 + 32;           // b1, [b2,] last bias (C <= 32)
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = a.S;
  const int n_tile = S * H1;
  const uint32_t a_bytes = kBM * kRowBytes;
  const uint32_t b_bytes = (uint32_t)n_tile * kRowBytes;
  uint8_t* stage_a = base;
  uint8_t* stage_b = base + (size_t)a.stages * a_bytes;
  uint8_t* w2s = stage_b + (size_t)a.stages * b_bytes;                     // [kTB][S][kW2Bytes]
  float* tails = reinterpret_cast<float*>(w2s + kTB * (size_t)S * kW2Bytes); // [kTB][S][kTailFloats]
  float* red = tails + kTB * (size_t)S * kTailFloats;                      // [S][4]
  // TMEM columns of spark s within a half: layer-1 accumulator, [z2,] logits
  auto col_h = [&](int sp) { return (uint32_t)(sp * H1); };
  auto col_z2 = [&](int sp) { return (uint32_t)(S * H1 + sp * H2); };
  auto col_lg = [&](int sp) { return (uint32_t)(S * (H1 + H2) + sp * NL); };
  Smem* sm = reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(red + 4 * S) + 15) & ~uintptr_t(15));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = a.m_tiles * a.n_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&sm->full[s], 1);
      mbar_init(&sm->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm->tmem_full[b], 1);
      mbar_init(&sm->tmem_empty[b], 1);
      mbar_init(&sm->a2_full[b], kEpiWarps);
      mbar_init(&sm->l2_full[b], 1);
      mbar_init(&sm->l2_empty[b], kEpiWarps);
      mbar_init(&sm->a3_full[b], kEpiWarps);
      mbar_init(&sm->l3_full[b], 1);
    }
    for (int b = 0; b < kTB; ++b) {
      mbar_init(&sm->tail_full[b], 1);
      mbar_init(&sm->tail_empty[b], kEpiWarps);
    }
    mbar_init(&sm->mma_done, 1);
    sm->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                 "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = sm->tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t it = 0;
      bool ok = true;
      int local = 0;
      const uint32_t tail_bytes = (uint32_t)(H1 + H2 + a.c_pad) * 4u +
                                  (uint32_t)kAtoms * (uint32_t)(kL3 ? H2 : a.C) * 128u +
                                  (uint32_t)kAtoms3 * (uint32_t)a.C * 128u;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++local) {
        const int mt = t % a.m_tiles, nt = t / a.m_tiles;
        const int row_x = mt * kBM;
        const int row_w = (a.first_spark + nt * S) * H1;
        {
          // biases, W2 [and W3] of the tile's sparks, for the epilogue and layers 2 [and 3]
          const int tb = local % kTB;
          const uint32_t tuse = (uint32_t)(local / kTB);
          if (!mbar_wait(&sm->abort_flag, &sm->tail_empty[tb], (tuse & 1u) ^ 1u, a.status, 1u, a.wait_budget)) break;
          const int s0 = nt * S;
          const int s_valid = min(S, a.count - s0);
          mbar_expect_tx(&sm->tail_full[tb], tail_bytes * (uint32_t)s_valid);
          for (int s = 0; s < s_valid; ++s) {
            const float* row = a.rows + (int64_t)(s0 + s) * a.ld;
            float* tl = tails + ((size_t)tb * S + s) * kTailFloats;
            bulk_load(tl, row + a.b1_off, (uint32_t)H1 * 4u, &sm->tail_full[tb]);
            if (kL3) bulk_load(tl + H1, row + a.b2_off, (uint32_t)H2 * 4u, &sm->tail_full[tb]);
            bulk_load(tl + H1 + H2, row + a.bl_off, (uint32_t)a.c_pad * 4u, &sm->tail_full[tb]);
            uint8_t* w2 = w2s + ((size_t)tb * S + s) * kW2Bytes;
#pragma unroll
            for (int at = 0; at < kAtoms; ++at)
              tma_load_3d(w2 + at * kAtomBytes, &tmap_w2, at * kAtomK2, 0, a.first_spark + s0 + s, &sm->tail_full[tb]);
#pragma unroll
            for (int at = 0; at < kAtoms3; ++at)
              tma_load_3d(w2 + kAtoms * kAtomBytes + at * kAtomBytes3, &tmap_w3, at * kAtomK2, 0, a.first_spark + s0 + s,
                          &sm->tail_full[tb]);
          }
        }
        for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
          const int s = (int)(it % (uint32_t)a.stages);
          const uint32_t ph = (it / (uint32_t)a.stages) & 1u;
          if (!mbar_wait(&sm->abort_flag, &sm->empty[s], ph ^ 1u, a.status, 1u, a.wait_budget)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sm->full[s], a_bytes + b_bytes);
          tma_load_2d(stage_a + (size_t)s * a_bytes, &tmap_x, kb * kBK, row_x, &sm->full[s]);
          tma_load_2d(stage_b + (size_t)s * b_bytes, &tmap_w, kb * kBK, row_w, &sm->full[s]);
        }
      }
      // drain: every issued copy must land before the CTA may exit
      for (int l = local - kTB > 0 ? local - kTB : 0; l < local; ++l)
        mbar_drain(&sm->tail_full[l % kTB], (uint32_t)((l / kTB) & 1), a.status);
      if (it > 0) {
        const uint32_t last = it - 1;
        for (uint32_t j = (last + 1 > (uint32_t)a.stages ? last + 1 - a.stages : 0); j <= last; ++j)
          mbar_drain(&sm->full[j % (uint32_t)a.stages], (j / (uint32_t)a.stages) & 1u, a.status);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc1 = instr_desc(kBM, n_tile, F8 ? 0u : 1u);
      const uint32_t idesc2 = instr_desc(kBM, kR2, 2u);
      const uint32_t idesc3 = instr_desc(kBM, NL, 2u);
      uint32_t it = 0;
      int local = 0;
      bool ok = true;
      // layer 2 [and 3] of the tile with local index j (global index tj):
      // logits = act(h + b1) W2^T, or z2 = act(h + b1) W2^T then logits = act(z2 + b2) W3^T
      auto layer2 = [&](int j, int tj) -> bool {
        const int bj = j & 1;
        const uint32_t uj = (uint32_t)(j >> 1);
        const int tj_buf = j % kTB;
        if (!mbar_wait(&sm->abort_flag, &sm->a2_full[bj], uj & 1u, a.status, 2u, a.wait_budget)) return false;
        if (!mbar_wait(&sm->abort_flag, &sm->tail_full[tj_buf], (uint32_t)(j / kTB) & 1u, a.status, 2u, a.wait_budget)) return false;
        if (!mbar_wait(&sm->abort_flag, &sm->l2_empty[bj], (uj & 1u) ^ 1u, a.status, 2u, a.wait_budget)) return false;
        tc_fence_after();
        const int ntj = tj / a.m_tiles;
        const int s_valid = min(S, a.count - ntj * S);
        const uint32_t half = tmem_base + (uint32_t)(bj * 256);
        for (int s = 0; s < s_valid; ++s) {
          const uint32_t w2 = smem_u32(w2s + ((size_t)tj_buf * S + s) * kW2Bytes);
#pragma unroll
          for (int kk = 0; kk < H1 / kUmmaK2; ++kk) {
            const uint32_t b_addr = w2 + (uint32_t)((kk * kUmmaK2) / kAtomK2) * kAtomBytes +
                                    (uint32_t)((kk * kUmmaK2) % kAtomK2) * 4u;
            mma_tf32_ta(half + (kL3 ? col_z2(s) : col_lg(s)), half + col_h(s) + (uint32_t)(kk * kUmmaK2),
                        smem_desc(b_addr), idesc2, kk > 0 ? 1u : 0u);
          }
        }
        mma_commit(&sm->l2_full[bj]);
        if (kL3) {
          if (!mbar_wait(&sm->abort_flag, &sm->a3_full[bj], uj & 1u, a.status, 2u, a.wait_budget)) return false;
          tc_fence_after();
          for (int s = 0; s < s_valid; ++s) {
            const uint32_t w3 = smem_u32(w2s + ((size_t)tj_buf * S + s) * kW2Bytes) + (uint32_t)(kAtoms * kAtomBytes);
#pragma unroll
            for (int kk = 0; kk < (kL3 ? H2 : 8) / kUmmaK2; ++kk) {
              const uint32_t b_addr = w3 + (uint32_t)((kk * kUmmaK2) / kAtomK2) * kAtomBytes3 +
                                      (uint32_t)((kk * kUmmaK2) % kAtomK2) * 4u;
              mma_tf32_ta(half + col_lg(s), half + col_z2(s) + (uint32_t)(kk * kUmmaK2), smem_desc(b_addr), idesc3,
                          kk > 0 ? 1u : 0u);
            }
          }
          mma_commit(&sm->l3_full[bj]);
        }
        mma_commit(&sm->tmem_empty[bj]);
        return true;
      };
      int prev_t = -1;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++local) {
        const int b = local & 1;
        const uint32_t use = (uint32_t)(local >> 1);
        if (!mbar_wait(&sm->abort_flag, &sm->tmem_empty[b], (use & 1u) ^ 1u, a.status, 2u, a.wait_budget)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * 256);
        for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
          const int s = (int)(it % (uint32_t)a.stages);
          const uint32_t ph = (it / (uint32_t)a.stages) & 1u;
          if (!mbar_wait(&sm->abort_flag, &sm->full[s], ph, a.status, 2u, a.wait_budget)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_addr = smem_u32(stage_a + (size_t)s * a_bytes);
          const uint32_t b_addr = smem_u32(stage_b + (size_t)s * b_bytes);
          const int nk = kb + 1 == a.k_blocks ? a.k_last : kRowBytes / kUmmaKBytes;
#pragma unroll
          for (int k = 0; k < kRowBytes / kUmmaKBytes; ++k) {
            if (k >= nk) break;
            if (F8)
              mma_e4m3(d_tmem, smem_desc(a_addr + k * kUmmaKBytes), smem_desc(b_addr + k * kUmmaKBytes), idesc1,
                       (kb > 0 || k > 0) ? 1u : 0u);
            else
              mma_bf16(d_tmem, smem_desc(a_addr + k * kUmmaKBytes), smem_desc(b_addr + k * kUmmaKBytes), idesc1,
                       (kb > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(&sm->empty[s]);
        }
        if (!ok) break;
        mma_commit(&sm->tmem_full[b]);
        if (local > 0 && !layer2(local - 1, prev_t)) {
          ok = false;
          break;
        }
        prev_t = t;
      }
      if (ok && local > 0) layer2(local - 1, prev_t);
      // every issued MMA completes before TMEM is released: one more commit, bounded wait
      mma_commit(&sm->mma_done);
      mbar_drain(&sm->mma_done, 0u, a.status);
    }
  } else {
    // ---------------- epilogue ----------------
    const int ew = warp - 2;                 // 0 .. kEpiWarps-1
    const int quad = warp & 3;               // TMEM lane quadrant this warp may access
    const int grp = ew >> 2;                 // which of the tile's sparks (every kGroups-th one)
    const int et = threadIdx.x - 64;         // 0 .. 32 kEpiWarps - 1
    const int row_in_tile = quad * 32 + lane;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
    int local = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++local) {
      const int mt = t % a.m_tiles, nt = t / a.m_tiles;
      const int b = local & 1;
      const uint32_t use = (uint32_t)(local >> 1);
      const int s0 = nt * S;
      const int s_valid = min(S, a.count - s0);
      const int64_t n = (int64_t)mt * kBM + row_in_tile;
      const bool valid_row = n < a.N;
      const int label = valid_row ? a.y[n] : 0;   // issued before the waits
      const int tb = local % kTB;
      bool ok = mbar_wait(&sm->abort_flag, &sm->tmem_full[b], use & 1u, a.status, 4u, a.wait_budget);
      ok = ok && mbar_wait(&sm->abort_flag, &sm->tail_full[tb], (uint32_t)(local / kTB) & 1u, a.status, 4u, a.wait_budget);
      if (epi_bar_any<kEpiWarps>(!ok || sm->abort_flag)) break;
      tc_fence_after();
      const float* tail = tails + (size_t)tb * S * kTailFloats;
      const uint32_t hbase = lane_base + (uint32_t)(b * 256);
      // act(h + b1) in place: the TMEM A operand of layer 2
      for (int s = grp; s < s_valid; s += kGroups) {
        const float* b1 = tail + (size_t)s * kTailFloats;
#pragma unroll 1
        for (int j0 = 0; j0 < H1; j0 += 8) {
          float h[8];
          const uint32_t col = hbase + col_h(s) + (uint32_t)j0;
          tmem_ld8(col, h);
          tmem_wait_ld();
          const float4 bb0 = *reinterpret_cast<const float4*>(b1 + j0);
          const float4 bb1 = *reinterpret_cast<const float4*>(b1 + j0 + 4);
          // h * scale + b1 (one rounding; exactly h + b1 when scale is 1)
          const float sc = a.scale;
          h[0] = act_f(a.act, fmaf(h[0], sc, bb0.x)); h[1] = act_f(a.act, fmaf(h[1], sc, bb0.y));
          h[2] = act_f(a.act, fmaf(h[2], sc, bb0.z)); h[3] = act_f(a.act, fmaf(h[3], sc, bb0.w));
          h[4] = act_f(a.act, fmaf(h[4], sc, bb1.x)); h[5] = act_f(a.act, fmaf(h[5], sc, bb1.y));
          h[6] = act_f(a.act, fmaf(h[6], sc, bb1.z)); h[7] = act_f(a.act, fmaf(h[7], sc, bb1.w));
          tmem_st8(col, h);
        }
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm->a2_full[b]);
      ok = mbar_wait(&sm->abort_flag, &sm->l2_full[b], use & 1u, a.status, 4u, a.wait_budget);
      if (epi_bar_any<kEpiWarps>(!ok || sm->abort_flag)) break;
      tc_fence_after();
      if (kL3) {
        // act(z2 + b2) in place: the TMEM A operand of layer 3
        for (int s = grp; s < s_valid; s += kGroups) {
          const float* b2 = tail + (size_t)s * kTailFloats + H1;
#pragma unroll 1
          for (int j0 = 0; j0 < H2; j0 += 8) {
            float h[8];
            const uint32_t col = hbase + col_z2(s) + (uint32_t)j0;
            tmem_ld8(col, h);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] = act_f(a.act2, h[q] + b2[j0 + q]);
            tmem_st8(col, h);
          }
        }
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm->a3_full[b]);
        ok = mbar_wait(&sm->abort_flag, &sm->l3_full[b], use & 1u, a.status, 4u, a.wait_budget);
        if (epi_bar_any<kEpiWarps>(!ok || sm->abort_flag)) break;
        tc_fence_after();
      }
      for (int s = grp; s < s_valid; s += kGroups) {
        const float* b2 = tail + (size_t)s * kTailFloats + H1 + H2;  // the last layer's bias
        float z[NL];
        const uint32_t col = hbase + col_lg(s);
#pragma unroll
        for (int q = 0; q < NL; q += 16) tmem_ld16(col + (uint32_t)q, z + q);
        tmem_wait_ld();
        float ce = 0.0f;
        if (valid_row) {
          const int C = a.C;
          float zmax = -INFINITY;
          float zy = 0.0f;
#pragma unroll
          for (int c = 0; c < NL; ++c) {
            if (c < C) {
              z[c] += b2[c];
              zmax = fmaxf(zmax, z[c]);
              if (c == label) zy = z[c];
            }
          }
          float se = 0.0f;
#pragma unroll
          for (int c = 0; c < NL; ++c)
            if (c < C) se += expf(z[c] - zmax);
          ce = (zmax + logf(se)) - zy;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ce += __shfl_xor_sync(0xffffffffu, ce, off);
        if (lane == 0) red[s * 4 + quad] = ce;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&sm->l2_empty[b]);
        mbar_arrive(&sm->tail_empty[tb]);
      }
      epi_bar<kEpiWarps>();
      if (et < s_valid) {
        const int s = et;
        const float v = ((red[s * 4 + 0] + red[s * 4 + 1]) + red[s * 4 + 2]) + red[s * 4 + 3];
        a.partial[(int64_t)mt * a.count + s0 + s] = v;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(kTmemCols) : "memory");
  }
}

std::string g_err;

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encoder() {
  static EncodeTiled fn = nullptr;
  if (fn) return fn;
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || p == nullptr) {
    cudaGetLastError();
    return nullptr;
  }
  fn = reinterpret_cast<EncodeTiled>(p);
  return fn;
}

bool encode(CUtensorMap* map, CUtensorMapDataType type, uint32_t rank, const void* ptr, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box,
            CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B) {
  EncodeTiled enc = get_encoder();
  if (!enc) {
    g_err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, type, rank, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    g_err = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
    return false;
  }
  return true;
}

int n2_of(int C) { return C <= 16 ? 16 : 32; }
// two layers: h2 = 0
int sparks_per_tile(int h1, int h2, int C) { return 256 / (h1 + h2 + n2_of(C)); }

template <int H1, int H2, int NL, bool F8>
cudaError_t launch_hn(const TcPlan& plan, const TcArgs& args, cudaStream_t s, bool prepare_only) {
  cudaError_t e = ensure_smem_limit<k_fitness_tc<H1, H2, NL, F8>>(plan.smem_bytes);
  if (e != cudaSuccess || prepare_only) return e;
  const int tiles = args.m_tiles * args.n_tiles;
  const int grid = tiles < plan.num_sms ? tiles : plan.num_sms;
  return launch_pdl(k_fitness_tc<H1, H2, NL, F8>, dim3(grid), dim3(threads_for(F8)), plan.smem_bytes, s, plan.tmap_x,
                    plan.tmap_w, plan.tmap_w2, plan.tmap_w3, args);
}

template <int H1, bool F8>
cudaError_t launch_h1(const TcPlan& plan, const TcArgs& args, cudaStream_t s, bool prep) {
  if (args.C <= 16) return launch_hn<H1, 0, 16, F8>(plan, args, s, prep);
  return launch_hn<H1, 0, 32, F8>(plan, args, s, prep);
}

// The kernel instance for the plan's network and precision: launched, or
// (prep) only given its shared-memory allowance.
cudaError_t dispatch(const TcPlan& plan, const Mlp& mlp, const TcArgs& a, cudaStream_t s, bool prep) {
  const int h1 = mlp.widths[1];
  if (mlp.n_layers == 3) {
    // three layers: (128, 64) or (64, 32), at most 16 classes
    const int h2 = mlp.widths[2];
    if (h1 == 128 && h2 == 64)
      return plan.f8 ? launch_hn<128, 64, 16, true>(plan, a, s, prep) : launch_hn<128, 64, 16, false>(plan, a, s, prep);
    if (h1 == 64 && h2 == 32)
      return plan.f8 ? launch_hn<64, 32, 16, true>(plan, a, s, prep) : launch_hn<64, 32, 16, false>(plan, a, s, prep);
    return cudaErrorInvalidValue;
  }
  switch (h1 * 2 + (plan.f8 ? 1 : 0)) {
    case 64: return launch_h1<32, false>(plan, a, s, prep);
    case 128: return launch_h1<64, false>(plan, a, s, prep);
    case 256: return launch_h1<128, false>(plan, a, s, prep);
    case 65: return launch_h1<32, true>(plan, a, s, prep);
    case 129: return launch_h1<64, true>(plan, a, s, prep);
    case 257: return launch_h1<128, true>(plan, a, s, prep);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool tc_supported(const int32_t* widths, int n_layers) {
  if (widths[0] % 8 != 0) return false;
  const int h1 = widths[1];
  if (n_layers == 2) {
    if (!(h1 == 32 || h1 == 64 || h1 == 128)) return false;
    return widths[2] >= 2 && widths[2] <= 32;
  }
  if (n_layers == 3) {
    // (h1, h2) in {(128, 64), (64, 32)}, at most 16 classes
    const int h2 = widths[2];
    if (!((h1 == 128 && h2 == 64) || (h1 == 64 && h2 == 32))) return false;
    return widths[3] >= 2 && widths[3] <= 16;
  }
  return false;
}

namespace {

// The pair plan's tile shape: S sparks per tile, `stages` pipeline stages, K-tail buffers for `kt` MMAs
// (0 = none), and the first-layer operand's maps, whose box is half a tile's rows.
mgfwa_status pair_shape(TcPlan& plan, const Mlp& mlp, int S, int stages, int kt) {
  const int h1 = mlp.widths[1], d_in = mlp.widths[0];
  const int esize = plan.f8 ? 1 : 2, bk = kRowBytes / esize;
  const CUtensorMapDataType dt = plan.f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  plan.sparks_per_tile = S;
  plan.n_tile = S * h1;
  plan.stages = stages;
  plan.ktail = kt;
  plan.smem_bytes = tc_pair_fixed_smem(mlp, S) + (size_t)stages * tc_pair_stage_bytes(h1, S) +
                    tc_pair_ktail_bytes(h1, S, kt);
  {
    // first-layer operand [max_rows*h1][d_in], box (one 128-byte row of K) x half a tile's rows
    cuuint64_t dims[2] = {(cuuint64_t)d_in, (cuuint64_t)plan.w_rows};
    cuuint64_t strides[1] = {(cuuint64_t)d_in * esize};
    cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)(plan.n_tile / 2)};
    if (!encode(&plan.tmap_w, dt, 2, plan.w_base, dims, strides, box)) return MGFWA_ECUDA;
  }
  {
    // the same operand viewed as [K atoms entirely inside d_in][rows][one 128-byte atom], two atoms a load
    const int n_full = d_in / bk > 0 ? d_in / bk : 1;
    cuuint64_t dw[3] = {(cuuint64_t)bk, (cuuint64_t)plan.w_rows, (cuuint64_t)n_full};
    cuuint64_t sw[2] = {(cuuint64_t)d_in * esize, (cuuint64_t)kRowBytes};
    cuuint32_t bw[3] = {(cuuint32_t)bk, (cuuint32_t)(plan.n_tile / 2), 2};
    if (!encode(&plan.tmap_wk, dt, 3, plan.w_base, dw, sw, bw)) return MGFWA_ECUDA;
  }
  if (tc_pair_ktail_mmas(mlp, plan.f8) > 0) {
    // the same operand, box one MMA's K (32 bytes) x half a tile's rows, 32-byte swizzle: the K-tail loads
    cuuint64_t dims[2] = {(cuuint64_t)d_in, (cuuint64_t)plan.w_rows};
    cuuint64_t strides[1] = {(cuuint64_t)d_in * esize};
    cuuint32_t box[2] = {(cuuint32_t)(32 / esize), (cuuint32_t)(plan.n_tile / 2)};
    if (!encode(&plan.tmap_wt, dt, 2, plan.w_base, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_32B))
      return MGFWA_ECUDA;
  } else {
    plan.tmap_wt = plan.tmap_w;  // unused: no partial atom for the K-tail buffers
  }
  return MGFWA_OK;
}

}  // namespace

mgfwa_status tc_plan(TcPlan& plan, const Mlp& mlp, const OpDesc& op, const float* rows, int64_t ld,
                     int64_t max_rows) {
  plan = TcPlan();
  if (op.kind != kOpBf16 && op.kind != kOpFp8) {
    g_err = "tensor-core path needs a BF16 or FP8 operand";
    return MGFWA_EINVAL;
  }
  const bool f8 = op.kind == kOpFp8;
  const int esize = f8 ? 1 : 2, bk = kRowBytes / esize;
  plan.f8 = f8;
  if (!tc_supported(mlp.widths, mlp.n_layers)) {
    g_err = "network shape not supported by the tensor-core path";
    return MGFWA_EINVAL;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    g_err = "cudaGetDeviceProperties failed";
    return MGFWA_ECUDA;
  }
  if (prop.major != 10) {
    g_err = "tensor-core path needs a Blackwell (sm_10x) GPU";
    return MGFWA_EINVAL;
  }
  const bool l3 = mlp.n_layers == 3;
  const int h1 = mlp.widths[1], d_in = mlp.widths[0], h2 = l3 ? mlp.widths[2] : 0;
  const int C = mlp.widths[mlp.n_layers];
  const int n2 = n2_of(C);
  plan.num_sms = prop.multiProcessorCount;
  const CUtensorMapDataType dt = f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (op.w2 && tc_pair_supported(mlp.widths, mlp.n_layers)) {
    // the CTA-pair kernel: 256 samples x S sparks per tile, each CTA loading half of either operand
    plan.pair = true;
    plan.pairs = plan.num_sms / 2;
    plan.w_base = op.base;
    plan.w_rows = max_rows * h1;
    const int nl = tc_pair_logit_rows(C);
    const int w2r = tc_pair_w2_rows(mlp.widths, mlp.n_layers);
    if (op.w2_rows != w2r || op.w2_h1 != h1 || (l3 && (!op.w3 || op.w3_rows != nl || op.w3_k != h2))) {
      g_err = "pair kernel: the BF16 W2 / W3 copies have the wrong shape";
      return MGFWA_EINVAL;
    }
    {
      // X [N][d_in], box (one 128-byte row of K) x 128 samples
      cuuint64_t dims[2] = {(cuuint64_t)d_in, (cuuint64_t)mlp.N};
      cuuint64_t strides[1] = {(cuuint64_t)d_in * esize};
      cuuint32_t box[2] = {(cuuint32_t)bk, kBM};
      if (!encode(&plan.tmap_x, dt, 2, mlp.Xop, dims, strides, box)) return MGFWA_ECUDA;
    }
    {
      // X viewed as [K atoms entirely inside d_in][N][one 128-byte atom] (the atom stride is 128 bytes),
      // so that one load brings two atoms; the partial last atom goes through the plain view above, whose
      // fill past d_in is zero
      const int n_full = d_in / bk > 0 ? d_in / bk : 1;
      cuuint64_t dx[3] = {(cuuint64_t)bk, (cuuint64_t)mlp.N, (cuuint64_t)n_full};
      cuuint64_t sx[2] = {(cuuint64_t)d_in * esize, (cuuint64_t)kRowBytes};
      cuuint32_t bx[3] = {(cuuint32_t)bk, kBM, 2};
      if (!encode(&plan.tmap_x3, dt, 3, mlp.Xop, dx, sx, bx)) return MGFWA_ECUDA;
    }
    {
      // BF16 W2 [max_rows][w2r][h1], box 64 x w2r/2 x 1 (one CTA's half of the rows, one K atom)
      cuuint64_t dims[3] = {(cuuint64_t)h1, (cuuint64_t)w2r, (cuuint64_t)max_rows};
      cuuint64_t strides[2] = {(cuuint64_t)h1 * 2, (cuuint64_t)w2r * h1 * 2};
      cuuint32_t box[3] = {64, (cuuint32_t)(w2r / 2), 1};
      if (!encode(&plan.tmap_w2b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, op.w2, dims, strides, box)) return MGFWA_ECUDA;
    }
    if (l3) {
      // BF16 W3 [max_rows][nl][h2], box 64 x nl/2 x 1
      cuuint64_t dims[3] = {(cuuint64_t)h2, (cuuint64_t)nl, (cuuint64_t)max_rows};
      cuuint64_t strides[2] = {(cuuint64_t)h2 * 2, (cuuint64_t)nl * h2 * 2};
      cuuint32_t box[3] = {64, (cuuint32_t)(nl / 2), 1};
      if (!encode(&plan.tmap_w3b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, op.w3, dims, strides, box)) return MGFWA_ECUDA;
    } else {
      plan.tmap_w3b = plan.tmap_w2b;  // unused by the two-layer kernels
    }
    if (tc_pair_ktail_mmas(mlp, f8) > 0) {
      // X, box one MMA's K (32 bytes) x 128 samples, 32-byte swizzle: the K-tail loads of the partial atom
      cuuint64_t dims[2] = {(cuuint64_t)d_in, (cuuint64_t)mlp.N};
      cuuint64_t strides[1] = {(cuuint64_t)d_in * esize};
      cuuint32_t box[2] = {(cuuint32_t)(32 / esize), kBM};
      if (!encode(&plan.tmap_xt, dt, 2, mlp.Xop, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_32B)) return MGFWA_ECUDA;
    } else {
      plan.tmap_xt = plan.tmap_x;  // unused
    }
    plan.tmap_w2 = plan.tmap_w2b;  // unused by the pair kernel
    plan.tmap_w3 = plan.tmap_w2b;
    // the default shape: the logits in the sparks' own columns, the deepest pipeline that fits, and the
    // K-tail buffers if they fit beside it
    const int S = tc_pair_sparks(mlp, true);
    const size_t limit = (size_t)prop.sharedMemPerBlockOptin;
    const int stages = tc_pair_stages_fit(mlp, S, limit);
    if (stages < 2) {
      g_err = "shared memory too small for the tensor-core pair tiles";
      return MGFWA_EINVAL;
    }
    const int kt_want = tc_pair_ktail_mmas(mlp, f8);
    const int kt = kt_want > 0 && tc_pair_stages_fit(mlp, S, limit, kt_want) >= stages ? kt_want : 0;
    plan.ready = true;
    const mgfwa_status st = pair_shape(plan, mlp, S, stages, kt);
    if (st != MGFWA_OK) plan.ready = false;
    return st;
  }
  plan.sparks_per_tile = sparks_per_tile(h1, h2, C);
  plan.n_tile = plan.sparks_per_tile * h1;
  const size_t a_bytes = (size_t)kBM * kRowBytes, b_bytes = (size_t)plan.n_tile * kRowBytes;
  const int tbufs = l3 ? 2 : kTailBufs;  // the kernel's kTB
  const size_t wt_bytes = (size_t)(h1 / kAtomK2) * (l3 ? h2 : n2) * 128 + (l3 ? (size_t)(h2 / kAtomK2) * n2 * 128 : 0);
  const size_t w2_bytes = tbufs * (size_t)plan.sparks_per_tile * wt_bytes;
  const size_t tail_bytes =
      sizeof(float) * (tbufs * (size_t)plan.sparks_per_tile * (h1 + h2 + 32) + 4 * plan.sparks_per_tile);
  const size_t fixed = 1024 + w2_bytes + tail_bytes + 16 + sizeof(Smem) + 64;
  const size_t limit = (size_t)prop.sharedMemPerBlockOptin;
  int stages = kMaxStages;
  while (stages > 2 && fixed + stages * (a_bytes + b_bytes) > limit) --stages;
  if (fixed + stages * (a_bytes + b_bytes) > limit) {
    g_err = "shared memory too small for the tensor-core tiles";
    return MGFWA_EINVAL;
  }
  plan.stages = stages;
  plan.smem_bytes = fixed + stages * (a_bytes + b_bytes);
  {
    // X [N][d_in], box (one 128-byte row of K) x 128
    cuuint64_t dims[2] = {(cuuint64_t)d_in, (cuuint64_t)mlp.N};
    cuuint64_t strides[1] = {(cuuint64_t)d_in * esize};
    cuuint32_t box[2] = {(cuuint32_t)bk, kBM};
    if (!encode(&plan.tmap_x, dt, 2, mlp.Xop, dims, strides, box)) return MGFWA_ECUDA;
  }
  {
    // first-layer operand [max_rows*h1][d_in], box (one 128-byte row of K) x n_tile
    cuuint64_t dims[2] = {(cuuint64_t)d_in, (cuuint64_t)(max_rows * h1)};
    cuuint64_t strides[1] = {(cuuint64_t)d_in * esize};
    cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)plan.n_tile};
    if (!encode(&plan.tmap_w, dt, 2, op.base, dims, strides, box)) return MGFWA_ECUDA;
  }
  {
    // W2 of every spark straight from the FP32 rows: [max_rows][C or h2][h1], box 32 x rows x 1
    const int r2 = l3 ? h2 : C;
    cuuint64_t dims[3] = {(cuuint64_t)h1, (cuuint64_t)r2, (cuuint64_t)max_rows};
    cuuint64_t strides[2] = {(cuuint64_t)h1 * 4, (cuuint64_t)ld * 4};
    cuuint32_t box[3] = {kAtomK2, (cuuint32_t)r2, 1};
    if (!encode(&plan.tmap_w2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, rows + mlp.w_off[1], dims, strides, box))
      return MGFWA_ECUDA;
  }
  if (l3) {
    // W3 [max_rows][C][h2], box 32 x C x 1
    cuuint64_t dims[3] = {(cuuint64_t)h2, (cuuint64_t)C, (cuuint64_t)max_rows};
    cuuint64_t strides[2] = {(cuuint64_t)h2 * 4, (cuuint64_t)ld * 4};
    cuuint32_t box[3] = {kAtomK2, (cuuint32_t)C, 1};
    if (!encode(&plan.tmap_w3, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, rows + mlp.w_off[2], dims, strides, box))
      return MGFWA_ECUDA;
  } else {
    plan.tmap_w3 = plan.tmap_w2;  // unused by the two-layer kernels
  }
  plan.ready = true;
  return MGFWA_OK;
}

const char* tc_last_error() { return g_err.c_str(); }

void tc_release(TcPlan& plan) { plan.ready = false; }

int launch_fitness_tc(const TcPlan& plan, const Mlp& mlp, int64_t first, const float* rows, int64_t ld,
                      int32_t count, float scale, float* partial, uint32_t* status, cudaStream_t s) {
  if (!plan.ready || count <= 0) return count <= 0 ? 0 : -1;
  if (plan.pair) return launch_fitness_pair(plan, mlp, first, rows, ld, count, scale, partial, status, s);
  TcArgs a;
  a.count = count;
  a.first_spark = (int32_t)first;
  a.m_tiles = (int32_t)((mlp.N + kBM - 1) / kBM);
  a.S = plan.sparks_per_tile;
  a.n_tiles = (count + a.S - 1) / a.S;
  const int bk = plan.f8 ? 128 : 64;
  a.k_blocks = (mlp.widths[0] + bk - 1) / bk;
  {
    const int ke = plan.f8 ? 32 : 16;                       // K elements per MMA
    const int rem = mlp.widths[0] - (a.k_blocks - 1) * bk;  // K elements of the last block
    a.k_last = (rem + ke - 1) / ke;
  }
  a.scale = scale;
  a.stages = plan.stages;
  const bool l3 = mlp.n_layers == 3;
  a.C = mlp.widths[mlp.n_layers];
  a.act = mlp.acts[0];
  a.act2 = l3 ? mlp.acts[1] : 0;
  a.c_pad = (a.C + 3) / 4 * 4;
  a.N = mlp.N;
  a.ld = ld;
  a.b1_off = mlp.b_off[0];
  a.b2_off = l3 ? mlp.b_off[1] : 0;
  a.bl_off = mlp.b_off[mlp.n_layers - 1];
  a.rows = rows;
  a.y = mlp.y;
  a.partial = partial;
  a.status = status;
  a.wait_budget = plan.wait_budget;
  return dispatch(plan, mlp, a, s, false) == cudaSuccess ? 1 : -1;
}

cudaError_t tc_prepare(TcPlan& plan, const Mlp& mlp) {
  if (!plan.ready) return cudaErrorInvalidValue;
  if (plan.pair) return tc_pair_prepare(plan, mlp);
  TcArgs a = {};
  a.C = mlp.widths[mlp.n_layers];
  return dispatch(plan, mlp, a, nullptr, true);
}

mgfwa_status tc_pair_configure(TcPlan& plan, const Mlp& mlp, int sparks_per_tile, int stages, int ktail) {
  if (!plan.ready || !plan.pair) return MGFWA_EINVAL;
  if (sparks_per_tile <= 0 ||
      (sparks_per_tile != tc_pair_sparks(mlp, true) && sparks_per_tile != tc_pair_sparks(mlp, false))) {
    g_err = "pair kernel: no tile of that many sparks for this network";
    return MGFWA_EINVAL;
  }
  int dev = 0, limit = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    g_err = "device query failed";
    return MGFWA_ECUDA;
  }
  if (stages < 2 || stages > tc_pair_stages_fit(mlp, sparks_per_tile, (size_t)limit)) {
    g_err = "pair kernel: that pipeline depth does not fit in shared memory";
    return MGFWA_EINVAL;
  }
  if (ktail < -1 || ktail > 1) {
    g_err = "pair kernel: the K-tail choice is -1, 0 or 1";
    return MGFWA_EINVAL;
  }
  const int kt_want = tc_pair_ktail_mmas(mlp, plan.f8);
  const bool kt_fits = kt_want > 0 && stages <= tc_pair_stages_fit(mlp, sparks_per_tile, (size_t)limit, kt_want);
  if (ktail == 1 && !kt_fits) {
    g_err = kt_want > 0 ? "pair kernel: the K-tail buffers do not fit beside that pipeline"
                        : "pair kernel: the network has no partial K atom for the K-tail buffers";
    return MGFWA_EINVAL;
  }
  const int kt = ktail != 0 && kt_fits ? kt_want : 0;
  const mgfwa_status st = pair_shape(plan, mlp, sparks_per_tile, stages, kt);
  if (st != MGFWA_OK) return st;
  if (tc_pair_prepare(plan, mlp) != cudaSuccess) {
    g_err = "pair kernel attributes";
    return MGFWA_ECUDA;
  }
  return MGFWA_OK;
}

namespace {

// Tuned choices per (device, operand type, d_in, h1, classes, 256-sample tiles rounded up to a power of
// two, launch rows rounded up to a power of two): sparks per tile, stages and the K-tail choice.
std::mutex g_tune_mu;
std::map<std::array<int64_t, 7>, std::array<int, 3>> g_tuned;

int64_t pow2_at_least(int64_t v) {
  int64_t r = 1;
  while (r < v) r <<= 1;
  return r;
}

}  // namespace

mgfwa_status tc_pair_tune(TcPlan& plan, const Mlp& mlp, const float* rows, int64_t ld, int32_t count, float scale,
                          float* partial, uint32_t* status, cudaStream_t s) {
  if (!plan.ready || !plan.pair || count <= 0) return MGFWA_OK;
  // MGFWA_TUNE=0 keeps the default tile (deterministic creation time, reproducible profiles)
  if (const char* env = std::getenv("MGFWA_TUNE"))
    if (env[0] == '0' && env[1] == '\0') return MGFWA_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return MGFWA_OK;
  }
  int dev = 0, limit = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    g_err = "device query failed";
    return MGFWA_ECUDA;
  }
  // the network: d_in, then the hidden widths and classes packed (each below 2^16)
  int64_t net = 0;
  for (int l = 1; l <= mlp.n_layers; ++l) net = (net << 16) | mlp.widths[l];
  const std::array<int64_t, 7> key = {dev, plan.f8 ? 1 : 0, mlp.widths[0], net, mlp.n_layers,
                                      pow2_at_least((mlp.N + 255) / 256), pow2_at_least(count)};
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto hit = g_tuned.find(key);
  if (hit != g_tuned.end()) {
    const mgfwa_status st = tc_pair_configure(plan, mlp, hit->second[0], hit->second[1], hit->second[2]);
    if (st == MGFWA_OK) plan.tuned = 1;
    return st;
  }
  // the candidates: both tile shapes, every depth from two to the deepest that fits, the partial K atom as a
  // stage and (where the buffers fit beside that depth) through the K-tail buffers
  std::vector<std::array<int, 3>> cand;
  const int kt_want = tc_pair_ktail_mmas(mlp, plan.f8);
  for (bool shared : {true, false}) {
    const int S = tc_pair_sparks(mlp, shared);
    if (S <= 0 || (!shared && S == tc_pair_sparks(mlp, true))) continue;
    const int fit = tc_pair_stages_fit(mlp, S, (size_t)limit);
    const int fit_kt = kt_want > 0 ? tc_pair_stages_fit(mlp, S, (size_t)limit, kt_want) : 0;
    for (int st = 2; st <= fit; ++st) {
      cand.push_back({S, st, 0});
      if (st <= fit_kt) cand.push_back({S, st, 1});
    }
  }
  if (cand.empty()) return MGFWA_OK;
  std::vector<float> best(cand.size(), 1e30f);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    g_err = "event creation failed";
    return MGFWA_ECUDA;
  }
  mgfwa_status st = MGFWA_OK;
  // the candidates interleaved over rounds (the first one untimed: module loads, clocks ramping), each
  // timed over two launches, the minimum kept
  constexpr int kRounds = 4, kLaunches = 2;
  for (int r = 0; r < kRounds && st == MGFWA_OK; ++r) {
    for (size_t c = 0; c < cand.size() && st == MGFWA_OK; ++c) {
      st = tc_pair_configure(plan, mlp, cand[c][0], cand[c][1], cand[c][2]);
      if (st != MGFWA_OK) break;
      if (launch_fitness_tc(plan, mlp, 0, rows, ld, count, scale, partial, status, s) < 0 ||
          cudaEventRecord(e0, s) != cudaSuccess) {
        st = MGFWA_ECUDA;
        break;
      }
      for (int l = 0; l < kLaunches; ++l)
        if (launch_fitness_tc(plan, mlp, 0, rows, ld, count, scale, partial, status, s) < 0) st = MGFWA_ECUDA;
      float ms = 0.0f;
      if (st != MGFWA_OK || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = MGFWA_ECUDA;
        break;
      }
      if (r > 0 && ms < best[c]) best[c] = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MGFWA_OK) {
    if (st == MGFWA_ECUDA) g_err = "pair kernel tuning launch failed";
    return st;
  }
  size_t pick = 0;
  for (size_t c = 1; c < cand.size(); ++c)
    if (best[c] < best[pick]) pick = c;
  st = tc_pair_configure(plan, mlp, cand[pick][0], cand[pick][1], cand[pick][2]);
  if (st != MGFWA_OK) return st;
  plan.tuned = 1;
  g_tuned[key] = cand[pick];
  return MGFWA_OK;
}

}  // namespace mgfwa
