// Tensor-core fitness on CTA pairs (GPU-MGFWA, Algorithm 1: "parallel
// evaluate all the fitness of the sparks") for two-layer networks with
// h1 in {64, 128}, written for sm_103a: tcgen05 MMAs over a pair of CTAs
// (cta_group::2) with TMEM accumulators and TMA loads.
//
// A tile is 256 samples x S whole sparks, S = floor(256 / (h1 + NL)) (three
// for the 784-64-10 network), NL = 16 or 32 logit columns per spark.  Layer
// 1 is one dense product of the shared batch X against the sparks' stacked
// first-layer weights: M = 256 (128 samples in each CTA of the pair), N =
// S * h1 (all the tile's hidden units), BF16 or E4M3 operands, FP32
// accumulation.  Each CTA loads its own 128 rows of X and its own half of
// the tile's W1 block, so every SM stages and reads half the B operand a
// one-CTA tile of the same shape would; the accumulator of each CTA holds
// its 128 samples x all N columns.
//
// The epilogue adds b1 (after the E4M3 scale), applies the activation and
// writes the result back into TMEM as packed BF16 pairs, in the first h1/2
// columns of each spark's h1.  Layer 2 is then one BF16 MMA chain per
// spark (M = 256, N = NL, K = h1) with A read from TMEM and B = the spark's
// W2, which the samplers store as BF16 beside the first-layer operand (each
// CTA holds half of the logit rows).  The logits land in columns of their
// own after the tile's accumulator (S * (h1 + NL) <= 256), so layer 1 of
// tile t+2 in the same TMEM half waits only for layer 2 of tile t to have
// read its activations, never for the epilogue.  The epilogue reads the
// logits, adds b2 and reduces the per-sample cross-entropy into one partial
// sum per (128-sample tile, spark): the same partial layout as the one-CTA
// kernel.  TMEM (512 columns) holds two halves of 256 columns, one per tile
// in flight; the MMA thread issues layer 2 of a tile as soon as both
// epilogues have written its activations, between K blocks of the next tile.
//
// Warp roles (both CTAs unless stated):
//   warp 0  TMA producer: per tile, the biases (bulk copies, completing on
//           this CTA's barrier) and this CTA's half of the tile's W2 rows;
//           then per K step this CTA's X tile and W1 half into a ring of
//           stages.  A K step is two 128-byte K atoms (one tiled load per
//           operand through a view of K as atoms x 128 bytes): a stage takes
//           about the same time to arrive whatever its size, so fewer, larger
//           stages carry more bytes per unit time.  The atom that d_in ends
//           in, when partial, is either a step of its own through the plain
//           view, whose fill past d_in is zero, or (the K-tail buffers) one
//           small load per MMA of it and per operand (32 bytes of K, 32-byte
//           swizzle, zero past d_in) into one of two K-tail buffers, issued
//           after the tile's first step: a stage costs about one ring cycle
//           whatever it carries, so a ring of whole two-atom stages saves
//           one cycle per tile.  The operand loads of both CTAs complete on
//           the even CTA's barriers (the CTA-pair form of the tiled load),
//           whose producer expects both halves' bytes, so the MMA thread
//           waits on one barrier per stage.
//   warp 1  TMEM allocation for the pair (both CTAs); in the even CTA, the
//           single-thread MMA issuer.
//   warps 2..  epilogue, one warp per spark of the tile and TMEM lane
//           quadrant (at least two per quadrant).
// Every wait is bounded.  A CTA whose wait gives up raises its own and its
// peer's abort flag and a bit in the status word; every role leaves its
// loop, the even CTA's producer waits (bounded) for the stages it armed, the
// MMA thread for its MMAs, and an aborting CTA lets its last copies land (a
// bounded pause: the odd CTA cannot observe the even CTA's barriers) before
// the pair meets at a cluster barrier and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <string>

#include "fitness_tc.cuh"
#include "tc_ptx.cuh"

namespace mgfwa {

namespace {

using namespace tc;

constexpr int kPM = 128;     // samples per CTA (a pair covers 256)
constexpr int kRowB = 128;   // bytes of K per stage row: one 128-byte swizzle row
constexpr int kMmaKB = 32;   // bytes of K per layer-1 MMA (16 BF16 or 32 E4M3)
constexpr int kMaxStg = 8;
constexpr int kTBufs = 3;    // tail buffers: the producer runs ahead of layer 2
constexpr int kCols = 512;   // two halves of 256 columns
constexpr int kKtBox = 32;   // bytes of K per K-tail load row: one MMA's K, one 32-byte swizzle row
constexpr int kMaxKt = 3;    // K-tail MMAs a buffer may hold

// Tile shapes (S sparks of h1 hidden units, N = S * h1 accumulator columns
// of a TMEM half of 256):
//  * "shared" S = 256 / h1 (N = 256): each spark's logits go into the second
//    half of its own columns, freed once its activations are packed as BF16
//    pairs into the first half, so the next layer 1 into the same TMEM half
//    waits for both epilogues to have read the logits;
//  * "separate" S = 256 / (h1 + nl): the logits have columns of their own
//    after the accumulators, so the next layer 1 waits only for layer 2 to
//    have read the activations, and layer 2 for the epilogues to have read
//    the logits of the tile before.
// Both give every spark bitwise the same fitness (its columns are its own
// sums in the same order); which is faster depends on the shape, and the
// plan's tuner times both.
__host__ __device__ constexpr int pair_sparks_shared(int h1) { return 256 / h1; }
__host__ __device__ constexpr int pair_sparks_separate(int h1, int nl) { return 256 / (h1 + nl); }
// Epilogue warps: one per spark and TMEM lane quadrant, at least two per quadrant.
__host__ __device__ constexpr int pair_groups(int S) { return S < 2 ? 2 : S; }
__host__ __device__ constexpr int pair_threads(int S) { return 64 + 128 * pair_groups(S); }

struct PairSmem {
  uint64_t full[kMaxStg];      // even CTA: both CTAs' loads of the stage landed
  uint64_t empty[kMaxStg];     // the stage's MMAs completed
  uint64_t tmem_full[2];       // layer 1 of the half's tile is complete
  uint64_t a2_full[2];         // even CTA: both CTAs wrote the half's first-layer activations
  uint64_t l2_full[2];         // layer 2 of the half's tile is complete
  uint64_t a3_full[2];         // three layers, even CTA: both CTAs wrote the half's second-layer activations
  uint64_t l3_full[2];         // three layers: layer 3 (the logits) of the half's tile is complete
  uint64_t tmem_empty[2];      // even CTA: the half is free for the next layer 1 (shared: both CTAs read its
                               // logits; separate: layer 2 read its activations)
  uint64_t l2_empty[2];        // even CTA, separate logits: both CTAs read the half's logits
  uint64_t bias_full[kTBufs];  // this CTA's biases of the buffer's tile landed
  uint64_t w2_full[kTBufs];    // even CTA: both CTAs' W2 (and W3) halves of the buffer's tile landed
  uint64_t w2_empty;           // three layers: layer 3 read the single W2/W3 buffer
  uint64_t kt_full[2];         // even CTA: both CTAs' K-tail loads of the buffer's tile landed
  uint64_t kt_empty[2];        // the K-tail MMAs of the buffer's tile completed
  uint64_t tail_empty[kTBufs]; // the MMAs and this CTA's epilogue are done with the buffer's tile
  uint64_t mma_done;
  uint32_t tmem_base;
  volatile int abort_flag;
};


__device__ __forceinline__ float act_f(int a, float v) { return a == kActTanh ? tanhf(v) : fmaxf(v, 0.0f); }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// shared::cluster address of this CTA's object `p` in CTA `rank` of the pair.
__device__ __forceinline__ uint32_t map_to(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Two FP32 values as a BF16 pair (round to nearest even), the lower K index
// in the low half.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// act(acc * sc + bias) of `n` accumulator columns of this warp's lanes, from
// column `src`, as packed BF16 pairs into the columns from `dst` (dst <= src).
// Sixteen columns are loaded with one wait, then packed and stored: a group
// writes [dst + g/2, dst + g/2 + 8) for the group at src + g, columns that
// this or an earlier group has read.
template <int n>
__device__ __forceinline__ void pack_layer(uint32_t src, uint32_t dst, const float* bias, float sc, int act) {
  constexpr int kG = n < 16 ? n : 16;
#pragma unroll 1
  for (int g = 0; g < n; g += kG) {
    float h[kG];
#pragma unroll
    for (int j0 = 0; j0 < kG; j0 += 16) tmem_ld16(src + (uint32_t)(g + j0), h + j0);
    tmem_wait_ld();
#pragma unroll
    for (int j0 = 0; j0 < kG; j0 += 16) {
      uint32_t pk[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float2 bb = *reinterpret_cast<const float2*>(bias + g + j0 + 2 * q);
        pk[q] = pack_bf16x2(act_f(act, fmaf(h[j0 + 2 * q], sc, bb.x)), act_f(act, fmaf(h[j0 + 2 * q + 1], sc, bb.y)));
      }
      tmem_st8u(dst + (uint32_t)((g + j0) / 2), pk);
    }
  }
}

// H2 > 0: three layers (h1 -> h2 -> logits, both hidden layers activated).
// Then the tile is always the shared shape (S = 256 / h1): per spark, the
// packed first-layer activations in its first h1/2 columns, layer 2's h2
// outputs in the next h2 columns, packed in place by the epilogue into h2/2
// columns, and the logits after them.  W2 and W3 (BF16 copies beside the
// first-layer operand, each CTA holding half of either's rows) share one
// buffer, loaded by the producer between K steps of the tile once layer 3 of
// the tile before has read it.
//
// kGroup: one launch over several handles' sparks.  Their tiles are laid end
// to end (member i's tiles from members[i].tile_start on), and each role
// walks ascending tiles with a cursor into the member table (device memory:
// the members' tensor maps and arguments).  Otherwise the kernel parameters
// hold the one launch's maps and `a` its arguments.  `a` also carries what
// every member shares: stages, the status word and the wait budget.
template <int H1, int H2, int NL, int S, bool F8, bool kGroup>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(pair_threads(S), 1)
    k_fitness_pair(const __grid_constant__ CUtensorMap tmap_x3, const __grid_constant__ CUtensorMap tmap_x,
                   const __grid_constant__ CUtensorMap tmap_w3, const __grid_constant__ CUtensorMap tmap_w,
                   const __grid_constant__ CUtensorMap tmap_w2, const __grid_constant__ CUtensorMap tmap_wl3,
                   const __grid_constant__ CUtensorMap tmap_xt, const __grid_constant__ CUtensorMap tmap_wt,
                   PairArgs a, const PairMember* __restrict__ members, int32_t n_members) {
  constexpr bool kL3 = H2 > 0;
  constexpr int kNT = S * H1;                              // layer-1 accumulator columns per tile
  constexpr bool kShared = kL3 || S * (H1 + NL) > 256;     // the logits share the spark's accumulator columns
  constexpr int kBK = F8 ? 128 : 64;                       // K elements per atom (one 128-byte row)
  constexpr int kGroups = pair_groups(S);                  // epilogue warps per TMEM lane quadrant
  constexpr int kEpi = 4 * kGroups;
  constexpr int kWB = kL3 ? 1 : kTBufs;                    // W2 (and W3) buffers
  constexpr int kN2 = kL3 ? H2 : NL;                       // layer-2 outputs per spark
  constexpr int kW2Atoms = H1 / 64;                        // 128-byte K atoms of a BF16 W2 row
  constexpr uint32_t kW2AtomBytes = (kN2 / 2) * 128;       // each CTA holds half of W2's rows
  constexpr uint32_t kW2Bytes = kW2Atoms * kW2AtomBytes;   // one spark's W2 half
  constexpr int kW3Atoms = kL3 ? H2 / 64 : 0;
  constexpr uint32_t kW3AtomBytes = (NL / 2) * 128;
  constexpr uint32_t kW3Bytes = kW3Atoms * kW3AtomBytes;   // one spark's W3 half
  constexpr uint32_t kWSpark = kW2Bytes + kW3Bytes;
  constexpr int kTailF = H1 + H2 + 32;                     // b1, b2 (three layers) and the logits' bias
  constexpr uint32_t kAtomA = kPM * kRowB;                 // one K atom of this CTA's 128 samples
  constexpr uint32_t kAtomB = (kNT / 2) * kRowB;           // one K atom of this CTA's half of the tile's W1 rows
  constexpr uint32_t kStageA = 2 * kAtomA;                 // a stage: two atoms of each operand
  constexpr uint32_t kStageB = 2 * kAtomB;
  constexpr uint32_t kKtA = kPM * kKtBox;                  // one K-tail MMA's K of this CTA's samples
  constexpr uint32_t kKtB = (kNT / 2) * kKtBox;            // and of its half of the tile's W1 rows
  constexpr int kKtElems = F8 ? 32 : 16;                   // K elements per K-tail load
  static_assert((kN2 / 2) % 8 == 0 && (NL / 2) % 8 == 0, "each W2 / W3 half is whole 8-row swizzle groups");
  static_assert(S >= 1 && kNT <= 256 && (!kShared || NL <= H1 / 2), "a tile's columns fit in a TMEM half");
  static_assert(!kL3 || (H2 % 64 == 0 && H2 <= H1 / 2 && H2 / 2 + NL <= H1 / 2 && NL == 16),
                "three layers: layer 2's outputs and the logits fit in the spark's second h1/2 columns");
  static_assert((kNT / 2) % 8 == 0 && kNT % 16 == 0, "a W1 half is whole 8-row groups; N is a multiple of 16");

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // [2 buffers][kt_region A loads, kt_region B loads], each a multiple of 1024 bytes, before the stages
  uint8_t* ktail = base;
  const uint32_t kt_buf = (uint32_t)a.kt_region * (kKtA + kKtB);
  auto kt_a = [&](int buf, int k) { return ktail + (uint32_t)buf * kt_buf + (uint32_t)k * kKtA; };
  auto kt_b = [&](int buf, int k) {
    return ktail + (uint32_t)buf * kt_buf + (uint32_t)a.kt_region * kKtA + (uint32_t)k * kKtB;
  };
  // the partial last atom of a member goes through the K-tail buffers when they can hold it
  auto kt_on = [&](const PairArgs& m) { return m.kt > 0 && m.kt <= a.kt_region; };
  uint8_t* stage_a = base + 2 * kt_buf;
  uint8_t* stage_b = stage_a + (size_t)a.stages * kStageA;
  uint8_t* w2s = stage_b + (size_t)a.stages * kStageB;                               // [kWB][S][kWSpark]
  float* tails = reinterpret_cast<float*>(w2s + (size_t)kWB * S * kWSpark);          // [kTBufs][S][kTailF]
  float* red = tails + (size_t)kTBufs * S * kTailF;                                  // [S][4]
  PairSmem* sm = reinterpret_cast<PairSmem*>((reinterpret_cast<uintptr_t>(red + 4 * S) + 15) & ~uintptr_t(15));

  // TMEM columns of spark s within a half: its accumulator / packed activations, layer 2's outputs / their
  // packed activations (three layers), its logits
  auto col_h = [](int sp) { return (uint32_t)(sp * H1); };
  auto col_l2 = [](int sp) {
    return kL3 ? (uint32_t)(sp * H1 + H1 / 2)
               : (kShared ? (uint32_t)(sp * H1 + H1 / 2) : (uint32_t)(S * H1 + sp * NL));
  };
  auto col_lg = [&](int sp) { return kL3 ? (uint32_t)(sp * H1 + H1 / 2 + H2 / 2) : col_l2(sp); };
  const uint32_t rank = cluster_rank();
  const bool lead = rank == 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
  const int tiles = kGroup ? members[n_members - 1].tile_start + members[n_members - 1].tiles : a.m_pairs * a.n_tiles;
  // the member of tile t (advancing `cur`) and t's index among that member's tiles
  auto member_at = [&](int t, int& cur) -> int {
    if constexpr (kGroup) {
      while (cur + 1 < n_members && t >= members[cur + 1].tile_start) ++cur;
      return t - members[cur].tile_start;
    } else {
      (void)cur;
      return t;
    }
  };
  auto args_of = [&](int cur) -> const PairArgs& { return kGroup ? members[cur].a : a; };
  // the W2 buffer of the tile with local index j, and the phase of its barriers for that tile
  auto w_buf = [](int j) { return kL3 ? 0 : j % kTBufs; };
  auto w_phase = [](int j) { return kL3 ? (uint32_t)(j & 1) : (uint32_t)(j / kTBufs) & 1u; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&sm->full[s], 1);
      mbar_init(&sm->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm->tmem_full[b], 1);
      mbar_init(&sm->a2_full[b], 2 * kEpi);
      mbar_init(&sm->l2_full[b], 1);
      mbar_init(&sm->a3_full[b], 2 * kEpi);
      mbar_init(&sm->l3_full[b], 1);
      mbar_init(&sm->tmem_empty[b], kShared ? 2 * kEpi : 1);
      mbar_init(&sm->l2_empty[b], 2 * kEpi);
    }
    for (int b = 0; b < kTBufs; ++b) {
      mbar_init(&sm->bias_full[b], 1);
      mbar_init(&sm->w2_full[b], 1);
      mbar_init(&sm->tail_empty[b], 1 + kEpi);
    }
    mbar_init(&sm->w2_empty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm->kt_full[b], 1);
      mbar_init(&sm->kt_empty[b], 1);
    }
    mbar_init(&sm->mma_done, 1);
    sm->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                 "n"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync();  // both CTAs' barriers initialised and TMEM allocated before any cross-CTA access
  tc_fence_after();
  const uint32_t tmem_base = sm->tmem_base;
  // the set-up above touches nothing the previous kernel writes, so it overlaps that kernel's tail
  griddep_wait();
  griddep_launch_dependents();

  // A wait that gives up also stops the peer CTA.
  const uint32_t peer_abort = map_to((const void*)&sm->abort_flag, rank ^ 1u);
  auto wait = [&](uint64_t* bar, uint32_t parity, uint32_t code) -> bool {
    if (mbar_wait(&sm->abort_flag, bar, parity, a.status, code, a.wait_budget)) return true;
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(peer_abort), "r"(1u) : "memory");
    return false;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs) ----------------
      uint32_t it = 0;
      int local = 0;
      bool ok = true;
      int cur = 0, fenced = -1;
      int w_last = -1;  // three layers: the last tile whose W2/W3 loads were issued
      int kt_n = 0;     // tiles whose K-tail loads were issued
      for (int t = pair; t < tiles && ok; t += npairs, ++local) {
        const int lt = member_at(t, cur);
        const PairArgs& m = args_of(cur);
        const CUtensorMap* mx3 = kGroup ? &members[cur].x3 : &tmap_x3;
        const CUtensorMap* mx = kGroup ? &members[cur].x : &tmap_x;
        const CUtensorMap* mw3 = kGroup ? &members[cur].w3 : &tmap_w3;
        const CUtensorMap* mw = kGroup ? &members[cur].w : &tmap_w;
        const CUtensorMap* mw2 = kGroup ? &members[cur].w2 : &tmap_w2;
        const CUtensorMap* mwl3 = kGroup ? &members[cur].wl3 : &tmap_wl3;
        const CUtensorMap* mxt = kGroup ? &members[cur].xt : &tmap_xt;
        const CUtensorMap* mwt = kGroup ? &members[cur].wt : &tmap_wt;
        if (kGroup && fenced != cur) {
          // the member's maps were written to global memory by the host: order the tensor-map proxy's reads
          for (const CUtensorMap* mp : {mx3, mx, mw3, mw, mw2, mwl3, mxt, mwt})
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mp) : "memory");
          fenced = cur;
        }
        const uint32_t bias_bytes = (uint32_t)(H1 + H2 + m.c_pad) * 4u;
        const int mt = lt % m.m_pairs, nt = lt / m.m_pairs;
        const int s0 = nt * S;
        const int s_valid = min(S, m.count - s0);
        const int tb = local % kTBufs;
        const uint32_t tuse = (uint32_t)(local / kTBufs);
        if (!wait(&sm->tail_empty[tb], (tuse & 1u) ^ 1u, 1u)) break;
        mbar_expect_tx(&sm->bias_full[tb], bias_bytes * (uint32_t)s_valid);
        for (int s = 0; s < s_valid; ++s) {
          const float* row = m.rows + (int64_t)(s0 + s) * m.ld;
          float* tl = tails + ((size_t)tb * S + s) * kTailF;
          bulk_load(tl, row + m.b1_off, (uint32_t)H1 * 4u, &sm->bias_full[tb]);
          if (kL3) bulk_load(tl + H1, row + m.b2_off, (uint32_t)H2 * 4u, &sm->bias_full[tb]);
          bulk_load(tl + H1 + H2, row + m.bl_off, (uint32_t)m.c_pad * 4u, &sm->bias_full[tb]);
        }
        // this CTA's W2 (and W3) halves; the even CTA's barrier expects both CTAs' bytes
        const int wb = w_buf(local);
        auto issue_w = [&]() {
          if (lead) mbar_expect_tx(&sm->w2_full[wb], 2u * kWSpark * (uint32_t)s_valid);
          const uint32_t w2_bar = map_to(&sm->w2_full[wb], 0u);
          for (int s = 0; s < s_valid; ++s) {
            uint8_t* w2 = w2s + ((size_t)wb * S + s) * kWSpark;
#pragma unroll
            for (int at = 0; at < kW2Atoms; ++at)
              tma_load_3d_pair(w2 + at * kW2AtomBytes, mw2, at * 64, (int)rank * (kN2 / 2), m.first_spark + s0 + s,
                               w2_bar);
#pragma unroll
            for (int at = 0; at < kW3Atoms; ++at)
              tma_load_3d_pair(w2 + kW2Bytes + at * kW3AtomBytes, mwl3, at * 64, (int)rank * (NL / 2),
                               m.first_spark + s0 + s, w2_bar);
          }
          w_last = local;
        };
        // two layers: W2 rides in the tail buffer just freed; three: once layer 3 of the tile before read
        // the single buffer, between this tile's K steps
        if (!kL3) issue_w();
        const int row_x = mt * (2 * kPM) + (int)rank * kPM;
        const int row_w = (m.first_spark + s0) * H1 + (int)rank * (kNT / 2);
        const int n_pairs = (m.n_full + 1) / 2;
        const bool kt = kt_on(m);
        const int steps = kt ? n_pairs : m.n_steps;
        for (int kb = 0; kb < steps; ++kb, ++it) {
          if (kL3 && w_last != local && mbar_test_wait(&sm->w2_empty, ((uint32_t)local & 1u) ^ 1u)) issue_w();
          const int st = (int)(it % (uint32_t)a.stages);
          const uint32_t ph = (it / (uint32_t)a.stages) & 1u;
          if (!wait(&sm->empty[st], ph ^ 1u, 1u)) {
            ok = false;
            break;
          }
          const uint32_t bar = map_to(&sm->full[st], 0u);
          if (kb < n_pairs) {
            // atoms 2 kb and 2 kb + 1 (the second one past n_full is zero fill)
            if (lead) mbar_expect_tx(&sm->full[st], 2u * (kStageA + kStageB));
            tma_load_3d_pair(stage_a + (size_t)st * kStageA, mx3, 0, row_x, 2 * kb, bar);
            tma_load_3d_pair(stage_b + (size_t)st * kStageB, mw3, 0, row_w, 2 * kb, bar);
          } else {
            // the partial last atom, zero past d_in
            if (lead) mbar_expect_tx(&sm->full[st], 2u * (kAtomA + kAtomB));
            tma_load_2d_pair(stage_a + (size_t)st * kStageA, mx, m.n_full * kBK, row_x, bar);
            tma_load_2d_pair(stage_b + (size_t)st * kStageB, mw, m.n_full * kBK, row_w, bar);
          }
          if (kt && kb == 0) {
            // the partial last atom into a K-tail buffer (needed only after the tile's last stage), zero
            // past d_in
            const int kbuf = kt_n & 1;
            if (!wait(&sm->kt_empty[kbuf], ((uint32_t)(kt_n >> 1) & 1u) ^ 1u, 1u)) {
              ++it;  // this step's stage is armed: the drain below counts it
              ok = false;
              break;
            }
            if (lead) mbar_expect_tx(&sm->kt_full[kbuf], 2u * (uint32_t)m.kt * (kKtA + kKtB));
            const uint32_t kbar = map_to(&sm->kt_full[kbuf], 0u);
            for (int k = 0; k < m.kt; ++k) {
              tma_load_2d_pair(kt_a(kbuf, k), mxt, m.n_full * kBK + k * kKtElems, row_x, kbar);
              tma_load_2d_pair(kt_b(kbuf, k), mwt, m.n_full * kBK + k * kKtElems, row_w, kbar);
            }
            ++kt_n;
          }
        }
        if (kL3 && ok && w_last != local) {
          if (!wait(&sm->w2_empty, ((uint32_t)local & 1u) ^ 1u, 1u)) {
            ok = false;
          } else {
            issue_w();
          }
        }
      }
      // copies land before the CTA may leave: this CTA's biases, and (even CTA) the stages and W2 it
      // armed, which also carry the odd CTA's bytes.  Short budgets: only an aborting run waits here.
      constexpr uint64_t kDrain = 1ull << 24;
      for (int l = local - kTBufs > 0 ? local - kTBufs : 0; l < local; ++l) {
        mbar_drain(&sm->bias_full[l % kTBufs], (uint32_t)((l / kTBufs) & 1), a.status, kDrain);
        if (lead && !kL3) mbar_drain(&sm->w2_full[l % kTBufs], (uint32_t)((l / kTBufs) & 1), a.status, kDrain);
      }
      if (lead && kL3 && w_last >= 0) mbar_drain(&sm->w2_full[0], (uint32_t)(w_last & 1), a.status, kDrain);
      if (lead)
        for (int j = kt_n > 2 ? kt_n - 2 : 0; j < kt_n; ++j)
          mbar_drain(&sm->kt_full[j & 1], (uint32_t)(j >> 1) & 1u, a.status, kDrain);
      if (lead && it > 0) {
        const uint32_t last = it - 1;
        for (uint32_t j = (last + 1 > (uint32_t)a.stages ? last + 1 - a.stages : 0); j <= last; ++j)
          mbar_drain(&sm->full[j % (uint32_t)a.stages], (j / (uint32_t)a.stages) & 1u, a.status, kDrain);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && lead) {
      // ---------------- MMA issuer (even CTA) ----------------
      const uint32_t idesc1 = instr_desc(2 * kPM, kNT, F8 ? 0u : 1u);
      const uint32_t idesc2 = instr_desc(2 * kPM, kN2, 1u);
      const uint32_t idesc3 = instr_desc(2 * kPM, NL, 1u);
      auto commit_both = [&](uint64_t* bar) {
        mma2_commit(map_to(bar, 0u));
        mma2_commit(map_to(bar, 1u));
      };
      // layer 2 of the tile with local index j is ready when both CTAs wrote its activations and both W2
      // halves landed (and, separate logits, both epilogues read the logits of the tile before in the half)
      auto l2_ready = [&](int j) -> bool {
        return mbar_test_wait(&sm->a2_full[j & 1], (uint32_t)(j >> 1) & 1u) &&
               mbar_test_wait(&sm->w2_full[w_buf(j)], w_phase(j)) &&
               (kShared || mbar_test_wait(&sm->l2_empty[j & 1], ((uint32_t)(j >> 1) & 1u) ^ 1u));
      };
      auto layer2 = [&](int j, int s_valid) -> bool {
        const int bj = j & 1;
        const int wbj = w_buf(j);
        if (!wait(&sm->a2_full[bj], (uint32_t)(j >> 1) & 1u, 2u)) return false;
        if (!wait(&sm->w2_full[wbj], w_phase(j), 2u)) return false;
        if (!kShared && !wait(&sm->l2_empty[bj], ((uint32_t)(j >> 1) & 1u) ^ 1u, 2u)) return false;
        tc_fence_after();
        const uint32_t half = tmem_base + (uint32_t)(bj * 256);
        for (int s = 0; s < s_valid; ++s) {
          const uint32_t w2 = smem_u32(w2s + ((size_t)wbj * S + s) * kWSpark);
#pragma unroll
          for (int kk = 0; kk < H1 / 16; ++kk) {
            const uint32_t b_addr = w2 + (uint32_t)((kk * 16) / 64) * kW2AtomBytes + (uint32_t)((kk * 16) % 64) * 2u;
            mma2_bf16_ta(half + col_l2(s), half + col_h(s) + (uint32_t)(kk * 8), smem_desc(b_addr), idesc2,
                         kk > 0 ? 1u : 0u);
          }
        }
        commit_both(&sm->l2_full[bj]);
        if (!kShared) mma2_commit(map_to(&sm->tmem_empty[bj], 0u));
        if (!kL3) commit_both(&sm->tail_empty[j % kTBufs]);
        return true;
      };
      // three layers: layer 3 (the logits) once both CTAs packed the second-layer activations
      auto layer3 = [&](int j, int s_valid) -> bool {
        const int bj = j & 1;
        if (!wait(&sm->a3_full[bj], (uint32_t)(j >> 1) & 1u, 2u)) return false;
        tc_fence_after();
        const uint32_t half = tmem_base + (uint32_t)(bj * 256);
        for (int s = 0; s < s_valid; ++s) {
          const uint32_t w3 = smem_u32(w2s + (size_t)s * kWSpark + kW2Bytes);
#pragma unroll
          for (int kk = 0; kk < H2 / 16; ++kk) {
            const uint32_t b_addr = w3 + (uint32_t)((kk * 16) / 64) * kW3AtomBytes + (uint32_t)((kk * 16) % 64) * 2u;
            mma2_bf16_ta(half + col_lg(s), half + col_l2(s) + (uint32_t)(kk * 8), smem_desc(b_addr), idesc3,
                         kk > 0 ? 1u : 0u);
          }
        }
        commit_both(&sm->l3_full[bj]);
        commit_both(&sm->w2_empty);
        commit_both(&sm->tail_empty[j % kTBufs]);
        return true;
      };
      uint32_t it = 0;
      int local = 0;
      bool ok = true;
      // the tile whose later layers are not all issued yet, its spark count, and its next layer (2 or 3)
      int pend = -1, pend_sv = 0, pend_layer = 2;
      // issue the pending tile's next layers: those that are ready, or (block) all of them
      auto advance = [&](bool block) -> bool {
        if (pend < 0) return true;
        if (pend_layer == 2) {
          if (!block && !l2_ready(pend)) return true;
          if (!layer2(pend, pend_sv)) return false;
          if (!kL3) {
            pend = -1;
            return true;
          }
          pend_layer = 3;
        }
        if constexpr (kL3) {
          if (!block && !mbar_test_wait(&sm->a3_full[pend & 1], (uint32_t)(pend >> 1) & 1u)) return true;
          if (!layer3(pend, pend_sv)) return false;
        }
        pend = -1;
        return true;
      };
      int cur = 0;
      int kt_n = 0;  // tiles whose K-tail MMAs were issued
      for (int t = pair; t < tiles && ok; t += npairs, ++local) {
        const int lt = member_at(t, cur);
        const PairArgs& m = args_of(cur);
        const int b = local & 1;
        const uint32_t use = (uint32_t)(local >> 1);
        if (!wait(&sm->tmem_empty[b], (use & 1u) ^ 1u, 2u)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * 256);
        const int n_pairs = (m.n_full + 1) / 2;
        const bool kt = kt_on(m);
        const int steps = kt ? n_pairs : m.n_steps;
        for (int kb = 0; kb < steps; ++kb, ++it) {
          if (!advance(false)) {
            ok = false;
            break;
          }
          const int st = (int)(it % (uint32_t)a.stages);
          const uint32_t ph = (it / (uint32_t)a.stages) & 1u;
          if (!wait(&sm->full[st], ph, 2u)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_addr = smem_u32(stage_a + (size_t)st * kStageA);
          const uint32_t b_addr = smem_u32(stage_b + (size_t)st * kStageB);
          // MMAs of this step: four per full atom (two atoms, or one if n_full is odd and this is its
          // last pair), k_last for the partial atom
          const int atoms = kb < n_pairs ? (2 * kb + 1 < m.n_full ? 2 : 1) : 1;
#pragma unroll
          for (int at = 0; at < 2; ++at) {
            if (at >= atoms) break;
            const int nk = kb < n_pairs ? kRowB / kMmaKB : m.k_last;
            const uint32_t aa = a_addr + (uint32_t)at * kAtomA, bb = b_addr + (uint32_t)at * kAtomB;
#pragma unroll
            for (int k = 0; k < kRowB / kMmaKB; ++k) {
              if (k >= nk) break;
              const uint32_t acc = (kb > 0 || at > 0 || k > 0) ? 1u : 0u;
              if (F8)
                mma2_e4m3(d_tmem, smem_desc(aa + k * kMmaKB), smem_desc(bb + k * kMmaKB), idesc1, acc);
              else
                mma2_bf16(d_tmem, smem_desc(aa + k * kMmaKB), smem_desc(bb + k * kMmaKB), idesc1, acc);
            }
          }
          commit_both(&sm->empty[st]);
        }
        if (!ok) break;
        if (kt) {
          // the partial last atom from its K-tail buffer, after every full atom (the same K order as a stage
          // of its own)
          const int kbuf = kt_n & 1;
          if (!wait(&sm->kt_full[kbuf], (uint32_t)(kt_n >> 1) & 1u, 2u)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int k = 0; k < m.kt; ++k) {
            const uint64_t da = smem_desc_sw32(smem_u32(kt_a(kbuf, k)));
            const uint64_t db = smem_desc_sw32(smem_u32(kt_b(kbuf, k)));
            if (F8)
              mma2_e4m3(d_tmem, da, db, idesc1, 1u);
            else
              mma2_bf16(d_tmem, da, db, idesc1, 1u);
          }
          commit_both(&sm->kt_empty[kbuf]);
          ++kt_n;
        }
        commit_both(&sm->tmem_full[b]);
        if (!advance(true)) {
          ok = false;
          break;
        }
        pend = local;
        pend_layer = 2;
        pend_sv = min(S, m.count - (lt / m.m_pairs) * S);
      }
      if (ok) advance(true);
      // every issued MMA completes before TMEM is released: one more commit, bounded wait
      mma2_commit(map_to(&sm->mma_done, 0u));
      mbar_drain(&sm->mma_done, 0u, a.status);
    }
  } else {
    // ---------------- epilogue (both CTAs) ----------------
    const int ew = warp - 2;            // 0 .. kEpi-1
    const int quad = warp & 3;          // TMEM lane quadrant this warp may access
    const int grp = ew >> 2;            // the tile's spark this warp takes (none when grp >= S)
    const int et = threadIdx.x - 64;    // 0 .. 32 kEpi - 1
    const int row_in_tile = quad * 32 + lane;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
    // Tiles are pipelined by one: a tile's logits are read into registers and its TMEM half handed back
    // at once, and its loss is taken during the next tile, between packing that tile's activations and
    // waiting for its logits, so the loss math overlaps the MMAs of the next tile's later layers.
    float zp[NL];
    struct Prev {
      bool on;
      bool valid_row;
      int label, cur, mt, s0, s_valid, tb;
    } prev = {false, false, 0, 0, 0, 0, 0, 0};
    // the loss of the tile in `prev` (its logits in zp): per-sample CE, the warp's sum per spark, the
    // tile's partial sums
    auto finish = [&]() {
      const PairArgs& m = args_of(prev.cur);
      const float* tail = tails + (size_t)prev.tb * S * kTailF;
      if (grp < prev.s_valid) {
        const int s = grp;
        const float* bl = tail + (size_t)s * kTailF + H1 + H2;
        float ce = 0.0f;
        if (prev.valid_row) {
          const int C = m.C;
          float zmax = -INFINITY;
          float zy = 0.0f;
#pragma unroll
          for (int c = 0; c < NL; ++c) {
            if (c < C) {
              zp[c] += bl[c];
              zmax = fmaxf(zmax, zp[c]);
              if (c == prev.label) zy = zp[c];
            }
          }
          // the fast exponential and logarithm (a few units in the last place: far inside the BF16 / E4M3
          // operands' error)
          float se = 0.0f;
#pragma unroll
          for (int c = 0; c < NL; ++c)
            if (c < C) se += __expf(zp[c] - zmax);
          ce = (zmax + __logf(se)) - zy;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ce += __shfl_xor_sync(0xffffffffu, ce, off);
        if (lane == 0) red[s * 4 + quad] = ce;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm->tail_empty[prev.tb]);
      epi_bar<kEpi>();
      const int m128 = prev.mt * 2 + (int)rank;
      if (et < prev.s_valid && m128 < m.m_tiles) {
        const int s = et;
        const float v = ((red[s * 4 + 0] + red[s * 4 + 1]) + red[s * 4 + 2]) + red[s * 4 + 3];
        m.partial[(int64_t)m128 * m.count + prev.s0 + s] = v;
      }
      prev.on = false;
    };
    int local = 0;
    int cur = 0;
    bool aborted = false;
    for (int t = pair; t < tiles; t += npairs, ++local) {
      const int lt = member_at(t, cur);
      const PairArgs& m = args_of(cur);
      const int mt = lt % m.m_pairs, nt = lt / m.m_pairs;
      const int b = local & 1;
      const uint32_t use = (uint32_t)(local >> 1);
      const int s0 = nt * S;
      const int s_valid = min(S, m.count - s0);
      const int64_t n = (int64_t)mt * (2 * kPM) + (int64_t)rank * kPM + row_in_tile;
      const bool valid_row = n < m.N;
      const int label = valid_row ? m.y[n] : 0;  // issued before the waits
      const int tb = local % kTBufs;
      bool ok = wait(&sm->tmem_full[b], use & 1u, 4u);
      ok = ok && wait(&sm->bias_full[tb], (uint32_t)(local / kTBufs) & 1u, 4u);
      if (epi_bar_any<kEpi>(!ok || sm->abort_flag)) {
        aborted = true;
        break;
      }
      tc_fence_after();
      const float* tail = tails + (size_t)tb * S * kTailF;
      const uint32_t hbase = lane_base + (uint32_t)(b * 256);
      // act(h * scale + b1) as packed BF16 into the spark's first h1/2 columns: layer 2's A operand
      if (grp < s_valid)
        pack_layer<H1>(hbase + col_h(grp), hbase + col_h(grp), tail + (size_t)grp * kTailF, m.scale, m.act);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(map_to(&sm->a2_full[b], 0u));
      if (prev.on) finish();
      ok = wait(&sm->l2_full[b], use & 1u, 4u);
      if constexpr (kL3) {
        // act(layer 2 + b2) packed in place: layer 3's A operand
        if (epi_bar_any<kEpi>(!ok || sm->abort_flag)) {
          aborted = true;
          break;
        }
        tc_fence_after();
        if (grp < s_valid)
          pack_layer<H2>(hbase + col_l2(grp), hbase + col_l2(grp), tail + (size_t)grp * kTailF + H1, 1.0f, m.act2);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(map_to(&sm->a3_full[b], 0u));
        ok = wait(&sm->l3_full[b], use & 1u, 4u);
      }
      if (epi_bar_any<kEpi>(!ok || sm->abort_flag)) {
        aborted = true;
        break;
      }
      tc_fence_after();
      // read this warp's logits, then give their columns back; the loss follows during the next tile
      if (grp < s_valid) {
#pragma unroll
        for (int q = 0; q < NL; q += 16) tmem_ld16(hbase + col_lg(grp) + (uint32_t)q, zp + q);
      }
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(map_to(kShared ? &sm->tmem_empty[b] : &sm->l2_empty[b], 0u));
      prev = {true, valid_row, label, cur, mt, s0, s_valid, tb};
    }
    if (!aborted && prev.on) finish();
  }

  if (sm->abort_flag) {
    // aborting: the odd CTA's last copies complete on the even CTA's barriers, which it cannot watch,
    // so let any copy in flight land (a bounded pause, far above a copy's latency) before leaving
    const long long t0 = clock64();
    while ((uint64_t)(clock64() - t0) < (1ull << 24)) {
    }
  }
  tc_fence_before();
  cluster_sync();  // the pair's MMAs are done and no cross-CTA access is pending
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(kCols) : "memory");
  }
}

template <int H1, int H2, int NL, int S, bool F8>
cudaError_t launch_pair(const TcPlan& plan, const PairArgs& args, cudaStream_t s, bool prepare_only, int* pairs_out,
                        const PairMember* members, int32_t n_members, int32_t group_tiles) {
  cudaError_t e = ensure_smem_limit<k_fitness_pair<H1, H2, NL, S, F8, false>>(plan.smem_bytes);
  if (e != cudaSuccess) return e;
  e = ensure_smem_limit<k_fitness_pair<H1, H2, NL, S, F8, true>>(plan.smem_bytes);
  if (e != cudaSuccess) return e;
  if (prepare_only) {
    // pairs that fit at once (one CTA per SM): the persistent grid
    if (pairs_out) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2 * (plan.num_sms / 2));
      cfg.blockDim = dim3(pair_threads(S));
      cfg.dynamicSmemBytes = plan.smem_bytes;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_fitness_pair<H1, H2, NL, S, F8, false>, &cfg) != cudaSuccess ||
          n < 1) {
        cudaGetLastError();
        n = plan.num_sms / 2;
      }
      *pairs_out = n;
    }
    return cudaSuccess;
  }
  if (members) {
    const int pairs = group_tiles < plan.pairs ? group_tiles : plan.pairs;
    return launch_pdl(k_fitness_pair<H1, H2, NL, S, F8, true>, dim3(2 * pairs), dim3(pair_threads(S)),
                      plan.smem_bytes, s, plan.tmap_x3, plan.tmap_x, plan.tmap_wk, plan.tmap_w, plan.tmap_w2b,
                      plan.tmap_w3b, plan.tmap_xt, plan.tmap_wt, args, members, n_members);
  }
  const int tiles = args.m_pairs * args.n_tiles;
  const int pairs = tiles < plan.pairs ? tiles : plan.pairs;
  return launch_pdl(k_fitness_pair<H1, H2, NL, S, F8, false>, dim3(2 * pairs), dim3(pair_threads(S)),
                    plan.smem_bytes, s, plan.tmap_x3, plan.tmap_x, plan.tmap_wk, plan.tmap_w, plan.tmap_w2b,
                    plan.tmap_w3b, plan.tmap_xt, plan.tmap_wt, args, static_cast<const PairMember*>(nullptr), 0);
}

// The kernel instance of the plan: h1 (and h2), the logit rows, the tile shape (shared or separate logits)
// and the operand type.
cudaError_t dispatch_pair(const TcPlan& plan, const Mlp& mlp, const PairArgs& a, cudaStream_t s, bool prep,
                          int* pairs_out, const PairMember* members = nullptr, int32_t n_members = 0,
                          int32_t group_tiles = 0) {
  const int h1 = mlp.widths[1], h2 = mlp.n_layers == 3 ? mlp.widths[2] : 0;
  const int nl = tc_pair_logit_rows(mlp.widths[mlp.n_layers]);
  if (h2 > 0) {
    if (h1 != 128 || h2 != 64 || nl != 16 || plan.sparks_per_tile != pair_sparks_shared(128))
      return cudaErrorInvalidValue;
    return plan.f8 ? launch_pair<128, 64, 16, 2, true>(plan, a, s, prep, pairs_out, members, n_members, group_tiles)
                   : launch_pair<128, 64, 16, 2, false>(plan, a, s, prep, pairs_out, members, n_members, group_tiles);
  }
  const bool shared = plan.sparks_per_tile == pair_sparks_shared(h1);
  if (!shared && plan.sparks_per_tile != pair_sparks_separate(h1, nl)) return cudaErrorInvalidValue;
  const int key = h1 * 8 + (nl == 32 ? 4 : 0) + (shared ? 2 : 0) + (plan.f8 ? 1 : 0);
#define MG_PAIR(H, L, SH, F)                                                                                    \
  launch_pair<H, 0, L, SH ? pair_sparks_shared(H) : pair_sparks_separate(H, L), F>(plan, a, s, prep, pairs_out, \
                                                                                    members, n_members, group_tiles)
#define MG_PAIR_CASES(H, L, NLK)                                   \
  case H * 8 + NLK + 0: return MG_PAIR(H, L, false, false);        \
  case H * 8 + NLK + 1: return MG_PAIR(H, L, false, true);         \
  case H * 8 + NLK + 2: return MG_PAIR(H, L, true, false);         \
  case H * 8 + NLK + 3: return MG_PAIR(H, L, true, true);
  switch (key) {
    MG_PAIR_CASES(64, 16, 0)
    MG_PAIR_CASES(64, 32, 4)
    MG_PAIR_CASES(128, 16, 0)
    MG_PAIR_CASES(128, 32, 4)
    default: return cudaErrorInvalidValue;
  }
#undef MG_PAIR_CASES
#undef MG_PAIR
}

// The arguments of one launch of `count` rows from `first` (as launch_fitness_tc makes them).
PairArgs make_args(const TcPlan& plan, const Mlp& mlp, int64_t first, const float* rows, int64_t ld, int32_t count,
                   float scale, float* partial, uint32_t* status) {
  PairArgs a = {};
  const int S = plan.sparks_per_tile;
  const bool l3 = mlp.n_layers == 3;
  a.count = count;
  a.first_spark = (int32_t)first;
  a.m_pairs = (int32_t)((mlp.N + 2 * kPM - 1) / (2 * kPM));
  a.m_tiles = (int32_t)((mlp.N + kPM - 1) / kPM);
  a.n_tiles = (count + S - 1) / S;
  const int bk = plan.f8 ? 128 : 64;
  {
    const int ke = plan.f8 ? 32 : 16;                 // K elements per MMA
    a.n_full = mlp.widths[0] / bk;
    const int rem = mlp.widths[0] - a.n_full * bk;   // K elements of the partial last atom
    a.k_last = (rem + ke - 1) / ke;
    a.n_steps = (a.n_full + 1) / 2 + (rem > 0 ? 1 : 0);
    a.kt = tc_pair_ktail_mmas(mlp, plan.f8);
    a.kt_region = plan.ktail;
  }
  a.stages = plan.stages;
  a.C = mlp.widths[mlp.n_layers];
  a.act = mlp.acts[0];
  a.act2 = l3 ? mlp.acts[1] : 0;
  a.c_pad = (a.C + 3) / 4 * 4;
  a.scale = scale;
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
  return a;
}

}  // namespace

bool tc_pair_supported(const int32_t* widths, int n_layers) {
  if (widths[0] % 8 != 0) return false;
  if (n_layers == 2) return (widths[1] == 64 || widths[1] == 128) && widths[2] >= 2 && widths[2] <= 32;
  return n_layers == 3 && widths[1] == 128 && widths[2] == 64 && widths[3] >= 2 && widths[3] <= 16;
}

int tc_pair_logit_rows(int C) { return C <= 16 ? 16 : 32; }

int tc_pair_w2_rows(const int32_t* widths, int n_layers) {
  return n_layers == 3 ? widths[2] : tc_pair_logit_rows(widths[2]);
}

int tc_pair_sparks(const Mlp& mlp, bool shared) {
  const int h1 = mlp.widths[1];
  if (mlp.n_layers == 3) return shared ? pair_sparks_shared(h1) : 0;
  return shared ? pair_sparks_shared(h1) : pair_sparks_separate(h1, tc_pair_logit_rows(mlp.widths[2]));
}

size_t tc_pair_fixed_smem(const Mlp& mlp, int S) {
  const int h1 = mlp.widths[1], h2 = mlp.n_layers == 3 ? mlp.widths[2] : 0;
  const int nl = tc_pair_logit_rows(mlp.widths[mlp.n_layers]);
  // W2 (and W3) halves of every spark of a tile, per buffer (three buffers for two layers, one for three)
  const size_t w_spark = h2 > 0 ? (size_t)(h1 / 64) * (h2 / 2) * 128 + (size_t)(h2 / 64) * (nl / 2) * 128
                                : (size_t)(h1 / 64) * (nl / 2) * 128;
  const size_t w2 = (size_t)(h2 > 0 ? 1 : kTBufs) * S * w_spark;
  const size_t tails = sizeof(float) * ((size_t)kTBufs * S * (h1 + h2 + 32) + 4 * (size_t)S);
  return 1024 + w2 + tails + 16 + sizeof(PairSmem) + 64;
}

size_t tc_pair_stage_bytes(int h1, int S) { return 2 * ((size_t)kPM * kRowB + (size_t)(S * h1 / 2) * kRowB); }

int tc_pair_ktail_mmas(const Mlp& mlp, bool f8) {
  const int bk = f8 ? 128 : 64, ke = f8 ? 32 : 16;  // K elements per atom and per MMA
  const int d_in = mlp.widths[0], rem = d_in % bk;
  const int k = (rem + ke - 1) / ke;
  return d_in >= bk && k >= 1 && k <= kMaxKt ? k : 0;
}

size_t tc_pair_ktail_bytes(int h1, int S, int mmas) {
  return 2 * (size_t)mmas * kKtBox * ((size_t)kPM + (size_t)(S * h1 / 2));
}

int tc_pair_max_stages() { return kMaxStg; }

int tc_pair_stages_fit(const Mlp& mlp, int S, size_t limit, int kt_mmas) {
  const size_t fixed = tc_pair_fixed_smem(mlp, S) + tc_pair_ktail_bytes(mlp.widths[1], S, kt_mmas),
               stage = tc_pair_stage_bytes(mlp.widths[1], S);
  int st = kMaxStg;
  while (st >= 2 && fixed + (size_t)st * stage > limit) --st;
  return st >= 2 ? st : 0;
}

int launch_fitness_pair(const TcPlan& plan, const Mlp& mlp, int64_t first, const float* rows, int64_t ld,
                        int32_t count, float scale, float* partial, uint32_t* status, cudaStream_t s) {
  const PairArgs a = make_args(plan, mlp, first, rows, ld, count, scale, partial, status);
  return dispatch_pair(plan, mlp, a, s, false, nullptr) == cudaSuccess ? 1 : -1;
}

void tc_pair_member(const TcPlan& plan, const Mlp& mlp, int64_t first, const float* rows, int64_t ld, int32_t count,
                    float scale, float* partial, uint32_t* status, PairMember* out) {
  out->x3 = plan.tmap_x3;
  out->x = plan.tmap_x;
  out->w3 = plan.tmap_wk;
  out->w = plan.tmap_w;
  out->w2 = plan.tmap_w2b;
  out->wl3 = plan.tmap_w3b;
  out->xt = plan.tmap_xt;
  out->wt = plan.tmap_wt;
  out->a = make_args(plan, mlp, first, rows, ld, count, scale, partial, status);
  out->tiles = out->a.m_pairs * out->a.n_tiles;
  out->tile_start = 0;
}

bool tc_pair_same_instance(const TcPlan& a, const Mlp& ma, const TcPlan& b, const Mlp& mb) {
  if (ma.n_layers != mb.n_layers || (ma.n_layers == 3 && ma.widths[2] != mb.widths[2])) return false;
  return a.ready && b.ready && a.pair && b.pair && a.f8 == b.f8 && ma.widths[1] == mb.widths[1] &&
         tc_pair_logit_rows(ma.widths[ma.n_layers]) == tc_pair_logit_rows(mb.widths[mb.n_layers]) &&
         a.sparks_per_tile == b.sparks_per_tile;
}

int launch_fitness_pair_group(const TcPlan& plan, const Mlp& mlp, const PairMember* table_dev, int32_t n,
                              uint32_t* status, cudaStream_t s, int32_t total_tiles) {
  if (n < 1 || total_tiles < 1) return 0;
  PairArgs a = {};
  a.stages = plan.stages;
  a.kt_region = plan.ktail;  // the shared-memory layout of the launch; a member with more K-tail MMAs takes
                             // its partial atom as a stage
  a.status = status;
  a.wait_budget = plan.wait_budget;
  return dispatch_pair(plan, mlp, a, s, false, nullptr, table_dev, n, total_tiles) == cudaSuccess
             ? 1
             : -1;
}

cudaError_t tc_pair_prepare(TcPlan& plan, const Mlp& mlp) {
  PairArgs a = {};
  int pairs = 0;
  cudaError_t e = dispatch_pair(plan, mlp, a, nullptr, true, &pairs);
  if (e == cudaSuccess) plan.pairs = pairs;
  return e;
}

}  // namespace mgfwa
