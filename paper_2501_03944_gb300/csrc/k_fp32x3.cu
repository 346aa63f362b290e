// FP32-accurate first layer on the tensor cores, for a few search vectors
// at once: act(X W1^T + b1) of R vectors (rows of the spark buffer, picked
// by an index) over the whole batch, written to [R][N][H] for the FP32
// output-layer kernel.  Used where FP32 accuracy is required (the elite
// re-score, the refinement's forward pass).
//
// Each FP32 operand v is split into three BF16 parts, each rounded to
// nearest: v1 = bf16(v), v2 = bf16(v - v1), v3 = bf16(v - v1 - v2) (the
// differences are exact in FP32; |v2| <= 2^-9 |v|, |v3| <= 2^-18 |v|, and
// v - v1 - v2 - v3 <= 2^-27 |v|).  Six tcgen05 kind::f16 MMAs (BF16 in,
// FP32 accumulate, K = 16) per K step accumulate a1b1 + a1b2 + a2b1 + a2b2
// + a1b3 + a3b1: the products of 8-bit significands are exact in FP32, and
// the dropped terms (a2b3, a3b2, a3b3 and the residuals) are below about
// 2^-25 of each product, under FP32's own rounding.  The tensor core's own
// accumulation rounds at every step, so the main products a1b1 go to two
// accumulators (even and odd K blocks) and the five corrections (about 2^-8
// of them) to a third; the epilogue adds the three in FP32.  That keeps the
// result within FP32 accuracy for K in the thousands.
//
// The parts are made once per operand by k_split_bf16x3 (X at create, the
// vectors' W1 blocks before each launch), so the layer itself is a plain
// TMA -> MMA pipeline.  One CTA per 128-sample tile and 128 / h1 vectors.
// Warp 0 issues TMA: per stage of 32 K-elements, the three X part tiles
// [128 samples x 32] and the three W1 part tiles [128 rows x 32] (64-byte
// rows, 64-byte swizzle).  Warp 1 issues the MMAs, both operands from shared
// memory.  Warps 2..5 read the accumulators (one sample row per thread),
// add b1, apply the activation and store the row, or run the fused output
// layer.  Every wait is bounded; a wait that gives up sets a bit in the
// status word and the CTA drains its copies and MMAs and returns.
#include <cuda.h>

#include "fp32x3.cuh"
#include "mgfwa_internal.cuh"

namespace mgfwa {
namespace {

constexpr int kBM = 128;
constexpr int kBKf = 32;           // FP32 K elements per stage (128 bytes)
constexpr int kMaxStages = 6;
constexpr int kParts = 3;          // BF16 parts per operand
constexpr int kThreads = 192;      // warp 0 TMA, warp 1 MMA, warps 2..5 convert + epilogue
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitBudget = 1ull << 32;

struct Bars {
  uint64_t full[kMaxStages];   // stage landed (TMA)
  uint64_t empty[kMaxStages];  // stage free (its MMAs completed)
  uint64_t done;
  uint32_t tmem_base;
  volatile int abort_flag;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false once this CTA aborts.
__device__ __forceinline__ bool mbar_wait(Bars* sb, uint64_t* b, uint32_t parity, uint32_t* status, uint32_t code) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, parity)) {
    if (sb->abort_flag) return false;
    if ((uint64_t)(clock64() - t0) > kWaitBudget) {
      sb->abort_flag = 1;
      atomicOr(status, code);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void mbar_drain(uint64_t* b, uint32_t parity, uint32_t* status) {
  const long long t0 = clock64();
  while (!mbar_try(b, parity)) {
    if ((uint64_t)(clock64() - t0) > kWaitBudget) {
      atomicOr(status, 16u);
      return;
    }
  }
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* m, int x, int y, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(b))
      : "memory");
}
__device__ __forceinline__ void tma_3d(void* dst, const CUtensorMap* m, int x, int y, int z, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(b))
      : "memory");
}
// Shared-memory matrix descriptor of a K-major BF16 operand in 64-byte
// swizzled rows (32 K-elements per row), 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;          // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                   // descriptor version for tcgen05
  d |= (uint64_t)4 << 61;                   // 64-byte swizzle
  return d;
}
// kind::f16 with BF16 A and B, FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// D (TMEM) (+)= A x B, both from shared memory, BF16 inputs.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Two consecutive K elements (a, b) -> their three BF16 parts, each packed
// with a in the low half (the lower K index first): v1 = bf16(v), v2 =
// bf16(v - v1), v3 = bf16(v - v1 - v2), round to nearest.
__device__ __forceinline__ void split2(float a, float b, uint32_t& p1, uint32_t& p2, uint32_t& p3) {
  const __nv_bfloat162 h1 = __floats2bfloat162_rn(a, b);
  const float ra = __fsub_rn(a, __low2float(h1)), rb = __fsub_rn(b, __high2float(h1));
  const __nv_bfloat162 h2 = __floats2bfloat162_rn(ra, rb);
  const __nv_bfloat162 h3 = __floats2bfloat162_rn(__fsub_rn(ra, __low2float(h2)), __fsub_rn(rb, __high2float(h2)));
  p1 = *reinterpret_cast<const uint32_t*>(&h1);
  p2 = *reinterpret_cast<const uint32_t*>(&h2);
  p3 = *reinterpret_cast<const uint32_t*>(&h3);
}

}  // namespace

// Part p of element pair e (elements 2e, 2e + 1) of source row r -- row
// idx[r] (or r) of src, elements from `off` -- goes to word
// dst[r * rstride + p * pstride + e], two BF16 per word.
__global__ void __launch_bounds__(256) k_split_bf16x3(const float* __restrict__ src, int64_t ld,
                                                      const int32_t* __restrict__ idx, int32_t rows, int64_t off,
                                                      int64_t pairs, uint32_t* __restrict__ dst, int64_t rstride,
                                                      int64_t pstride) {
  griddep_wait();
  griddep_launch_dependents();
  const int64_t total = (int64_t)rows * pairs;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / pairs, e = t - r * pairs;
    const float2 v =
        *reinterpret_cast<const float2*>(src + (int64_t)(idx ? idx[r] : r) * ld + off + 2 * e);
    uint32_t p1, p2, p3;
    split2(v.x, v.y, p1, p2, p3);
    uint32_t* d = dst + r * rstride + e;
    d[0] = p1;
    d[pstride] = p2;
    d[2 * pstride] = p3;
  }
}

namespace {

struct Args {
  int32_t N;        // samples
  int32_t d_in;
  int32_t k_blocks;
  int32_t act;
  int64_t ld;       // FP32 row stride of the spark buffer
  int64_t b1_off;   // offset of b1 in a row
  const float* rows;
  const int32_t* idx;  // vector r is spark row idx[r] (or r)
  int32_t R;        // vectors
  float* out;       // [R][N][H] (unless the output layer is fused)
  uint32_t* status;
  // fused output layer (two-layer nets, objective only): loss[r][n] from the
  // logits W2 a + b2 of the vector's row, instead of the activations
  float* loss;      // [R][N], or null
  int64_t w2_off, b2_off;
  int32_t C;
  const int32_t* y;
};

// Each CTA takes V = 128 / H vectors, so that every MMA is M=128, N=128:
// the tensor core's cost per instruction barely depends on N at these
// widths, so fewer, wider products are the faster way through the six.
// Shared memory per stage: the three X part tiles and the three part tiles
// of the V stacked W1 blocks, 128 rows x 64 bytes each.  TMEM: the
// accumulators (main even, main odd, corrections: 3 x 128 columns).
constexpr int kN = 128;
constexpr int kMaxC = 32;           // classes of a fused output layer
constexpr int kStages = 4;
constexpr uint32_t kPartBytes = 128 * 64;  // one part tile of a stage (X or W1)
constexpr uint32_t kStageBytes = 2 * kParts * kPartBytes;
static_assert(3 * kN <= kTmemCols, "accumulators fit in TMEM");
static_assert(kStages <= kMaxStages, "barrier arrays");

// NL: register slots for the logits of a fused output layer (C <= NL).
template <int H, int NL>
__global__ void __launch_bounds__(kThreads, 1)
    k_l1_fp32x3(const __grid_constant__ CUtensorMap tmap_xs, const __grid_constant__ CUtensorMap tmap_ws, Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  constexpr int V = kN / H;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // part p of stage s: X at base + (s * 2 + 0) * 3 parts, W1 at (s * 2 + 1) * 3 parts
  auto Xp = [&](int p, int s) { return base + ((size_t)s * 2 * kParts + p) * kPartBytes; };
  auto Wp = [&](int p, int s) { return base + ((size_t)s * 2 * kParts + kParts + p) * kPartBytes; };
  Bars* sb = reinterpret_cast<Bars*>(base + (size_t)kStages * kStageBytes);
  float* w2s = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(sb) + ((sizeof(Bars) + 15) & ~size_t(15)));
  float* b2s = w2s + (size_t)V * kMaxC * H;  // fused output layer: W2 [V][C][H], b2 [V][C] of the CTA's vectors

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x, r0 = blockIdx.y * V;
  // vector v of this CTA: r0 + v, or (past the last vector) the last one again, computed and not stored
  auto vec_of = [&](int v) { return r0 + v < a.R ? r0 + v : a.R - 1; };
  auto row_of = [&](int v) { return a.idx ? a.idx[vec_of(v)] : vec_of(v); };
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sb->full[s], 1);
      mbar_init(&sb->empty[s], 1);
    }
    mbar_init(&sb->done, 1);
    sb->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sb->tmem_base)),
                 "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sb->tmem_base;
  // the set-up above touches nothing the previous kernel writes, so it overlaps that kernel's tail
  griddep_wait();
  griddep_launch_dependents();

  if (warp == 0) {
    if (lane == 0) {
      int vz[V];
#pragma unroll
      for (int v = 0; v < V; ++v) vz[v] = vec_of(v) * kParts;  // the vector's first part in the W1 part buffer
      int kb = 0;
      for (; kb < a.k_blocks; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        if (!mbar_wait(sb, &sb->empty[s], ph ^ 1u, a.status, 1u)) break;
        mbar_expect_tx(&sb->full[s], kStageBytes);
#pragma unroll
        for (int p = 0; p < kParts; ++p) {
          tma_3d(Xp(p, s), &tmap_xs, kb * kBKf, mt * kBM, p, &sb->full[s]);
#pragma unroll
          for (int v = 0; v < V; ++v)
            tma_3d(Wp(p, s) + (size_t)v * H * 64, &tmap_ws, kb * kBKf, 0, vz[v] + p, &sb->full[s]);
        }
      }
      // every issued copy lands before the CTA may exit
      for (int j = kb - kStages > 0 ? kb - kStages : 0; j < kb; ++j)
        mbar_drain(&sb->full[j % kStages], (uint32_t)(j / kStages) & 1u, a.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, kN);
      int kb = 0;
      for (; kb < a.k_blocks; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        if (!mbar_wait(sb, &sb->full[s], ph, a.status, 2u)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t x1 = smem_u32(Xp(0, s)), x2 = smem_u32(Xp(1, s)), x3 = smem_u32(Xp(2, s));
        const uint32_t w1 = smem_u32(Wp(0, s)), w2 = smem_u32(Wp(1, s)), w3 = smem_u32(Wp(2, s));
        const uint32_t d_main = tmem + (uint32_t)((kb & 1) * kN), d_corr = tmem + (uint32_t)(2 * kN);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t o = (uint32_t)j * 32u;  // byte offset of this K step (16 BF16) in a 64-byte row
          const uint32_t first = (kb < 2 && j == 0) ? 0u : 1u;     // this main accumulator's first product
          const uint32_t first_c = (kb == 0 && j == 0) ? 0u : 1u;  // the corrections' first
          mma_bf16(d_main, smem_desc_sw64(x1 + o), smem_desc_sw64(w1 + o), idesc, first);
          mma_bf16(d_corr, smem_desc_sw64(x1 + o), smem_desc_sw64(w2 + o), idesc, first_c);
          mma_bf16(d_corr, smem_desc_sw64(x2 + o), smem_desc_sw64(w1 + o), idesc, 1u);
          mma_bf16(d_corr, smem_desc_sw64(x2 + o), smem_desc_sw64(w2 + o), idesc, 1u);
          mma_bf16(d_corr, smem_desc_sw64(x1 + o), smem_desc_sw64(w3 + o), idesc, 1u);
          mma_bf16(d_corr, smem_desc_sw64(x3 + o), smem_desc_sw64(w1 + o), idesc, 1u);
        }
        mma_commit(&sb->empty[s]);
      }
      mma_commit(&sb->done);  // after every issued MMA (also on abort)
    }
  } else {
    const int ct = threadIdx.x - 64;   // 0..127
    const int q = warp & 3;            // TMEM lane quadrant this warp may access
    const int rrow = q * 32 + lane;    // this thread's sample row of the tile = its TMEM lane
    const uint32_t lanes = tmem + ((uint32_t)(q * 32) << 16);
    const bool fused = a.loss != nullptr;
    if (fused) {
      // W2 and b2 of the CTA's vectors, read by the epilogue below (ordered by the named barrier there)
      for (int e = ct; e < V * a.C * H; e += 128) {
        const int v = e / (a.C * H), rem = e - v * (a.C * H);
        w2s[e] = a.rows[(int64_t)row_of(v) * a.ld + a.w2_off + rem];
      }
      for (int e = ct; e < V * a.C; e += 128) {
        const int v = e / a.C;
        b2s[e] = a.rows[(int64_t)row_of(v) * a.ld + a.b2_off + (e - v * a.C)];
      }
    }
    // epilogue: row = this thread's TMEM lane; columns [v H, (v + 1) H) are vector r0 + v
    mbar_drain(&sb->done, 0u, a.status);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int64_t n = (int64_t)mt * kBM + rrow;
    const bool valid = !sb->abort_flag && n < a.N;
    const bool odd = a.k_blocks > 1;  // the odd-block accumulator holds products
    if (fused) {
      asm volatile("bar.sync 1, 128;" ::: "memory");  // W2, b2 staged by all four warps
      const int yn = valid ? a.y[n] : 0;
#pragma unroll 1
      for (int v = 0; v < V; ++v) {
        const float* bias = a.rows + (int64_t)row_of(v) * a.ld + a.b1_off;
        const float* w2 = w2s + (size_t)v * a.C * H;
        // logits in the order of the CUDA-core output layer: z_c = b2_c, then fma over j ascending
        float z[NL];
#pragma unroll
        for (int c = 0; c < NL; ++c) z[c] = c < a.C ? b2s[v * a.C + c] : 0.f;
        // 8 hidden units at a time; the next 8 are loaded from TMEM while these are used
        float x[8], x1[8], xc[8], nx[8], nx1[8], nxc[8];
        {
          const uint32_t col = (uint32_t)(v * H);
          tmem_ld8(lanes + col, x);
          tmem_ld8(lanes + (uint32_t)kN + col, x1);
          tmem_ld8(lanes + (uint32_t)(2 * kN) + col, xc);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
#pragma unroll 1
        for (int j0 = 0; j0 < H; j0 += 8) {
          const bool more = j0 + 8 < H;
          if (more) {
            const uint32_t col = (uint32_t)(v * H + j0 + 8);
            tmem_ld8(lanes + col, nx);
            tmem_ld8(lanes + (uint32_t)kN + col, nx1);
            tmem_ld8(lanes + (uint32_t)(2 * kN) + col, nxc);
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float zz = ((odd ? x[i] + x1[i] : x[i]) + xc[i]) + bias[j0 + i];
            x[i] = a.act == kActTanh ? tanhf(zz) : fmaxf(zz, 0.f);
          }
#pragma unroll
          for (int c = 0; c < NL; ++c) {
            if (c < a.C) {
              const float4 w0 = *reinterpret_cast<const float4*>(w2 + (size_t)c * H + j0);
              const float4 w1 = *reinterpret_cast<const float4*>(w2 + (size_t)c * H + j0 + 4);
              z[c] = fmaf(x[0], w0.x, z[c]);
              z[c] = fmaf(x[1], w0.y, z[c]);
              z[c] = fmaf(x[2], w0.z, z[c]);
              z[c] = fmaf(x[3], w0.w, z[c]);
              z[c] = fmaf(x[4], w1.x, z[c]);
              z[c] = fmaf(x[5], w1.y, z[c]);
              z[c] = fmaf(x[6], w1.z, z[c]);
              z[c] = fmaf(x[7], w1.w, z[c]);
            }
          }
          if (more) {
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              x[i] = nx[i];
              x1[i] = nx1[i];
              xc[i] = nxc[i];
            }
          }
        }
        if (valid && r0 + v < a.R) {
          float zmax = z[0];
#pragma unroll
          for (int c = 1; c < NL; ++c)
            if (c < a.C) zmax = fmaxf(zmax, z[c]);
          float se = 0.f, zy = 0.f;
#pragma unroll
          for (int c = 0; c < NL; ++c) {
            if (c < a.C) {
              se += expf(z[c] - zmax);
              if (c == yn) zy = z[c];
            }
          }
          a.loss[(int64_t)(r0 + v) * a.N + n] = (zmax + logf(se)) - zy;
        }
      }
    }
#pragma unroll 1
    for (int v = 0; v < (fused ? 0 : V); ++v) {
      const bool store = valid && r0 + v < a.R;
      const float* bias = a.rows + (int64_t)row_of(v) * a.ld + a.b1_off;
      float* out = a.out + ((int64_t)(r0 + v) * a.N + n) * H;
#pragma unroll 1
      for (int j0 = 0; j0 < H; j0 += 8) {
        const uint32_t c = (uint32_t)(v * H + j0);
        float x[8], x1[8], xc[8];
        tmem_ld8(lanes + c, x);
        tmem_ld8(lanes + (uint32_t)kN + c, x1);
        tmem_ld8(lanes + (uint32_t)(2 * kN) + c, xc);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = (odd ? x[i] + x1[i] : x[i]) + xc[i];
        if (store) {
          float o[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float z = x[i] + bias[j0 + i];
            o[i] = a.act == kActTanh ? tanhf(z) : fmaxf(z, 0.f);
          }
          *reinterpret_cast<float4*>(out + j0) = make_float4(o[0], o[1], o[2], o[3]);
          *reinterpret_cast<float4*>(out + j0 + 4) = make_float4(o[4], o[5], o[6], o[7]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols) : "memory");
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
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

// BF16 part tiles: 32 K-elements (64 bytes) per row, 64-byte swizzle.
bool encode_bf16(CUtensorMap* map, const void* ptr, const cuuint64_t* dims, const cuuint64_t* strides,
                 const cuuint32_t* box) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t smem_bytes() {
  return 1024 + (size_t)kStages * kStageBytes + ((sizeof(Bars) + 15) & ~size_t(15)) +
         sizeof(float) * ((size_t)kN * kMaxC + (size_t)kN / 32 * kMaxC) + 64;
}

template <int H, int NL>
cudaError_t go_nl(const L1Plan& pl, const Args& a, int R, cudaStream_t s, bool prep) {
  cudaError_t e = ensure_smem_limit<k_l1_fp32x3<H, NL>>(smem_bytes());
  if (e != cudaSuccess || prep) return e;
  constexpr int V = kN / H;
  const dim3 grid((unsigned)((a.N + kBM - 1) / kBM), (unsigned)((R + V - 1) / V));
  return launch_pdl(k_l1_fp32x3<H, NL>, grid, dim3(kThreads), smem_bytes(), s, pl.tmap_xs, pl.tmap_ws, a);
}

template <int H>
cudaError_t go(const L1Plan& pl, const Args& a, int R, cudaStream_t s, bool prep) {
  if (prep) {
    const cudaError_t e = go_nl<H, 16>(pl, a, R, s, true);
    return e != cudaSuccess ? e : go_nl<H, 32>(pl, a, R, s, true);
  }
  return a.loss && a.C > 16 ? go_nl<H, 32>(pl, a, R, s, false) : go_nl<H, 16>(pl, a, R, s, false);
}

int split_launch(const float* src, int64_t ld, const int32_t* idx, int32_t rows, int64_t off, int64_t pairs,
                 uint32_t* dst, int64_t rstride, int64_t pstride, cudaStream_t s) {
  const int64_t total = (int64_t)rows * pairs;
  const int64_t blocks = (total + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 4096 ? (blocks < 1 ? 1 : blocks) : 4096);
  return launch_pdl(k_split_bf16x3, dim3(grid), dim3(256), 0, s, src, ld, idx, rows, off, pairs, dst, rstride,
                    pstride) == cudaSuccess
             ? 1
             : -1;
}

}  // namespace

bool l1_fp32x3_supported(const Mlp& mlp) {
  const int h1 = mlp.widths[1];
  return mlp.widths[0] % 8 == 0 && (h1 == 32 || h1 == 64 || h1 == 128);
}

int64_t l1_fp32x3_x_words(const Mlp& mlp) { return 3 * mlp.N * (mlp.widths[0] / 2); }
int64_t l1_fp32x3_w_words(const Mlp& mlp, int64_t max_rows) {
  return 3 * max_rows * (int64_t)mlp.widths[1] * (mlp.widths[0] / 2);
}

bool l1_fp32x3_plan(L1Plan& pl, const Mlp& mlp, const float* rows, int64_t ld, int64_t max_rows, uint32_t* xs,
                    uint32_t* ws) {
  pl = L1Plan();
  if (!l1_fp32x3_supported(mlp) || !xs || !ws) return false;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major != 10) {
    cudaGetLastError();
    return false;
  }
  const int64_t d_in = mlp.widths[0], h1 = mlp.widths[1];
  {
    // X parts [3][N][d_in] BF16, box 32 x 128 x 1
    cuuint64_t dims[3] = {(cuuint64_t)d_in, (cuuint64_t)mlp.N, 3};
    cuuint64_t strides[2] = {(cuuint64_t)d_in * 2, (cuuint64_t)(mlp.N * d_in * 2)};
    cuuint32_t box[3] = {kBKf, kBM, 1};
    if (!encode_bf16(&pl.tmap_xs, xs, dims, strides, box)) return false;
  }
  {
    // W1 parts of the launch's vectors [max_rows][3][h1][d_in] BF16, box 32 x h1 x 1
    cuuint64_t dims[3] = {(cuuint64_t)d_in, (cuuint64_t)h1, (cuuint64_t)(3 * max_rows)};
    cuuint64_t strides[2] = {(cuuint64_t)d_in * 2, (cuuint64_t)(h1 * d_in * 2)};
    cuuint32_t box[3] = {kBKf, (cuuint32_t)h1, 1};
    if (!encode_bf16(&pl.tmap_ws, ws, dims, strides, box)) return false;
  }
  pl.rows = rows;
  pl.ld = ld;
  pl.xs = xs;
  pl.ws = ws;
  pl.max_rows = max_rows;
  pl.ready = true;
  Args a = {};
  const bool prep_ok = (h1 == 32 ? go<32>(pl, a, 0, nullptr, true)
                        : h1 == 64 ? go<64>(pl, a, 0, nullptr, true)
                                   : go<128>(pl, a, 0, nullptr, true)) == cudaSuccess;
  if (!prep_ok) {
    cudaGetLastError();
    pl.ready = false;
  }
  return pl.ready;
}

int launch_l1_split_x(const L1Plan& pl, const Mlp& mlp, cudaStream_t s) {
  if (!pl.ready) return 0;
  const int64_t pairs = mlp.widths[0] / 2;
  return split_launch(mlp.X, mlp.widths[0], nullptr, (int32_t)mlp.N, 0, pairs, pl.xs, pairs, mlp.N * pairs, s);
}

bool l1_fp32x3_fuses_output(const Mlp& mlp) { return mlp.n_layers == 2 && mlp.widths[2] <= kMaxC; }

int launch_l1_fp32x3(const L1Plan& pl, const Mlp& mlp, const int32_t* idx, int32_t R, float* out,
                     uint32_t* status, cudaStream_t s, float* loss) {
  if (!pl.ready || R <= 0) return R <= 0 ? 0 : -1;
  if (R > pl.max_rows) return -1;
  Args a;
  a.N = (int32_t)mlp.N;
  a.d_in = mlp.widths[0];
  a.k_blocks = (mlp.widths[0] + kBKf - 1) / kBKf;
  a.act = mlp.acts[0];
  a.ld = pl.ld;
  a.b1_off = mlp.b_off[0];
  a.rows = pl.rows;
  a.idx = idx;
  a.R = R;
  a.out = out;
  a.status = status;
  a.loss = nullptr;
  if (loss) {
    if (!l1_fp32x3_fuses_output(mlp)) return -1;
    a.loss = loss;
    a.w2_off = mlp.w_off[1];
    a.b2_off = mlp.b_off[1];
    a.C = mlp.widths[2];
    a.y = mlp.y;
  }
  // the launch's W1 blocks -> their BF16 parts [R][3][h1][d_in]
  const int64_t pairs = (int64_t)mlp.widths[1] * (mlp.widths[0] / 2);
  if (split_launch(pl.rows, pl.ld, idx, R, mlp.w_off[0], pairs, pl.ws, 3 * pairs, pairs, s) < 0) return -1;
  cudaError_t e;
  switch (mlp.widths[1]) {
    case 32: e = go<32>(pl, a, R, s, false); break;
    case 64: e = go<64>(pl, a, R, s, false); break;
    case 128: e = go<128>(pl, a, R, s, false); break;
    default: return -1;
  }
  return e == cudaSuccess ? 2 : -1;
}

// ---------------------------------------------------------------------------
// The testbed network's layers (the paper's Eq. 1 objective) at FP32 accuracy
// on the tensor cores: out[r][j] = act(sum_i A[r][i] W[j][i] + b[j]) for a
// layer whose input A (the sparks, or the previous layer's output) and
// weights W are both given as three BF16 parts, the same six products and
// three accumulators as above.  One CTA per 128 rows x 128 outputs x one
// K split of kNetKPer 32-element blocks (splits = ceil(fan_in / 128): a
// number fixed by the layer's fan-in alone).  With one split the epilogue
// adds the bias, applies the activation and writes the FP32 output and/or
// its three BF16 parts (the next tensor-core layer's A); with several, each
// split's CTA writes its partial sum ((even + odd) + corrections) and a
// second kernel adds the partials in split order, then the bias.  A row's
// outputs are sums over its own inputs in an order fixed by the layer's
// fan-in, so a spark's value does not depend on which rows share the
// launch.

namespace {

constexpr int kNetKPer = 4;  // 32-element K blocks per split

struct NetX3Args {
  int32_t rows;        // rows of this launch (A rows [0, rows))
  int32_t k_blocks;    // 32-element K blocks of the fan-in
  int32_t splits;      // K splits (gridDim.z); > 1: partial sums into `partial`
  float* partial;      // [splits][rows][n]
  int32_t n;           // fan-out
  int32_t act;         // activation, or < 0 for none
  const float* bias;   // [n]
  float* out;          // FP32 output [rows][ldo], or null
  int64_t ldo;
  uint32_t* parts;     // the output's BF16 parts, plane p at parts + p * plane_words, row r at + r * n / 2; or null
  int64_t plane_words;
  uint32_t* status;
};

__device__ __forceinline__ float net_act(int a, float v) {
  if (a == kActTanh) return tanhf(v);
  if (a == kActGelu) return 0.5f * v * (1.0f + erff(v * 0.70710678118654752f));
  return fmaxf(v, 0.0f);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_net_x3(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_w, NetX3Args a) {
  griddep_wait();
  griddep_launch_dependents();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  auto Ap = [&](int p, int s) { return base + ((size_t)s * 2 * kParts + p) * kPartBytes; };
  auto Wp = [&](int p, int s) { return base + ((size_t)s * 2 * kParts + kParts + p) * kPartBytes; };
  Bars* sb = reinterpret_cast<Bars*>(base + (size_t)kStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x, nt = blockIdx.y;
  // this CTA's K blocks [kb0, kb0 + nkb)
  const int kb0 = (int)blockIdx.z * kNetKPer;
  const int nkb = min(kNetKPer, a.k_blocks - kb0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sb->full[s], 1);
      mbar_init(&sb->empty[s], 1);
    }
    mbar_init(&sb->done, 1);
    sb->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sb->tmem_base)),
                 "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sb->tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      int kb = 0;
      for (; kb < nkb; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        if (!mbar_wait(sb, &sb->empty[s], ph ^ 1u, a.status, 1u)) break;
        mbar_expect_tx(&sb->full[s], kStageBytes);
#pragma unroll
        for (int p = 0; p < kParts; ++p) {
          tma_3d(Ap(p, s), &tmap_a, (kb0 + kb) * kBKf, mt * kBM, p, &sb->full[s]);
          tma_3d(Wp(p, s), &tmap_w, (kb0 + kb) * kBKf, nt * kN, p, &sb->full[s]);
        }
      }
      for (int j = kb - kStages > 0 ? kb - kStages : 0; j < kb; ++j)
        mbar_drain(&sb->full[j % kStages], (uint32_t)(j / kStages) & 1u, a.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, kN);
      int kb = 0;
      for (; kb < nkb; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        if (!mbar_wait(sb, &sb->full[s], ph, a.status, 2u)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t x1 = smem_u32(Ap(0, s)), x2 = smem_u32(Ap(1, s)), x3 = smem_u32(Ap(2, s));
        const uint32_t w1 = smem_u32(Wp(0, s)), w2 = smem_u32(Wp(1, s)), w3 = smem_u32(Wp(2, s));
        const uint32_t d_main = tmem + (uint32_t)((kb & 1) * kN), d_corr = tmem + (uint32_t)(2 * kN);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t o = (uint32_t)j * 32u;
          const uint32_t first = (kb < 2 && j == 0) ? 0u : 1u;
          const uint32_t first_c = (kb == 0 && j == 0) ? 0u : 1u;
          mma_bf16(d_main, smem_desc_sw64(x1 + o), smem_desc_sw64(w1 + o), idesc, first);
          mma_bf16(d_corr, smem_desc_sw64(x1 + o), smem_desc_sw64(w2 + o), idesc, first_c);
          mma_bf16(d_corr, smem_desc_sw64(x2 + o), smem_desc_sw64(w1 + o), idesc, 1u);
          mma_bf16(d_corr, smem_desc_sw64(x2 + o), smem_desc_sw64(w2 + o), idesc, 1u);
          mma_bf16(d_corr, smem_desc_sw64(x1 + o), smem_desc_sw64(w3 + o), idesc, 1u);
          mma_bf16(d_corr, smem_desc_sw64(x3 + o), smem_desc_sw64(w1 + o), idesc, 1u);
        }
        mma_commit(&sb->empty[s]);
      }
      mma_commit(&sb->done);
    }
  } else {
    const int q = warp & 3;
    const int rrow = q * 32 + lane;
    const uint32_t lanes = tmem + ((uint32_t)(q * 32) << 16);
    mbar_drain(&sb->done, 0u, a.status);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int64_t r = (int64_t)mt * kBM + rrow;
    const bool valid = !sb->abort_flag && r < a.rows;
    const bool odd = nkb > 1;
    const int half_n = a.n / 2;
    const bool split = a.splits > 1;
#pragma unroll 1
    for (int j0 = 0; j0 < kN; j0 += 8) {
      const int col = nt * kN + j0;
      float x[8], x1[8], xc[8];
      tmem_ld8(lanes + (uint32_t)j0, x);
      tmem_ld8(lanes + (uint32_t)(kN + j0), x1);
      tmem_ld8(lanes + (uint32_t)(2 * kN + j0), xc);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (!valid || col >= a.n) continue;
      if (split) {
        // this split's partial sums; the bias and the activation follow the split-ordered sum
        float* prow = a.partial + ((int64_t)blockIdx.z * a.rows + r) * a.n;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (col + i < a.n) prow[col + i] = (odd ? x[i] + x1[i] : x[i]) + xc[i];
        continue;
      }
      float o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float z = ((odd ? x[i] + x1[i] : x[i]) + xc[i]) + (col + i < a.n ? a.bias[col + i] : 0.0f);
        o[i] = a.act >= 0 ? net_act(a.act, z) : z;
      }
      if (a.out) {
        float* orow = a.out + r * a.ldo;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (col + i < a.n) orow[col + i] = o[i];
      }
      if (a.parts) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          if (col + i >= a.n) break;
          uint32_t p1, p2, p3;
          split2(o[i], o[i + 1], p1, p2, p3);
          uint32_t* d = a.parts + r * half_n + (col + i) / 2;
          d[0] = p1;
          d[a.plane_words] = p2;
          d[2 * a.plane_words] = p3;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols) : "memory");
  }
}

// The split layer's outputs: z = ((p_0 + p_1) + ...) + b, activated, into the FP32 output and/or the BF16
// parts (one thread per pair of outputs of a row).
__global__ void __launch_bounds__(256) k_net_x3_reduce(NetX3Args a) {
  griddep_wait();
  griddep_launch_dependents();
  const int64_t half_n = a.n / 2;
  const int64_t total = (int64_t)a.rows * half_n;
  const int64_t plane = (int64_t)a.rows * a.n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / half_n, j = 2 * (t - r * half_n);
    const float* p = a.partial + r * a.n + j;
    float z0 = p[0], z1 = p[1];
    for (int s = 1; s < a.splits; ++s) {
      z0 += p[s * plane];
      z1 += p[s * plane + 1];
    }
    z0 += a.bias[j];
    z1 += a.bias[j + 1];
    if (a.act >= 0) {
      z0 = net_act(a.act, z0);
      z1 = net_act(a.act, z1);
    }
    if (a.out) {
      a.out[r * a.ldo + j] = z0;
      a.out[r * a.ldo + j + 1] = z1;
    }
    if (a.parts) {
      uint32_t p1, p2, p3;
      split2(z0, z1, p1, p2, p3);
      uint32_t* d = a.parts + r * half_n + j / 2;
      d[0] = p1;
      d[a.plane_words] = p2;
      d[2 * a.plane_words] = p3;
    }
  }
}

size_t net_x3_smem() { return 1024 + (size_t)kStages * kStageBytes + ((sizeof(Bars) + 15) & ~size_t(15)) + 64; }

}  // namespace

bool net_x3_layer(int fi, int fo) { return fi % 8 == 0 && fo >= 16 && fo % 2 == 0; }

int net_x3_splits(int fan_in) { return (fan_in + kNetKPer * kBKf - 1) / (kNetKPer * kBKf); }

int64_t net_x3_words(const NetOut& net, int64_t max_rows) {
  int64_t w = 2 * 3 * max_rows * (int64_t)((net.wmax + 1) / 2);
  int ks = 1;
  for (int l = 0; l < net.n_layers; ++l)
    if (net_x3_layer(net.widths[l], net.widths[l + 1]) && net_x3_splits(net.widths[l]) > ks)
      ks = net_x3_splits(net.widths[l]);
  if (ks > 1) w += (int64_t)ks * max_rows * net.wmax;  // the split layers' FP32 partial sums
  for (int l = 0; l < net.n_layers; ++l)
    if (net_x3_layer(net.widths[l], net.widths[l + 1])) w += 3 * (int64_t)net.widths[l + 1] * (net.widths[l] / 2);
  return w;
}

bool net_x3_plan(NetX3Plan& pl, const NetOut& net, int64_t max_rows, uint32_t* buf) {
  pl = NetX3Plan();
  if (!buf) return false;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major != 10) {
    cudaGetLastError();
    return false;
  }
  pl.max_rows = max_rows;
  const int64_t act_words = 3 * max_rows * (int64_t)((net.wmax + 1) / 2);
  pl.act_parts[0] = buf;
  pl.act_parts[1] = buf + act_words;
  uint32_t* wcur = buf + 2 * act_words;
  int ks = 1;
  for (int l = 0; l < net.n_layers; ++l)
    if (net_x3_layer(net.widths[l], net.widths[l + 1]) && net_x3_splits(net.widths[l]) > ks)
      ks = net_x3_splits(net.widths[l]);
  if (ks > 1) {
    pl.partial = reinterpret_cast<float*>(wcur);
    wcur += (int64_t)ks * max_rows * net.wmax;
  }
  bool any = false;
  for (int l = 0; l < net.n_layers; ++l) {
    const int fi = net.widths[l], fo = net.widths[l + 1];
    pl.tc[l] = net_x3_layer(fi, fo);
    if (!pl.tc[l]) continue;
    any = true;
    pl.w_parts[l] = wcur;
    wcur += 3 * (int64_t)fo * (fi / 2);
    {
      // the layer's input parts [3][max_rows][fi] in buffer l & 1, box 32 x 128 x 1
      cuuint64_t dims[3] = {(cuuint64_t)fi, (cuuint64_t)max_rows, 3};
      cuuint64_t strides[2] = {(cuuint64_t)fi * 2, (cuuint64_t)(max_rows * fi * 2)};
      cuuint32_t box[3] = {kBKf, kBM, 1};
      if (!encode_bf16(&pl.tmap_a[l], pl.act_parts[l & 1], dims, strides, box)) return false;
    }
    {
      // the weights' parts [3][fo][fi], box 32 x 128 x 1 (rows past fo are zero fill)
      cuuint64_t dims[3] = {(cuuint64_t)fi, (cuuint64_t)fo, 3};
      cuuint64_t strides[2] = {(cuuint64_t)fi * 2, (cuuint64_t)((int64_t)fo * fi * 2)};
      cuuint32_t box[3] = {kBKf, (cuuint32_t)kN, 1};
      if (!encode_bf16(&pl.tmap_w[l], pl.w_parts[l], dims, strides, box)) return false;
    }
  }
  if (!any || ensure_smem_limit<k_net_x3>(net_x3_smem()) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  pl.ready = true;
  return true;
}

int launch_net_x3_split_w(const NetX3Plan& pl, const NetOut& net, cudaStream_t s) {
  if (!pl.ready) return 0;
  int n = 0;
  for (int l = 0; l < net.n_layers; ++l) {
    if (!pl.tc[l]) continue;
    const int fi = net.widths[l], fo = net.widths[l + 1];
    const int64_t pairs = fi / 2;
    if (split_launch(net.params + net.w_off[l], fi, nullptr, fo, 0, pairs, pl.w_parts[l], pairs, (int64_t)fo * pairs,
                     s) < 0)
      return -1;
    ++n;
  }
  return n;
}

int launch_net_output_x3(const NetX3Plan& pl, const NetOut& net, const float* rows, int64_t ld, int32_t count,
                         float* fit, float* scratch, int64_t scratch_ld, uint32_t* status, cudaStream_t s) {
  if (count <= 0) return 0;
  if (!pl.ready || count > pl.max_rows) return -1;
  int n = 0;
  const float* a = rows;  // the FP32 input of the next CUDA-core layer
  int64_t lda = ld;
  for (int l = 0; l < net.n_layers; ++l) {
    const int fi = net.widths[l], fo = net.widths[l + 1];
    const bool last = l + 1 == net.n_layers;
    const bool next_tc = !last && pl.tc[l + 1];
    float* o = last ? fit : scratch + (int64_t)(l & 1) * scratch_ld * count;
    const int64_t ldo = last ? 1 : scratch_ld;
    const float* b = net.params + net.b_off[l];
    const int32_t ak = last ? -1 : net.acts[l];
    if (pl.tc[l]) {
      if (l == 0) {
        // the sparks -> their BF16 parts in buffer 0
        const int64_t pairs = fi / 2;
        if (split_launch(rows, ld, nullptr, count, 0, pairs, pl.act_parts[0], pairs, pl.max_rows * pairs, s) < 0)
          return -1;
        ++n;
      }
      NetX3Args x;
      x.rows = count;
      x.k_blocks = (fi + kBKf - 1) / kBKf;
      x.splits = net_x3_splits(fi);
      x.partial = pl.partial;
      x.n = fo;
      x.act = ak;
      x.bias = b;
      x.out = next_tc ? nullptr : o;
      x.ldo = ldo;
      x.parts = next_tc ? pl.act_parts[(l + 1) & 1] : nullptr;
      x.plane_words = pl.max_rows * (fo / 2);
      x.status = status;
      const dim3 grid((unsigned)((count + kBM - 1) / kBM), (unsigned)((fo + kN - 1) / kN), (unsigned)x.splits);
      if (launch_pdl(k_net_x3, grid, dim3(kThreads), net_x3_smem(), s, pl.tmap_a[l], pl.tmap_w[l], x) !=
          cudaSuccess)
        return -1;
      ++n;
      if (x.splits > 1) {
        const int64_t pairs = (int64_t)count * (fo / 2);
        const unsigned blocks = (unsigned)((pairs + 255) / 256 < 4096 ? (pairs + 255) / 256 : 4096);
        if (launch_pdl(k_net_x3_reduce, dim3(blocks), dim3(256), 0, s, x) != cudaSuccess) return -1;
        ++n;
      }
    } else {
      if (launch_net_layer(a, lda, count, net.params + net.w_off[l], b, fi, fo, ak, o, ldo, s) < 0) return -1;
      ++n;
      if (next_tc) {
        // this layer's FP32 output -> the next layer's parts
        const int64_t pairs = fo / 2;
        if (split_launch(o, ldo, nullptr, count, 0, pairs, pl.act_parts[(l + 1) & 1], pairs, pl.max_rows * pairs,
                         s) < 0)
          return -1;
        ++n;
      }
    }
    a = o;
    lda = ldo;
  }
  return n;
}

}  // namespace mgfwa
