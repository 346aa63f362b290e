// FP32-accurate first layer on the tensor cores, for a few search vectors
// at once: act(X W1^T + b1) of R vectors (rows of the spark buffer, picked
// by an index) over the whole batch, written to [R][N][H] for the FP32
// output-layer kernel.  Used where FP32 accuracy is required (the elite
// re-score, the refinement's forward pass).
//
// Each FP32 operand v is split into three TF32-exact parts: v1 = v with its
// low 13 mantissa bits cleared, v2 = the same of v - v1, v3 = v - v1 - v2
// (all exact in FP32; |v2| <= 2^-10 |v|, |v3| <= 2^-20 |v|).  Six tcgen05
// kind::tf32 MMAs per K step accumulate a1b1 + a1b2 + a2b1 + a2b2 + a1b3 +
// a3b1 in FP32: the products are exact, and the dropped terms (a2b3, a3b2,
// a3b3, and the TF32 reading of v3) are below 2^-29 of each product.  The
// tensor core's own accumulation rounds at every step, so the main products
// a1b1 go to two accumulators (even and odd K blocks) and the five
// corrections (about 2^-10 of them) to a third; the epilogue adds the three
// in FP32.  That keeps the result within FP32 accuracy for K in the
// thousands.
//
// One CTA per (128-sample tile, vector): warp 0 issues TMA (FP32 tiles of X
// and W1, 32 K-elements = one 128-byte swizzle row), warps 2..5 split each
// landed stage in place (v1 over the FP32 tile, v2 and v3 into two twin
// buffers at the same offsets, so the swizzled layout carries over
// unchanged), warp 1 issues the MMAs into H TMEM columns, and warps 2..5
// finally read the
// accumulator (one sample row per thread), add b1, apply the activation and
// store the row.  Every wait is bounded; a wait that gives up sets a bit in
// the status word and the CTA drains its copies and MMAs and returns.
#include <cuda.h>

#include "fp32x3.cuh"
#include "mgfwa_internal.cuh"

namespace mgfwa {
namespace {

constexpr int kBM = 128;
constexpr int kBKf = 32;           // FP32 K elements per stage (128 bytes)
constexpr int kMaxStages = 3;
constexpr int kParts = 3;          // TF32 parts per operand
constexpr int kThreads = 192;      // warp 0 TMA, warp 1 MMA, warps 2..5 convert + epilogue
constexpr uint64_t kWaitBudget = 1ull << 32;

struct Bars {
  uint64_t full[kMaxStages];
  uint64_t conv[kMaxStages];
  uint64_t empty[kMaxStages];
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
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
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

// v -> (v1, v2, v3): v1 the TF32 truncation of v, v2 that of v - v1, v3 the rest.
__device__ __forceinline__ void split1(float v, float& p1, float& p2, float& p3) {
  p1 = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
  const float r = v - p1;
  p2 = __uint_as_float(__float_as_uint(r) & 0xFFFFE000u);
  p3 = r - p2;
}

// Elements [t, n) step 128 of a stage buffer: v1 in place, v2 and v3 to the twins.
__device__ __forceinline__ void split3(float4* p1, float4* p2, float4* p3, int n, int t) {
  for (int e = t; e < n; e += 128) {
    const float4 v = p1[e];
    float4 x, y, z;
    split1(v.x, x.x, y.x, z.x);
    split1(v.y, x.y, y.y, z.y);
    split1(v.z, x.z, y.z, z.z);
    split1(v.w, x.w, y.w, z.w);
    p1[e] = x;
    p2[e] = y;
    p3[e] = z;
  }
}

struct Args {
  int32_t N;        // samples
  int32_t d_in;
  int32_t k_blocks;
  int32_t act;
  int64_t ld;       // FP32 row stride of the spark buffer
  int64_t b1_off;   // offset of b1 in a row
  const float* rows;
  const int32_t* idx;  // vector r is spark row idx[r] (or r)
  float* out;       // [R][N][H]
  uint32_t* status;
};

// Stages that fit: 3 parts of the X and W1 tiles per stage.
constexpr int stages_for(int h) { return h >= 128 ? 2 : kMaxStages; }

template <int H>
__global__ void __launch_bounds__(kThreads, 1)
    k_l1_fp32x3(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_w, Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  constexpr int kStages = stages_for(H);
  constexpr uint32_t kABytes = kBM * 128;  // one stage of the X tile (FP32)
  constexpr uint32_t kBBytes = H * 128;    // one stage of the W1 tile (FP32)
  constexpr uint32_t kTmemCols = H == 32 ? 128 : (H == 64 ? 256 : 512);  // >= 3 H columns: main even, main odd, corrections
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // part p of stage s: A at base + (p * kStages + s) * kABytes, B after all A parts
  uint8_t* a_part = base;
  uint8_t* b_part = base + (size_t)kParts * kStages * kABytes;
  auto A = [&](int p, int s) { return a_part + ((size_t)p * kStages + s) * kABytes; };
  auto Bp = [&](int p, int s) { return b_part + ((size_t)p * kStages + s) * kBBytes; };
  Bars* sb = reinterpret_cast<Bars*>(b_part + (size_t)kParts * kStages * kBBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x, r = blockIdx.y;
  const int row = a.idx ? a.idx[r] : r;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sb->full[s], 1);
      mbar_init(&sb->conv[s], 4);
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
      for (; kb < a.k_blocks; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        if (!mbar_wait(sb, &sb->empty[s], ph ^ 1u, a.status, 1u)) break;
        mbar_expect_tx(&sb->full[s], kABytes + kBBytes);
        tma_2d(A(0, s), &tmap_x, kb * kBKf, mt * kBM, &sb->full[s]);
        tma_3d(Bp(0, s), &tmap_w, kb * kBKf, 0, row, &sb->full[s]);
      }
      // every issued copy lands before the CTA may exit
      for (int j = kb - kStages > 0 ? kb - kStages : 0; j < kb; ++j)
        mbar_drain(&sb->full[j % kStages], (uint32_t)(j / kStages) & 1u, a.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(kBM, H);
      int kb = 0;
      for (; kb < a.k_blocks; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        if (!mbar_wait(sb, &sb->conv[s], ph, a.status, 2u)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a1 = smem_u32(A(0, s)), a2 = smem_u32(A(1, s)), a3 = smem_u32(A(2, s));
        const uint32_t b1 = smem_u32(Bp(0, s)), b2 = smem_u32(Bp(1, s)), b3 = smem_u32(Bp(2, s));
        const uint32_t d_main = tmem + (uint32_t)((kb & 1) * H), d_corr = tmem + (uint32_t)(2 * H);
#pragma unroll
        for (int k = 0; k < kBKf / 8; ++k) {
          const uint32_t o = (uint32_t)k * 32u;
          const uint32_t first = (kb < 2 && k == 0) ? 0u : 1u;        // this main accumulator's first product
          const uint32_t first_c = (kb == 0 && k == 0) ? 0u : 1u;     // the corrections' first product
          mma_tf32(d_main, smem_desc(a1 + o), smem_desc(b1 + o), idesc, first);
          mma_tf32(d_corr, smem_desc(a1 + o), smem_desc(b2 + o), idesc, first_c);
          mma_tf32(d_corr, smem_desc(a2 + o), smem_desc(b1 + o), idesc, 1u);
          mma_tf32(d_corr, smem_desc(a2 + o), smem_desc(b2 + o), idesc, 1u);
          mma_tf32(d_corr, smem_desc(a1 + o), smem_desc(b3 + o), idesc, 1u);
          mma_tf32(d_corr, smem_desc(a3 + o), smem_desc(b1 + o), idesc, 1u);
        }
        mma_commit(&sb->empty[s]);
      }
      mma_commit(&sb->done);  // after every issued MMA (also on abort)
    }
  } else {
    // split each landed stage: hi in place, lo into the twin buffer
    const int ct = threadIdx.x - 64;  // 0..127
    bool ok = true;
    for (int kb = 0; kb < a.k_blocks && ok; ++kb) {
      const int s = kb % kStages;
      const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
      // the twin buffers of this stage are free once the stage's MMAs completed
      ok = mbar_wait(sb, &sb->full[s], ph, a.status, 4u);
      if (!ok) break;
      split3(reinterpret_cast<float4*>(A(0, s)), reinterpret_cast<float4*>(A(1, s)),
             reinterpret_cast<float4*>(A(2, s)), (int)(kABytes / 16), ct);
      split3(reinterpret_cast<float4*>(Bp(0, s)), reinterpret_cast<float4*>(Bp(1, s)),
             reinterpret_cast<float4*>(Bp(2, s)), (int)(kBBytes / 16), ct);
      // generic-proxy writes become visible to the tensor core's (async proxy) reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&sb->conv[s]);
    }
    // epilogue: row = this thread's TMEM lane
    const int q = warp & 3;            // lane quadrant this warp may access
    const int rrow = q * 32 + lane;
    mbar_drain(&sb->done, 0u, a.status);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int64_t n = (int64_t)mt * kBM + rrow;
    const float* bias = a.rows + (int64_t)row * a.ld + a.b1_off;
    float* out = a.out + ((int64_t)r * a.N + n) * H;
    const bool valid = ok && !sb->abort_flag && n < a.N;
    const uint32_t lanes = tmem + ((uint32_t)(q * 32) << 16);
    const bool odd = a.k_blocks > 1;  // the odd-block accumulator holds products
#pragma unroll 1
    for (int j0 = 0; j0 < H; j0 += 8) {
      float v[8], v1[8], vc[8];
      tmem_ld8(lanes + (uint32_t)j0, v);
      tmem_ld8(lanes + (uint32_t)(H + j0), v1);
      tmem_ld8(lanes + (uint32_t)(2 * H + j0), vc);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = (odd ? v[i] + v1[i] : v[i]) + vc[i];
      if (valid) {
        float o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float z = v[i] + bias[j0 + i];
          o[i] = a.act == kActTanh ? tanhf(z) : fmaxf(z, 0.f);
        }
        *reinterpret_cast<float4*>(out + j0) = make_float4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<float4*>(out + j0 + 4) = make_float4(o[4], o[5], o[6], o[7]);
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

bool encode(CUtensorMap* map, uint32_t rank, const void* ptr, const cuuint64_t* dims, const cuuint64_t* strides,
            const cuuint32_t* box) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t smem_bytes(int H) {
  return 1024 + (size_t)stages_for(H) * kParts * ((size_t)kBM * 128 + (size_t)H * 128) + sizeof(Bars) + 64;
}

template <int H>
cudaError_t go(const L1Plan& pl, const Args& a, int R, cudaStream_t s, bool prep) {
  cudaError_t e = ensure_smem_limit<k_l1_fp32x3<H>>(smem_bytes(H));
  if (e != cudaSuccess || prep) return e;
  const dim3 grid((unsigned)((a.N + kBM - 1) / kBM), (unsigned)R);
  k_l1_fp32x3<H><<<grid, kThreads, smem_bytes(H), s>>>(pl.tmap_x, pl.tmap_w, a);
  return cudaPeekAtLastError();
}

}  // namespace

bool l1_fp32x3_supported(const Mlp& mlp) {
  const int h1 = mlp.widths[1];
  return mlp.widths[0] % 4 == 0 && (h1 == 32 || h1 == 64 || h1 == 128);
}

bool l1_fp32x3_plan(L1Plan& pl, const Mlp& mlp, const float* rows, int64_t ld, int64_t max_rows) {
  pl = L1Plan();
  if (!l1_fp32x3_supported(mlp)) return false;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major != 10) {
    cudaGetLastError();
    return false;
  }
  const int d_in = mlp.widths[0], h1 = mlp.widths[1];
  {
    cuuint64_t dims[2] = {(cuuint64_t)d_in, (cuuint64_t)mlp.N};
    cuuint64_t strides[1] = {(cuuint64_t)d_in * 4};
    cuuint32_t box[2] = {kBKf, kBM};
    if (!encode(&pl.tmap_x, 2, mlp.X, dims, strides, box)) return false;
  }
  {
    // W1 of every spark row: [max_rows][h1][d_in], box 32 x h1 x 1
    cuuint64_t dims[3] = {(cuuint64_t)d_in, (cuuint64_t)h1, (cuuint64_t)max_rows};
    cuuint64_t strides[2] = {(cuuint64_t)d_in * 4, (cuuint64_t)ld * 4};
    cuuint32_t box[3] = {kBKf, (cuuint32_t)h1, 1};
    if (!encode(&pl.tmap_w, 3, rows + mlp.w_off[0], dims, strides, box)) return false;
  }
  pl.rows = rows;
  pl.ld = ld;
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

int launch_l1_fp32x3(const L1Plan& pl, const Mlp& mlp, const int32_t* idx, int32_t R, float* out,
                     uint32_t* status, cudaStream_t s) {
  if (!pl.ready || R <= 0) return R <= 0 ? 0 : -1;
  Args a;
  a.N = (int32_t)mlp.N;
  a.d_in = mlp.widths[0];
  a.k_blocks = (mlp.widths[0] + kBKf - 1) / kBKf;
  a.act = mlp.acts[0];
  a.ld = pl.ld;
  a.b1_off = mlp.b_off[0];
  a.rows = pl.rows;
  a.idx = idx;
  a.out = out;
  a.status = status;
  cudaError_t e;
  switch (mlp.widths[1]) {
    case 32: e = go<32>(pl, a, R, s, false); break;
    case 64: e = go<64>(pl, a, R, s, false); break;
    case 128: e = go<128>(pl, a, R, s, false); break;
    default: return -1;
  }
  return e == cudaSuccess ? 1 : -1;
}

}  // namespace mgfwa
