// Philox-driven sampling kernels: firework initialisation, explosion sparks
// and multi-guiding sparks, each with the random mapping of out-of-bound
// coordinates (GPU-MGFWA, Algorithm 1: init, explosion + mapping, multi-
// guiding + mapping).
//
// Every state value is produced with explicitly rounded FP32 intrinsics
// (__fmaf_rn, __fadd_rn, ...), which the compiler never contracts or
// reorders, so the positions are a pure function of (seed, generation,
// unit, coordinate) and the firework state.
//
// Layout: rows of Dp floats (Dp a multiple of 64, so each row starts on a
// 256-byte boundary); one thread owns four consecutive coordinates, i.e.
// one Philox4x32 block, and moves them with 16-byte loads and stores.  The
// tensor-core operand of a spark is the first w1_elems coordinates of its
// row, stored contiguously (row-major [h1][d_in]) as BF16 (one 8-byte store
// per thread) or as E4M3 of coordinate * inv_scale (one 4-byte store).
#include <cuda_fp8.h>

#include "mgfwa_internal.cuh"

namespace mgfwa {

namespace {

constexpr int kThreads = 128;

// Reading of the population-based random mapping: a coordinate outside
// [lb, ub] is redrawn uniformly in the firework's amplitude box clipped to
// the bounds, lo + u (hi - lo).
__device__ __forceinline__ float map_coord(float x, float amp, float lb, float ub, float u) {
  float lo = __fsub_rn(x, amp);
  float hi = __fadd_rn(x, amp);
  if (lo < lb) lo = lb;
  if (hi > ub) hi = ub;
  return __fmaf_rn(u, __fsub_rn(hi, lo), lo);
}

__device__ __forceinline__ void store_bf16x4(__nv_bfloat16* dst, float a, float b, float c, float d) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(a, b);
  __nv_bfloat162 hi = __floats2bfloat162_rn(c, d);
  uint2 v;
  v.x = *reinterpret_cast<uint32_t*>(&lo);
  v.y = *reinterpret_cast<uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(dst) = v;
}

// Four E4M3 values of (v * inv) (round to nearest even, saturating), one
// 4-byte store.
__device__ __forceinline__ void store_fp8x4(uint8_t* dst, float inv, float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a * inv, b * inv), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c * inv, d * inv), __NV_SATFINITE, __NV_E4M3);
  *reinterpret_cast<uint32_t*>(dst) = lo | (hi << 16);
}

// Coordinates [d0, d0 + 4) of operand row `row` (d0 < w1_elems).
__device__ __forceinline__ void store_op4(const OpDesc& op, int64_t row, int64_t d0, float a, float b, float c,
                                          float d) {
  uint8_t* base = static_cast<uint8_t*>(op.base);
  if (op.kind == kOpFp8)
    store_fp8x4(base + row * op.w1_elems + d0, op.inv_scale, a, b, c, d);
  else
    store_bf16x4(reinterpret_cast<__nv_bfloat16*>(base) + row * op.w1_elems + d0, a, b, c, d);
}

// Coordinates [d0, d0 + 4) of row `row` into a BF16 copy of one weight
// matrix [classes][k] (at coordinate `off` of a spark row; `row_elems` per
// spark in the copy) when they lie in it (k is a multiple of 4 and the
// matrix starts on a multiple of 4, so the four never straddle two of its
// rows).
__device__ __forceinline__ void store_copy4(void* copy, int64_t off, int32_t k, int32_t classes, int64_t row_elems,
                                            int64_t row, int64_t d0, float a, float b, float c, float d) {
  const int64_t e = d0 - off;
  if (e < 0 || e >= (int64_t)classes * k) return;
  const int64_t cls = e / k;
  const int64_t j = e - cls * k;
  store_bf16x4(static_cast<__nv_bfloat16*>(copy) + row * row_elems + cls * k + j, a, b, c, d);
}

// The BF16 copies of W2 and W3 (where the descriptor has them).
__device__ __forceinline__ void store_w2_4(const OpDesc& op, int64_t row, int64_t d0, float a, float b, float c,
                                           float d) {
  store_copy4(op.w2, op.w2_off, op.w2_h1, op.w2_classes, op.w2_row_elems(), row, d0, a, b, c, d);
  if (op.w3) store_copy4(op.w3, op.w3_off, op.w3_k, op.w3_classes, op.w3_row_elems(), row, d0, a, b, c, d);
}

// grid (coordinate blocks, B * mu): global firework z = b * mu + i (Philox
// unit: the firework's index in its run, i + fw_off).
__global__ void __launch_bounds__(kThreads) k_init(Problem p, float* __restrict__ fw_x,
                                                   float* __restrict__ fw_amp) {
  griddep_wait();
  griddep_launch_dependents();
  const int z = blockIdx.y;
  const int b = z / p.mu, i = z - b * p.mu;
  const int64_t c4 = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t d0 = c4 * 4;
  if (blockIdx.x == 0 && threadIdx.x == 0) fw_amp[z] = p.amp0;
  if (d0 >= p.Dp) return;
  uint32_t k0, k1;
  run_key(p, b, k0, k1);
  const uint4 r = philox4x32_10(make_uint4((uint32_t)c4, (uint32_t)(i + p.fw_off), 0u, kInit), k0, k1);
  const float width = __fsub_rn(p.ub, p.lb);
  float v[4];
#pragma unroll
  for (int l = 0; l < 4; ++l)
    v[l] = (d0 + l < p.D) ? __fmaf_rn(u24(lane_of(r, l)), width, p.lb) : 0.0f;
  *reinterpret_cast<float4*>(fw_x + (int64_t)z * p.Dp + d0) = make_float4(v[0], v[1], v[2], v[3]);
}

// 2u - 1 for u = (r >> 8) 2^-24, as one FMA: (r >> 8) 2^-23 - 1 is exact in
// FP32 (a multiple of 2^-23 in [-1, 1)), so the value equals the two-step
// form 2u - 1 bit for bit.
__device__ __forceinline__ float signed_u24(uint32_t r) {
  return __fmaf_rn(__uint2float_rn(r >> 8), 0x1p-23f, -1.0f);
}

// grid (coordinate blocks, lambda, B * mu): one block covers kExplodeBlocks *
// kThreads Philox blocks (4 coordinates each) of one spark row; each thread
// takes kExplodeBlocks of them, kThreads apart, so a warp's stores stay
// contiguous.  Global firework z = b * mu + i, spark row z * lam + j, Philox
// unit (i + fw_off) * lam + j of run b's stream.  The thread's firework
// coordinates are loaded first; per Philox block the explosion draw, then
// the mapping stream's block for the coordinates outside [lb, ub].  While the
// firework's amplitude is at least a quarter of the box, nearly every block
// has such a coordinate and the mapping block is drawn unconditionally (no
// vote, so the compiler interleaves it with the next block's draw); below
// that it is drawn only when a lane of the warp needs it (a warp-uniform
// branch).  The values are the same either way: a mapped value replaces only
// an out-of-bound coordinate.  Threads whose four blocks all lie inside the
// row's first D coordinates (all but the row's last few) skip the per-
// coordinate range checks.  Two more exact shortcuts, each chosen per
// firework: with symmetric bounds (lb = -ub) a coordinate is out of bounds
// iff |v| > ub; with an amplitude of at least ub - lb (rounded up), the
// mapping box of every firework coordinate (fireworks lie inside the bounds)
// is the whole of [lb, ub], so the mapped value is lb + u (ub - lb).
constexpr int kExplodeBlocks = 4;

template <bool kAlwaysMap, bool kFull, bool kSym, bool kBox>
__device__ __forceinline__ void explode_blocks(const Problem& p, const PhiloxKeys& rk, uint32_t unit, uint32_t gen,
                                               float amp, uint32_t c0, const float* __restrict__ xrow,
                                               float* __restrict__ srow, const OpDesc& op, uint32_t row,
                                               uint8_t* op_row, __nv_bfloat16* op_row16) {
  const float lb = p.lb, ub = p.ub;
  const uint32_t n4 = (uint32_t)(p.Dp / 4);
  const uint32_t full4 = (uint32_t)(p.D / 4);  // blocks whose 4 coordinates are all < D
  const uint32_t D = (uint32_t)p.D;
  const uint32_t w1e = (uint32_t)op.w1_elems;
  const uint32_t w2lo = (uint32_t)op.w2_off, w2len = (uint32_t)(op.w2_classes * op.w2_h1);
  const uint32_t w3lo = (uint32_t)op.w3_off, w3len = (uint32_t)(op.w3_classes * op.w3_k);
  float4 x4[kExplodeBlocks];
#pragma unroll
  for (int h = 0; h < kExplodeBlocks; ++h) {
    const uint32_t c4 = c0 + (uint32_t)h * kThreads;
    x4[h] = (kFull || c4 < n4) ? *reinterpret_cast<const float4*>(xrow + (size_t)c4 * 4)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int h = 0; h < kExplodeBlocks; ++h) {
    const uint32_t c4 = c0 + (uint32_t)h * kThreads;
    const bool live = kFull || c4 < n4;
    const uint32_t d0 = c4 * 4u;
    const uint4 r = philox4x32_10(make_uint4(c4, unit, gen, kExplode), rk);
    float v[4];
    bool oob[4];
    bool any = false;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      v[l] = __fmaf_rn(amp, signed_u24(lane_of(r, l)), lane_of(x4[h], l));
      oob[l] = kSym ? fabsf(v[l]) > ub : (v[l] < lb || v[l] > ub);
      if (!kFull) oob[l] = oob[l] && live && (c4 < full4 || d0 + (uint32_t)l < D);
      any |= oob[l];
    }
    if (kAlwaysMap || __any_sync(0xffffffffu, any)) {
      const uint4 r2 = philox4x32_10(make_uint4(c4, unit, gen, kMap), rk);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const float m = kBox ? __fmaf_rn(u24(lane_of(r2, l)), __fsub_rn(ub, lb), lb)
                             : map_coord(lane_of(x4[h], l), amp, lb, ub, u24(lane_of(r2, l)));
        v[l] = oob[l] ? m : v[l];
      }
    }
    if (!live) continue;
    if (!kFull && c4 >= full4) {
#pragma unroll
      for (int l = 0; l < 4; ++l)
        if (d0 + (uint32_t)l >= D) v[l] = 0.0f;
    }
    *reinterpret_cast<float4*>(srow + d0) = make_float4(v[0], v[1], v[2], v[3]);
    if (d0 < w1e) {
      if (op.kind == kOpBf16)
        store_bf16x4(op_row16 + d0, v[0], v[1], v[2], v[3]);
      else if (op.kind == kOpFp8)
        store_fp8x4(op_row + d0, op.inv_scale, v[0], v[1], v[2], v[3]);
    }
    if (d0 - w2lo < w2len || d0 - w3lo < w3len) store_w2_4(op, row, d0, v[0], v[1], v[2], v[3]);
  }
}

__global__ void __launch_bounds__(kThreads) k_explode(Problem p, const uint32_t* __restrict__ gens_done,
                                                      const float* __restrict__ fw_x,
                                                      const float* __restrict__ fw_amp,
                                                      float* __restrict__ sparks, const OpDesc op) {
  griddep_wait();
  griddep_launch_dependents();
  const uint32_t gen = *gens_done + 1u;  // this generation (the counter is advanced by the selection)
  const uint32_t z = blockIdx.z;
  const uint32_t b = z / (uint32_t)p.mu, i = z - b * (uint32_t)p.mu;
  const uint32_t row = z * (uint32_t)p.lam + blockIdx.y;
  const uint32_t unit = (i + (uint32_t)p.fw_off) * (uint32_t)p.lam + blockIdx.y;
  uint32_t k0, k1;
  run_key(p, (int)b, k0, k1);
  const PhiloxKeys rk = philox_keys(k0, k1);  // shared by the thread's Philox blocks
  const float amp = fw_amp[z];
  const float* xrow = fw_x + (size_t)z * (size_t)p.Dp;
  float* srow = sparks + (size_t)row * (size_t)p.Dp;
  uint8_t* op_row = op.kind == kOpNone ? nullptr : static_cast<uint8_t*>(op.base) + (size_t)row * op.row_bytes();
  __nv_bfloat16* op_row16 = reinterpret_cast<__nv_bfloat16*>(op_row);
  const uint32_t c0 = blockIdx.x * (uint32_t)(kExplodeBlocks * kThreads) + threadIdx.x;
  const bool full = c0 + (uint32_t)((kExplodeBlocks - 1) * kThreads) < (uint32_t)(p.D / 4);
  const bool always_map = __fmul_rn(4.0f, amp) >= __fsub_rn(p.ub, p.lb);
  const bool box = amp >= __fsub_ru(p.ub, p.lb);
  const bool sym = p.lb == -p.ub;
#define MG_EXPLODE(A, F, SY, BX) explode_blocks<A, F, SY, BX>(p, rk, unit, gen, amp, c0, xrow, srow, op, row, op_row, \
                                                               op_row16)
  if (!full)
    MG_EXPLODE(false, false, false, false);
  else if (box)
    sym ? MG_EXPLODE(true, true, true, true) : MG_EXPLODE(true, true, false, true);
  else if (always_map)
    sym ? MG_EXPLODE(true, true, true, false) : MG_EXPLODE(true, true, false, false);
  else
    sym ? MG_EXPLODE(false, true, true, false) : MG_EXPLODE(false, true, false, false);
#undef MG_EXPLODE
}

// Multi-guiding sparks, reading: group q of firework i has ranked index
// lists top (best first) and bottom (worst first);
//   GV = (sum top rows - sum bottom rows) / k,  G = x + beta GV,
// each sum in list order, then the random mapping with its own stream.
// KU > 0: k == KU, all 2k row loads in flight before the ordered sums, with
// registers for exactly those rows; KU == 0: any k, two rows at a time.
// Lagged multi-guiding: with gv_out the vectors GV are also stored (row
// z * m + q, [Dp]); with gv_in the sums are skipped and the given vectors
// used instead; with a null `guides` only the vectors are produced.
template <int KU>
__global__ void __launch_bounds__(kThreads) k_guide(Problem p, const uint32_t* __restrict__ gens_done,
                                                    const float* __restrict__ fw_x,
                                                    const float* __restrict__ fw_amp,
                                                    const float* __restrict__ sparks,
                                                    const int32_t* __restrict__ top,
                                                    const int32_t* __restrict__ bottom,
                                                    const float* __restrict__ gv_in, float* __restrict__ gv_out,
                                                    float* __restrict__ guides, const OpDesc op) {
  griddep_wait();
  griddep_launch_dependents();
  const uint32_t gen = *gens_done + 1u;
  const int i = blockIdx.z;               // global firework z = b * mu + i_local
  const int gq = i * p.m + blockIdx.y;    // global guiding row z * m + q
  const int run = i / p.mu;
  const uint32_t gunit = (uint32_t)((i - run * p.mu + p.fw_off) * p.m + (int)blockIdx.y);  // (index in run) * m + q
  uint32_t k0, k1;
  run_key(p, run, k0, k1);
  const int64_t c4 = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t d0 = c4 * 4;
  if (d0 >= p.Dp) return;
  const int k = p.k;
  const float fk = (float)k;
  float gvl[4];
  if (gv_in) {
    const float4 g4 = *reinterpret_cast<const float4*>(gv_in + (int64_t)gq * p.Dp + d0);
    gvl[0] = g4.x; gvl[1] = g4.y; gvl[2] = g4.z; gvl[3] = g4.w;
  } else {
  const int32_t* t = top + (int64_t)gq * k;
  const int32_t* b = bottom + (int64_t)gq * k;
  const float* fs = sparks + (int64_t)i * p.lam * p.Dp + d0;
  float4 st, sb;
  if (KU > 0) {
    // all 2k loads in flight before the ordered sums
    float4 a[KU > 0 ? KU : 1], c[KU > 0 ? KU : 1];
#pragma unroll
    for (int r = 0; r < KU; ++r) {
      a[r] = *reinterpret_cast<const float4*>(fs + (int64_t)t[r] * p.Dp);
      c[r] = *reinterpret_cast<const float4*>(fs + (int64_t)b[r] * p.Dp);
    }
    st = a[0];
    sb = c[0];
#pragma unroll
    for (int r = 1; r < KU; ++r) {
      st.x = __fadd_rn(st.x, a[r].x); st.y = __fadd_rn(st.y, a[r].y);
      st.z = __fadd_rn(st.z, a[r].z); st.w = __fadd_rn(st.w, a[r].w);
      sb.x = __fadd_rn(sb.x, c[r].x); sb.y = __fadd_rn(sb.y, c[r].y);
      sb.z = __fadd_rn(sb.z, c[r].z); sb.w = __fadd_rn(sb.w, c[r].w);
    }
  } else {
    st = *reinterpret_cast<const float4*>(fs + (int64_t)t[0] * p.Dp);
    sb = *reinterpret_cast<const float4*>(fs + (int64_t)b[0] * p.Dp);
    for (int r = 1; r < k; ++r) {
      const float4 a = *reinterpret_cast<const float4*>(fs + (int64_t)t[r] * p.Dp);
      const float4 c = *reinterpret_cast<const float4*>(fs + (int64_t)b[r] * p.Dp);
      st.x = __fadd_rn(st.x, a.x); st.y = __fadd_rn(st.y, a.y);
      st.z = __fadd_rn(st.z, a.z); st.w = __fadd_rn(st.w, a.w);
      sb.x = __fadd_rn(sb.x, c.x); sb.y = __fadd_rn(sb.y, c.y);
      sb.z = __fadd_rn(sb.z, c.z); sb.w = __fadd_rn(sb.w, c.w);
    }
  }
#pragma unroll
  for (int l = 0; l < 4; ++l) gvl[l] = __fdiv_rn(__fsub_rn(lane_of(st, l), lane_of(sb, l)), fk);
  if (gv_out)
    *reinterpret_cast<float4*>(gv_out + (int64_t)gq * p.Dp + d0) = make_float4(gvl[0], gvl[1], gvl[2], gvl[3]);
  }
  if (!guides) return;
  const float amp = fw_amp[i];
  const float4 x4 = *reinterpret_cast<const float4*>(fw_x + (int64_t)i * p.Dp + d0);
  float v[4];
  bool out_of_bounds = false;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    v[l] = __fmaf_rn(p.beta, gvl[l], lane_of(x4, l));
    out_of_bounds |= (d0 + l < p.D) && (v[l] < p.lb || v[l] > p.ub);
  }
  if (out_of_bounds) {
    const uint4 r2 = philox4x32_10(make_uint4((uint32_t)c4, gunit, gen, kGmap), k0, k1);
#pragma unroll
    for (int l = 0; l < 4; ++l)
      if (v[l] < p.lb || v[l] > p.ub) v[l] = map_coord(lane_of(x4, l), amp, p.lb, p.ub, u24(lane_of(r2, l)));
  }
#pragma unroll
  for (int l = 0; l < 4; ++l)
    if (d0 + l >= p.D) v[l] = 0.0f;
  *reinterpret_cast<float4*>(guides + (int64_t)gq * p.Dp + d0) = make_float4(v[0], v[1], v[2], v[3]);
  if (op.kind != kOpNone && d0 < op.w1_elems) store_op4(op, gq, d0, v[0], v[1], v[2], v[3]);
  if (op.w2) store_w2_4(op, gq, d0, v[0], v[1], v[2], v[3]);
}

// The operand copies of `count` FP32 rows: the first-layer block and, with
// op.w2, the BF16 W2.  grid (coordinate blocks up to op_span(op), rows).
__global__ void k_to_operand(const float* __restrict__ rows, int64_t ld, const OpDesc op) {
  griddep_wait();
  griddep_launch_dependents();
  const int row = blockIdx.y;
  const int64_t d0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * 4;
  const bool in_w1 = d0 < op.w1_elems;
  const bool in_w2 = (op.w2 && d0 >= op.w2_off && d0 < op.w2_off + (int64_t)op.w2_classes * op.w2_h1) ||
                     (op.w3 && d0 >= op.w3_off && d0 < op.w3_off + (int64_t)op.w3_classes * op.w3_k);
  if (!in_w1 && !in_w2) return;
  const float4 v = *reinterpret_cast<const float4*>(rows + (int64_t)row * ld + d0);
  if (in_w1) store_op4(op, row, d0, v.x, v.y, v.z, v.w);
  if (in_w2) store_w2_4(op, row, d0, v.x, v.y, v.z, v.w);
}

// Coordinates k_to_operand covers: the first-layer block, and W2 (and W3) when copied.
inline int64_t op_span(const OpDesc& op) {
  int64_t end = op.w1_elems;
  if (op.w2 && op.w2_off + (int64_t)op.w2_classes * op.w2_h1 > end) end = op.w2_off + (int64_t)op.w2_classes * op.w2_h1;
  if (op.w3 && op.w3_off + (int64_t)op.w3_classes * op.w3_k > end) end = op.w3_off + (int64_t)op.w3_classes * op.w3_k;
  return end;
}

__global__ void k_f32_to_op(const float* __restrict__ src, int64_t n, int32_t kind, float inv, void* dst) {
  griddep_wait();
  griddep_launch_dependents();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    if (kind == kOpFp8)
      static_cast<uint8_t*>(dst)[e] = (uint8_t)__nv_cvt_float_to_fp8(src[e] * inv, __NV_SATFINITE, __NV_E4M3);
    else
      static_cast<__nv_bfloat16*>(dst)[e] = __float2bfloat16_rn(src[e]);
  }
}

inline unsigned blocks_for(int64_t n4) { return (unsigned)((n4 + kThreads - 1) / kThreads); }

}  // namespace

int launch_init(const Problem& p, float* fw_x, float* fw_amp, cudaStream_t s) {
  dim3 grid(blocks_for(p.Dp / 4), p.B * p.mu);
  k_init<<<grid, kThreads, 0, s>>>(p, fw_x, fw_amp);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_explode(const Problem& p, const uint32_t* gens_done, const float* fw_x, const float* fw_amp, float* sparks,
                   const OpDesc& op, cudaStream_t s) {
  dim3 grid((unsigned)((p.Dp / 4 + kExplodeBlocks * kThreads - 1) / (kExplodeBlocks * kThreads)), p.lam, p.B * p.mu);
  return launch_pdl(k_explode, grid, dim3(kThreads), 0, s, p, gens_done, fw_x, fw_amp, sparks, op) == cudaSuccess
             ? 1
             : -1;
}

int launch_guide(const Problem& p, const uint32_t* gens_done, const float* fw_x, const float* fw_amp, const float* sparks,
                 const int32_t* top, const int32_t* bottom, float* guides, const OpDesc& op_guides,
                 cudaStream_t s, const float* gv_in, float* gv_out) {
  dim3 grid(blocks_for(p.Dp / 4), p.m, p.B * p.mu);
  cudaError_t e;
  const int ku = gv_in ? 0 : p.k;  // given vectors: no row loads to unroll
  switch (ku) {
#define MG_GUIDE_K(K) \
  case K: e = launch_pdl(k_guide<K>, grid, dim3(kThreads), 0, s, p, gens_done, fw_x, fw_amp, sparks, top, bottom, \
                         gv_in, gv_out, guides, op_guides); break;
    MG_GUIDE_K(1) MG_GUIDE_K(2) MG_GUIDE_K(3) MG_GUIDE_K(4) MG_GUIDE_K(5) MG_GUIDE_K(6) MG_GUIDE_K(7) MG_GUIDE_K(8)
#undef MG_GUIDE_K
    default: e = launch_pdl(k_guide<0>, grid, dim3(kThreads), 0, s, p, gens_done, fw_x, fw_amp, sparks, top, bottom,
                            gv_in, gv_out, guides, op_guides);
  }
  return e == cudaSuccess ? 1 : -1;
}

int launch_to_operand(const float* rows, int64_t ld, int32_t count, const OpDesc& op, cudaStream_t s) {
  if (count <= 0 || op.kind == kOpNone) return 0;
  dim3 grid(blocks_for(op_span(op) / 4), count);
  k_to_operand<<<grid, kThreads, 0, s>>>(rows, ld, op);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_f32_to_op(const float* src, int64_t n, int32_t kind, float inv_scale, void* dst, cudaStream_t s) {
  if (n <= 0) return 0;
  const unsigned blocks = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_f32_to_op<<<blocks, 256, 0, s>>>(src, n, kind, inv_scale, dst);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mgfwa
