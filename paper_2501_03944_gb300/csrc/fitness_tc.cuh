// Tensor-core (tcgen05, sm_103a) fitness path: plan and launcher.
#pragma once

#include <cuda.h>

#include "mgfwa.h"
#include "mgfwa_internal.cuh"

namespace mgfwa {

struct TcPlan {
  bool ready = false;
  bool f8 = false;      // E4M3 operands (else BF16)
  bool pair = false;    // the CTA-pair kernel (two layers, h1 in {64, 128}); else the one-CTA kernel
  int pairs = 0;        // CTA pairs resident at once (the pair kernel's persistent grid)
  uint64_t wait_budget = 0;  // clock64 ticks before a bounded wait gives up (0 = the kernels' default, ~2 s)
  CUtensorMap tmap_w2b; // pair kernel: BF16 W2 [P][16 or 32][h1], box 64 x half the rows x 1, 128B swizzle
  CUtensorMap tmap_x3;  // pair kernel: X viewed as [K atoms][N][one 128-byte atom], box one atom x 128 x 2 atoms
  CUtensorMap tmap_wk;  // pair kernel: the first-layer operand viewed the same way, box one atom x half a tile x 2
  CUtensorMap tmap_x;   // X  [N][d_in], box 128 rows x 128 bytes of K, 128B swizzle
  CUtensorMap tmap_w;   // op [P*h1][d_in], box n_tile rows x 128 bytes of K, 128B swizzle
  CUtensorMap tmap_w2;  // W2 inside the FP32 spark rows [P][C or h2][h1], box 32 x rows x 1, 128B swizzle
  CUtensorMap tmap_w3;  // three layers: W3 [P][C][h2], box 32 x C x 1
  int num_sms = 0;
  int sparks_per_tile = 0;  // whole sparks per N-tile
  int n_tile = 0;           // accumulator columns per tile (sparks_per_tile * h1)
  int stages = 0;           // shared-memory pipeline depth
  size_t smem_bytes = 0;
};

// True if the tensor-core path handles this network: d_in % 8 == 0 and
// either two linear layers with h1 in {32, 64, 128} and 2..32 classes, or
// three with (h1, h2) in {(128, 64), (64, 32)} and 2..16 classes.
bool tc_supported(const int32_t* widths, int n_layers);

// True if the CTA-pair kernel handles this network: two linear layers,
// h1 in {64, 128}, 2..32 classes, d_in % 8 == 0.  It needs the BF16 copy of
// W2 (OpDesc::w2) with tc_pair_logit_rows(C) rows per spark.
bool tc_pair_supported(const int32_t* widths, int n_layers);
int tc_pair_logit_rows(int C);

// Encode the tensor maps over the handle's X copy (mlp.Xop), first-layer
// operand (BF16 or E4M3, op.kind) and FP32 spark rows (`sparks`, row stride
// `ld`, `max_rows` rows).  E4M3 needs d_in % 16 == 0 (16-byte rows).
mgfwa_status tc_plan(TcPlan& plan, const Mlp& mlp, const OpDesc& op, const float* sparks, int64_t ld,
                     int64_t max_rows);
const char* tc_last_error();
// Give the plan's kernel its shared-memory allowance now (not at its first
// launch, which may be inside a stream capture).
cudaError_t tc_prepare(TcPlan& plan, const Mlp& mlp);
void tc_release(TcPlan& plan);

// Fitness of `count` sparks starting at spark row `first` of the planned
// buffers: per-(m-tile, spark) partial cross-entropy sums into
// partial[mtiles][count].  `rows` points at spark `first`'s FP32 row (stride
// ld).  The layer-1 accumulator is multiplied by `scale` before the bias
// (1 for BF16).  A device-side wait that gives up sets *status and returns.
int launch_fitness_tc(const TcPlan& plan, const Mlp& mlp, int64_t first, const float* rows, int64_t ld,
                      int32_t count, float scale, float* partial, uint32_t* status, cudaStream_t s);

// The CTA-pair kernel's pieces (k_fitness_pair.cu), used by tc_plan and
// launch_fitness_tc.
int tc_pair_sparks(int h1, int C);  // sparks per tile: floor(256 / (h1 + logit rows))
size_t tc_pair_fixed_smem(int h1, int C);
size_t tc_pair_stage_bytes(int h1, int C);
int tc_pair_max_stages();
cudaError_t tc_pair_prepare(TcPlan& plan, const Mlp& mlp);
int launch_fitness_pair(const TcPlan& plan, const Mlp& mlp, int64_t first, const float* rows, int64_t ld,
                        int32_t count, float scale, float* partial, uint32_t* status, cudaStream_t s);

}  // namespace mgfwa
