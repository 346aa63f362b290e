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
  CUtensorMap tmap_w2b; // pair kernel: BF16 W2 [P][16 or 32 (two layers) or h2][h1], box 64 x half the rows x 1,
                        // 128B swizzle
  CUtensorMap tmap_w3b; // pair kernel, three layers: BF16 W3 [P][16][h2], box 64 x 8 x 1
  CUtensorMap tmap_x3;  // pair kernel: X viewed as [K atoms][N][one 128-byte atom], box one atom x 128 x 2 atoms
  CUtensorMap tmap_wk;  // pair kernel: the first-layer operand viewed the same way, box one atom x half a tile x 2
  CUtensorMap tmap_xt;  // pair kernel: X, box one MMA's K (32 bytes) x 128, 32B swizzle (the partial last atom)
  CUtensorMap tmap_wt;  // pair kernel: the first-layer operand, box 32 bytes x half a tile's rows, 32B swizzle
  CUtensorMap tmap_x;   // X  [N][d_in], box 128 rows x 128 bytes of K, 128B swizzle
  CUtensorMap tmap_w;   // op [P*h1][d_in], box n_tile rows x 128 bytes of K, 128B swizzle
  CUtensorMap tmap_w2;  // W2 inside the FP32 spark rows [P][C or h2][h1], box 32 x rows x 1, 128B swizzle
  CUtensorMap tmap_w3;  // three layers: W3 [P][C][h2], box 32 x C x 1
  int num_sms = 0;
  int sparks_per_tile = 0;  // whole sparks per N-tile
  int n_tile = 0;           // accumulator columns per tile (sparks_per_tile * h1)
  int stages = 0;           // shared-memory pipeline depth
  size_t smem_bytes = 0;
  int tuned = 0;            // pair kernel: 1 if the tile shape and depth were chosen by timing
  int ktail = 0;            // pair kernel: MMAs of the partial last K atom taken through the K-tail buffers
                            // (their shared memory is reserved), 0 = the atom is a pipeline stage of its own
  const void* w_base = nullptr;  // pair kernel: the first-layer operand and its rows (for re-encoding W1's maps)
  int64_t w_rows = 0;
};

// True if the tensor-core path handles this network: d_in % 8 == 0 and
// either two linear layers with h1 in {32, 64, 128} and 2..32 classes, or
// three with (h1, h2) in {(128, 64), (64, 32)} and 2..16 classes.
bool tc_supported(const int32_t* widths, int n_layers);

// True if the CTA-pair kernel handles this network (d_in % 8 == 0): two
// linear layers with h1 in {64, 128} and 2..32 classes, or three with
// (h1, h2) = (128, 64) and 2..16 classes.  It needs the BF16 copy of W2
// (OpDesc::w2) with tc_pair_w2_rows rows per spark, and with three layers
// that of W3 (OpDesc::w3) with tc_pair_logit_rows(C) rows.
bool tc_pair_supported(const int32_t* widths, int n_layers);
int tc_pair_logit_rows(int C);
int tc_pair_w2_rows(const int32_t* widths, int n_layers);

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

// Arguments of one launch of the CTA-pair kernel (one handle's rows).
struct PairArgs {
  int32_t count;        // sparks in this launch
  int32_t first_spark;  // first spark row of the launch (operand tensor maps)
  int32_t m_pairs;      // 256-sample tiles
  int32_t m_tiles;      // 128-sample tiles (rows of `partial`)
  int32_t n_tiles;
  int32_t n_full;       // K atoms entirely inside d_in
  int32_t n_steps;      // K steps per tile: ceil(n_full / 2), plus one for a partial last atom
  int32_t k_last;       // layer-1 MMAs in the partial last atom (0 if d_in ends on an atom)
  int32_t kt;           // k_last when the partial atom may go through the K-tail buffers (some full atom
                        // before it), else 0; it does when kt <= kt_region of the launch
  int32_t kt_region;    // the launch's K-tail buffers (MMAs per buffer; 0 = none): the shared-memory layout
  int32_t stages;
  int32_t C;            // classes (<= NL)
  int32_t act;
  int32_t act2;         // three layers: the second hidden layer's activation
  int32_t c_pad;        // C rounded up to 4 (floats of the logits' bias copied)
  float scale;          // layer-1 accumulator multiplier (1 for BF16; 1 / (inv_x inv_w) for E4M3)
  int64_t N;
  int64_t ld;           // FP32 row stride of the sparks
  int64_t b1_off;
  int64_t b2_off;       // three layers: the second hidden layer's bias
  int64_t bl_off;       // the logits' bias
  const float* rows;    // FP32 spark rows of this launch (biases)
  const int32_t* y;
  float* partial;       // [m_tiles][count]
  uint32_t* status;
  uint64_t wait_budget; // clock64 ticks before a wait gives up (0 = the default)
};

// One member of a grouped launch: its tensor maps and arguments, in device
// memory, and where its tiles start among the launch's (aligned as the
// tensor maps require, which the array's allocation honours).
struct PairMember {
  CUtensorMap x3, x, w3, w, w2, wl3;  // wl3: the BF16 W3 copy (three layers)
  CUtensorMap xt, wt;                  // the partial last atom's loads through the K-tail buffers
  PairArgs a;
  int32_t tile_start, tiles;
};

// The member entry of one launch's worth of rows (as launch_fitness_tc would
// make them) of a handle on the pair kernel.
void tc_pair_member(const TcPlan& plan, const Mlp& mlp, int64_t first, const float* rows, int64_t ld, int32_t count,
                    float scale, float* partial, uint32_t* status, PairMember* out);
// True if two pair plans run the same kernel instance (h1, logit rows,
// operand type), so their launches can be grouped.
bool tc_pair_same_instance(const TcPlan& a, const Mlp& ma, const TcPlan& b, const Mlp& mb);
// One launch of the pair kernel over `n` members (table_dev: n entries in
// device memory, tile_start filled, laid end to end, total_tiles in all);
// `plan` gives the instance, shared-memory size and grid.  Returns 1, or -1
// after a launch error.
int launch_fitness_pair_group(const TcPlan& plan, const Mlp& mlp, const PairMember* table_dev, int32_t n,
                              uint32_t* status, cudaStream_t s, int32_t total_tiles);

// The CTA-pair kernel's pieces (k_fitness_pair.cu), used by tc_plan and
// launch_fitness_tc.  Sparks per tile: 256 / h1 when the logits share the
// sparks' columns, else 256 / (h1 + logit rows) (two layers only; 0 for
// three).
int tc_pair_sparks(const Mlp& mlp, bool shared);
size_t tc_pair_fixed_smem(const Mlp& mlp, int sparks_per_tile);
size_t tc_pair_stage_bytes(int h1, int sparks_per_tile);
// MMAs of the network's partial last K atom that the K-tail buffers can take
// (1 .. 3, with at least one full atom before it), else 0; and the shared
// memory of both K-tail buffers for `mmas` of them.
int tc_pair_ktail_mmas(const Mlp& mlp, bool f8);
size_t tc_pair_ktail_bytes(int h1, int sparks_per_tile, int mmas);
int tc_pair_max_stages();
// Deepest pipeline of the tile shape that fits the device's shared memory
// (`limit` bytes per block) beside K-tail buffers for `kt_mmas` MMAs, or 0
// if not even two stages fit.
int tc_pair_stages_fit(const Mlp& mlp, int sparks_per_tile, size_t limit, int kt_mmas = 0);

// Set a pair plan's tile shape, pipeline depth and K-tail buffers
// (re-encoding the W1 maps, whose box is half a tile's rows) and its
// kernel's attributes.  ktail: 1 = the partial last K atom through the
// K-tail buffers, 0 = as a stage of its own, -1 = the buffers where the
// network has such an atom and they fit beside the pipeline.  MGFWA_EINVAL
// for a shape the kernel does not have, a depth that does not fit, or
// ktail = 1 where the network has no such atom or the buffers do not fit.
// Every shape, depth and K-tail choice gives every spark bitwise the same
// fitness.
mgfwa_status tc_pair_configure(TcPlan& plan, const Mlp& mlp, int sparks_per_tile, int stages, int ktail = -1);
// Time every tile shape, depth and K-tail choice on `count` rows of the planned buffers
// (as launch_fitness_tc would run them, on stream s; `partial` is
// overwritten) and keep the fastest.  Choices are cached per device and
// problem shape for the process, so a second handle of the same shape
// times nothing.  Skipped (the plan's default stays) while s is capturing.
mgfwa_status tc_pair_tune(TcPlan& plan, const Mlp& mlp, const float* rows, int64_t ld, int32_t count, float scale,
                          float* partial, uint32_t* status, cudaStream_t s);
cudaError_t tc_pair_prepare(TcPlan& plan, const Mlp& mlp);
int launch_fitness_pair(const TcPlan& plan, const Mlp& mlp, int64_t first, const float* rows, int64_t ld,
                        int32_t count, float scale, float* partial, uint32_t* status, cudaStream_t s);

}  // namespace mgfwa
