// FP32-accurate first layer on the tensor cores (k_fp32x3.cu): plan and
// launcher.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mgfwa_internal.cuh"

namespace mgfwa {

// The layer's operands as BF16 parts: X's three parts [3][N][d_in], made
// once (launch_l1_split_x), and the three parts of the W1 blocks of the
// vectors of one launch [max_rows][3][h1][d_in], made by each launch; tensor
// maps over both.  rows/ld: the FP32 rows the vectors come from.
struct L1Plan {
  bool ready = false;
  CUtensorMap tmap_xs;
  CUtensorMap tmap_ws;
  const float* rows = nullptr;
  int64_t ld = 0;
  uint32_t* xs = nullptr;
  uint32_t* ws = nullptr;
  int64_t max_rows = 0;
};

// d_in % 8 == 0 and h1 in {32, 64, 128}.
bool l1_fp32x3_supported(const Mlp& mlp);

// 32-bit words of the X parts and of the W1 parts of max_rows vectors (two
// BF16 per word).
int64_t l1_fp32x3_x_words(const Mlp& mlp);
int64_t l1_fp32x3_w_words(const Mlp& mlp, int64_t max_rows);

// False (plan not ready) when unsupported or not on a Blackwell GPU; the
// callers then use the CUDA-core products.
bool l1_fp32x3_plan(L1Plan& pl, const Mlp& mlp, const float* rows, int64_t ld, int64_t max_rows, uint32_t* xs,
                    uint32_t* ws);

// X -> its BF16 parts in the plan's buffer (once, after X is on the device).
int launch_l1_split_x(const L1Plan& pl, const Mlp& mlp, cudaStream_t s);

// out[r][n][j] = act(X[n] . W1_j + b1_j) of rows idx[r] (or r) of the
// planned buffer, r < R; FP32-accurate (split BF16 products).  With loss
// (two-layer nets with at most 32 classes, l1_fp32x3_fuses_output), the
// output layer runs in the same kernel instead: loss[r][n] is the sample's
// cross-entropy of the logits W2 a + b2, computed in the same order as the
// CUDA-core output layer, and out is not written.  A device wait that gives
// up sets *status.  Returns kernels enqueued or -1.
bool l1_fp32x3_fuses_output(const Mlp& mlp);
int launch_l1_fp32x3(const L1Plan& pl, const Mlp& mlp, const int32_t* idx, int32_t R, float* out, uint32_t* status,
                     cudaStream_t s, float* loss = nullptr);

// The testbed network on the tensor cores at FP32 accuracy (three BF16
// parts per operand, six products, three accumulators).  A layer runs there
// when fan_in % 8 == 0, fan_out >= 16 and fan_out is even (net_x3_layer);
// the others, among them the final 1-output layer, on the CUDA cores.
struct NetX3Plan {
  bool ready = false;
  bool tc[kNetMaxLayers] = {};
  CUtensorMap tmap_a[kNetMaxLayers];  // layer l's input parts [3][max_rows][fan_in] in act_parts[l & 1]
  CUtensorMap tmap_w[kNetMaxLayers];  // layer l's weight parts [3][fan_out][fan_in]
  uint32_t* act_parts[2] = {nullptr, nullptr};
  uint32_t* w_parts[kNetMaxLayers] = {};
  float* partial = nullptr;  // the split layers' partial sums [splits][max_rows][fan_out]
  int64_t max_rows = 0;
};
bool net_x3_layer(int fan_in, int fan_out);
// 32-bit words of the plan's buffers (two BF16 per word).
int64_t net_x3_words(const NetOut& net, int64_t max_rows);
// False (plan not ready) off a Blackwell GPU or when no layer qualifies.
bool net_x3_plan(NetX3Plan& pl, const NetOut& net, int64_t max_rows, uint32_t* buf);
// The weights -> their parts (once, after the parameters are on the device).
int launch_net_x3_split_w(const NetX3Plan& pl, const NetOut& net, cudaStream_t s);
// fit[r] = the network's output for spark row r < count (as
// launch_net_output, `scratch` [2][count][scratch_ld] FP32 for the CUDA-core
// layers).  A device wait that gives up sets *status.  Kernels or -1.
int launch_net_output_x3(const NetX3Plan& pl, const NetOut& net, const float* rows, int64_t ld, int32_t count,
                         float* fit, float* scratch, int64_t scratch_ld, uint32_t* status, cudaStream_t s);

}  // namespace mgfwa
