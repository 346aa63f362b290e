// Gradient of the MLP cross-entropy for R search vectors (k_grad.cu) and
// the hybrid refinement's small kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fp32x3.cuh"
#include "mgfwa_internal.cuh"

namespace mgfwa {

// Scratch layout (float offsets into one device slice of `floats` floats)
// for R vectors of one MLP: per hidden layer l = 1..L-1 its activations
// and (with gradients) its dZ, the per-sample losses, and the split-K
// partials of the largest product.
struct GradPlan {
  int32_t R = 0;
  int32_t num_sms = 0;
  bool forward_only = false;  // objective only (no derivative buffers)
  int64_t act_off[4] = {};
  int64_t dz_off[4] = {};
  int64_t loss_off = 0;
  int64_t partial_off = 0;
  int64_t floats = 0;
};

GradPlan grad_plan(const Mlp& mlp, int32_t R, int32_t num_sms, bool forward_only = false);

// Forward pass of the R rows W (stride ld) on the batch; with G non-null
// also the gradient into G (same stride; padding untouched); with f_out
// non-null the FP32 objective of each row.  With idx, row r is W[idx[r]]
// and its objective goes to f_out[idx[r]] (objective only).  Returns
// kernels enqueued or -1.
// With l1 (a ready plan over the same rows W, stride ld), the first layer
// runs on the tensor cores at FP32 accuracy (status: its wait-timeout word).
// Whether launch_grad runs the first layer of this plan on the tensor cores:
// the plan over the rows is ready and its (128-sample tile, vector) pairs
// number at least half the SMs; fewer vectors keep the CUDA-core products,
// whose split-K gives every SM work.
bool l1_on_tensor_cores(const GradPlan& gp, const Mlp& mlp, const L1Plan* l1);

int launch_grad(const GradPlan& gp, const Mlp& mlp, const float* W, int64_t ld, float* scratch, float* G,
                float* f_out, cudaStream_t s, const int32_t* idx = nullptr, const L1Plan* l1 = nullptr,
                uint32_t* status = nullptr);

// w <- min(max(fma(-lr, g, w), lb), ub) on the first D coordinates of R rows.
int launch_sgd(float* w, const float* g, int32_t R, int64_t D, int64_t Dp, float lr, float lb, float ub,
               cudaStream_t s);

// Per run r: elite[r] = first minimum of fw_f[r*mu .. r*mu + mu), its row copied to w[r].
int launch_refine_pick(const float* fw_x, const float* fw_f, int32_t R, int32_t mu, int64_t Dp, float* w,
                       int32_t* elite, cudaStream_t s);

// Per run r: if fr[r] is strictly below the elite's fitness, the elite
// firework takes w[r] and fr[r]; the run's best-so-far likewise.  flags
// ([R] int32 device scratch) carries the decisions to the row copies.
int launch_refine_accept(const float* w, const float* fr, const int32_t* elite, int32_t* flags, float* fw_x,
                         float* fw_f, float* best_x, float* best_f, int32_t R, int32_t mu, int64_t Dp,
                         cudaStream_t s);

}  // namespace mgfwa
