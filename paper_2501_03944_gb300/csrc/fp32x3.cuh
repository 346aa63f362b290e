// FP32-accurate first layer on the tensor cores (k_fp32x3.cu): plan and
// launcher.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mgfwa_internal.cuh"

namespace mgfwa {

// Tensor maps over the FP32 batch X and over the first-layer weights of a
// buffer of FP32 rows (row stride ld floats, max_rows rows).
struct L1Plan {
  bool ready = false;
  CUtensorMap tmap_x;
  CUtensorMap tmap_w;
  const float* rows = nullptr;
  int64_t ld = 0;
};

// d_in % 4 == 0 and h1 in {32, 64, 128}.
bool l1_fp32x3_supported(const Mlp& mlp);

// False (plan not ready) when unsupported or not on a Blackwell GPU; the
// callers then use the CUDA-core products.
bool l1_fp32x3_plan(L1Plan& pl, const Mlp& mlp, const float* rows, int64_t ld, int64_t max_rows);

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

}  // namespace mgfwa
