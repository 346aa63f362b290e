// mgfwa_evaluate_fp32_noalloc: FP32 fitness of caller-owned device buffers
// without any device allocation.
//
// Some callers cannot call cudaMalloc: a host process whose device memory is
// owned and budgeted by another framework's allocator (every byte must come
// from that allocator or not at all), or a latency-critical loop where
// cudaMalloc / cudaFree may synchronise the whole device.  For them this
// entry point runs the FP32 fitness kernels with their scratch (the
// per-sample-tile partial sums of the cross-entropy) in a fixed array that
// lives in the library's own device image, so a call allocates nothing.
//
// That array is a file-scope __device__ object: every GPU on which the
// library's device code is loaded holds it (kScratchFloats floats = 1 MiB)
// until the process exits.  With CUDA's default lazy module loading the code
// is loaded on a device at its first use there (the first launch or symbol
// lookup), so the first call on a device may take device memory for it; it
// belongs in the caller's set-up.  Host code cannot use the array's name as a
// device address (in host code the name is a host-side stand-in); its device
// address is taken once per device with cudaGetSymbolAddress and cached per
// device ordinal, for the device's primary context.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "mgfwa.h"
#include "mgfwa_internal.cuh"

namespace {

// Partial sums, [sample tiles of 128][count]; every entry a call reads is
// written by the same call first, so nothing needs clearing between calls.
constexpr int64_t kScratchFloats = int64_t(1) << 18;
__device__ __align__(256) float g_noalloc_partial[kScratchFloats];

constexpr int kMaxDevices = 64;
float* g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up on
// the first call that runs on that device).
cudaError_t scratch_on_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = static_cast<float*>(p);
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

mgfwa_status reject(mgfwa_status st, const char* msg) {
  mgfwa::set_thread_error(msg);
  return st;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" MGFWA_API mgfwa_status mgfwa_evaluate_fp32_noalloc(int32_t n_layers, const int32_t* widths,
                                                              const int32_t* acts, int64_t n_samples,
                                                              const float* X_dev, const int32_t* y_dev,
                                                              const float* rows_dev, int64_t ld, int32_t count,
                                                              float* fitness_dev, void* cuda_stream) {
  mgfwa::set_thread_error("");
  if (n_layers < 2 || n_layers > 3 || !widths || !acts)
    return reject(MGFWA_EINVAL, "noalloc: need 2 or 3 layers with widths and activations");
  if (!X_dev || !y_dev || !rows_dev || !fitness_dev) return reject(MGFWA_EINVAL, "noalloc: null device pointer");
  if (n_samples < 1 || n_samples > mgfwa::kMaxSamples)
    return reject(MGFWA_EINVAL, "noalloc: n_samples must be in [1, 65535 * 128]");
  if (count < 1 || count > 65535) return reject(MGFWA_EINVAL, "noalloc: count must be in [1, 65535]");
  int64_t params = 0;
  for (int l = 0; l < n_layers; ++l) {
    if (widths[l] < 1 || widths[l + 1] < 1) return reject(MGFWA_EINVAL, "noalloc: layer widths must be >= 1");
    params += (int64_t)widths[l] * widths[l + 1] + widths[l + 1];
  }
  if (widths[0] % 8 != 0) return reject(MGFWA_EINVAL, "noalloc: d_in must be a multiple of 8");
  for (int l = 1; l < n_layers; ++l) {
    if (widths[l] > 192) return reject(MGFWA_EINVAL, "noalloc: hidden widths must be <= 192");
    if (acts[l - 1] != MGFWA_ACT_TANH && acts[l - 1] != MGFWA_ACT_RELU)
      return reject(MGFWA_EINVAL, "noalloc: unknown activation");
  }
  if (widths[n_layers] < 2 || widths[n_layers] > 32) return reject(MGFWA_EINVAL, "noalloc: class count must be in [2, 32]");
  if (ld < params || ld % 4 != 0) return reject(MGFWA_EINVAL, "noalloc: ld must be >= D and a multiple of 4");
  if (!aligned16(X_dev) || !aligned16(rows_dev)) return reject(MGFWA_EINVAL, "noalloc: X and rows must be 16-byte aligned");
  const int64_t mtiles = (n_samples + 127) / 128;
  if (mtiles * (int64_t)count > kScratchFloats) {
    char msg[160];
    snprintf(msg, sizeof(msg), "noalloc: ceil(n_samples/128) * count = %lld exceeds the fixed scratch of %lld floats",
             (long long)(mtiles * count), (long long)kScratchFloats);
    return reject(MGFWA_EINVAL, msg);
  }

  mgfwa::Mlp mlp = {};
  mlp.n_layers = n_layers;
  for (int l = 0; l <= n_layers; ++l) mlp.widths[l] = widths[l];
  for (int l = 0; l + 1 < n_layers; ++l) mlp.acts[l] = acts[l];
  int64_t off = 0;
  for (int l = 0; l < n_layers; ++l) {
    mlp.w_off[l] = off;
    off += (int64_t)widths[l] * widths[l + 1];
    mlp.b_off[l] = off;
    off += widths[l + 1];
  }
  mlp.N = n_samples;
  mlp.X = X_dev;
  mlp.y = y_dev;
  mlp.w1_elems = (int64_t)widths[0] * widths[1];

  float* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return reject(MGFWA_ECUDA, "noalloc: cudaGetSymbolAddress of the scratch array failed");
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (mgfwa::launch_fitness_simt_main(mlp, rows_dev, ld, count, scratch, s) < 0 ||
      mgfwa::launch_fitness_finish(scratch, (int32_t)mtiles, count, n_samples, fitness_dev, s) < 0) {
    cudaError_t e = cudaGetLastError();
    char msg[160];
    snprintf(msg, sizeof(msg), "noalloc: kernel launch failed: %s", cudaGetErrorString(e));
    return reject(MGFWA_ECUDA, msg);
  }
  return MGFWA_OK;
}
