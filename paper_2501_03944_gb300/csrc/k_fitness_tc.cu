// Tensor-core fitness path (placeholder until the tcgen05 kernel lands).
#include "fitness_tc.cuh"

namespace mgfwa {

bool tc_supported(const int32_t*, int) { return false; }
mgfwa_status tc_plan(TcPlan&, const Mlp&, const __nv_bfloat16*, int64_t) { return MGFWA_EINVAL; }
const char* tc_last_error() { return "tensor-core path not built"; }
void tc_release(TcPlan& plan) { plan.ready = false; }
int launch_fitness_tc(const TcPlan&, const Mlp&, int64_t, const float*, int64_t, int32_t, float*, uint32_t*,
                      cudaStream_t) {
  return -1;
}

}  // namespace mgfwa
