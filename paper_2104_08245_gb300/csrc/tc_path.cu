#include "tc_path.cuh"

namespace nolsm {
nolsm_status solve_tc(nolsm_plan*, double, const nolsm_options&, int64_t, int64_t, cudaStream_t) {
  set_error("tensor-core path not built");
  return NOLSM_ERR_UNSUPPORTED;
}
void tc_release(nolsm_plan*) {}
}  // namespace nolsm
