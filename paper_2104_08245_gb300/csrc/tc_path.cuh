// Tensor-core (tcgen05) sign-iteration path: declarations shared with the ABI layer.
#pragma once
#include "nolsm_internal.cuh"

namespace nolsm {

// a4-a7 for the low-precision modes on the FP32 A cache prepared by prepare_fp64(..., false).
nolsm_status solve_tc(nolsm_plan* plan, double mu, const nolsm_options& o, int64_t j0, int64_t j1, const SolveSpec& spec,
                      cudaStream_t st);

// products per Newton-Schulz product in the main phase of a precision (1 or 3)
int main_terms(int precision);

// frees the tensor-core path's workspaces held by the plan
void tc_release(nolsm_plan* plan);

}  // namespace nolsm
