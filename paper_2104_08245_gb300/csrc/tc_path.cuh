// Tensor-core (tcgen05) sign-iteration path: declarations shared with the ABI layer.
#pragma once
#include "nolsm_internal.cuh"

namespace nolsm {

// a4-a7 for the low-precision modes on the FP32 A cache prepared by prepare_fp64(..., false).
nolsm_status solve_tc(nolsm_plan* plan, double mu, const nolsm_options& o, int64_t j0, int64_t j1, const SolveSpec& spec,
                      cudaStream_t st);

// products per Newton-Schulz product in the main phase of a precision (1 or 3)
int main_terms(int precision);

// a2-a3 by the coupled Newton-Schulz inverse square root on the tensor cores (Eqs. inv1-inv3), for the
// submatrices order[0, count) of one preparation chunk: T_J(S), T_J(H0) gathered in FP64 at ws +
// (a_off[J] - a_base) and chunk_n2 further; A_J (FP32) to Aout + a_off[J]; T_J(S)^-1 (FP32) to Xout +
// a_off[J] - a_base; prep_out[J] = kSubOk, or kSubRefine when the iteration did not reach tol_inv within
// max_inv steps (the FP64 preparation then takes the submatrix), or kSubTimeout.
struct NsInvArgs {
  const int32_t* order;         // largest first
  int32_t count;
  int32_t n_large;              // how many of them (a prefix of order) have n above 192
  int32_t max_n;
  const double* ws;
  int64_t a_base, chunk_n2;
  float* Aout;
  float* Xout;
  int32_t* prep_out;
  float tol_inv;
  int32_t max_inv;
};
nolsm_status launch_ns_inverse(nolsm_plan* plan, const NsInvArgs& a, cudaStream_t st);

// frees the tensor-core path's workspaces held by the plan
void tc_release(nolsm_plan* plan);

// launch shape chosen in this process for (mode 0 sign / 1 inverse, precision, bucket 0: n <= 192 / 1: n > 192):
// 0 or 1, or -1 while not measured
int tc_shape_choice(int mode, int precision, int bucket);

}  // namespace nolsm
