// Bound sources for a4 (power iteration, learned predictor) and the learned predictor's network (a10).
#pragma once
#include "nolsm_internal.cuh"

namespace nolsm {

constexpr int kFeatures = 7, kWidth = 128, kOutputs = 3;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kFeatures * kWidth;
constexpr int kOffW2 = kOffB1 + kWidth;
constexpr int kOffB2 = kOffW2 + kWidth * kWidth;
constexpr int kOffW3 = kOffB2 + kWidth;
constexpr int kOffB3 = kOffW3 + kWidth * kOutputs;
constexpr int kParams = kOffB3 + kOutputs;   // 17,923

struct PowArgs {
  int32_t j0;                 // first submatrix (range mode)
  const int32_t* list;        // or: submatrices by CTA (-1: none)
  const int32_t* sub_n; const int64_t* a_off; const int32_t* prep_status;
  const double* lam;          // Gershgorin interval
  double* lam_p;              // out: power-iteration interval
  int32_t iters;
};

struct FeatArgs {
  int32_t j0, j1;
  const int32_t* sub_n; const int32_t* nbf; const int32_t* nb_ptr; const int32_t* nb_idx;
  const double* lam; const double* onsite;
  double mu;
  float* feat;                // [n_mol][kFeatures]
};

// Power-iteration bounds for [j0, j1) (list == nullptr) or for list[0, count) on the A of a preparation class.
nolsm_status power_bounds(nolsm_plan* plan, int cls, int64_t j0, int64_t j1, const int32_t* list, int32_t count,
                          cudaStream_t st);
// Features of [j0, j1) at mu into plan->feat.
nolsm_status features(nolsm_plan* plan, double mu, int64_t j0, int64_t j1, cudaStream_t st);
// Learned interval and step budget of [j0, j1) from plan->feat with the plan's network.
nolsm_status mlp_bounds(nolsm_plan* plan, int64_t j0, int64_t j1, int32_t max_iter, cudaStream_t st);
// Training targets t [J][3] = (power lo, power hi, iters / 16) of [j0, j1) from the plan's last solve.
nolsm_status training_targets(nolsm_plan* plan, int64_t j0, int64_t j1, float* t, cudaStream_t st);
// Submatrices of [j0, j1) that failed the convergence test into plan->rerun; returns their number.
nolsm_status failed_list(nolsm_plan* plan, int64_t j0, int64_t j1, cudaStream_t st, int32_t* count);

}  // namespace nolsm
