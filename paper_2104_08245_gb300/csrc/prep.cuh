// Preparation kernels (prep_kernels.cu): arguments shared with the host driver in fp64_path.cu.
#pragma once
#include "nolsm_internal.cuh"

namespace nolsm {

// internal preparation status: the submatrix is prepared again with the FP64 factorisation
constexpr int32_t kSubRefine = 64;

struct PrepArgs {
  int32_t j0;                 // first submatrix of the chunk (one CTA per submatrix)
  const int32_t* order = nullptr;   // mixed preparation: CTA -> submatrix, largest first (null: j0 + CTA)
  const int32_t* sub_n; const int32_t* sub_c0; const int32_t* nbf;
  const int64_t* a_off; const int64_t* c_off;
  int64_t a_base;             // a_off of the chunk's first submatrix
  int64_t chunk_n2;           // offset of the gathered T_J(H0) half of the workspace
  double* ws;                 // gathered T_J(S) (factored in place) and T_J(H0)
  double* Q;                  // centre columns of T_J(S)^-1, n x b row-major at c_off
  double* lam;                // Gershgorin interval of A_J
  int32_t* prep_status;
  int32_t only_flagged = 0;   // k_prepare: take only submatrices the mixed preparation flagged
  // mixed preparation (low-precision paths)
  float* L32 = nullptr;       // FP32 factors, same offsets as ws (a_off - a_base)
  int64_t c_base = 0;         // c_off of the chunk's first submatrix
  float2* Qp = nullptr;       // q as hi + lo FP32 pairs for the residual, n x b at c_off - c_base
  float* W32 = nullptr;       // FP32 corrections of Q, n x b at c_off - c_base
  int32_t fallback_max_n = 0; // largest n the FP64 preparation takes (shared-memory panel)
  // symmetric form M = L^-1 T_J(H0) L^-T (mixed preparation only)
  int32_t sym = 0;
  float* Ysym = nullptr;      // L^-1 T_J(H0), same offsets as ws
  double* Wc = nullptr;       // W_c = L^-1 E_c, n x b at c_off (plan-wide)
  float* cond = nullptr;      // estimate of cond(T_J(S)) per submatrix (nullable), see Prepared::cond
};

// The symmetric form's finishing step: D_c = L^-T U (U left in Dc by the sign kernel), traces.
struct SymArgs {
  int32_t j0;
  const int32_t* list;        // or: submatrices by CTA
  const int32_t* sub_n; const int32_t* nbf; const int64_t* a_off; const int64_t* c_off;
  const int32_t* prep_status;
  const float* L;             // FP32 factors of every submatrix, at a_off
  const double* Sc; const double* Hc;
  double* Dc; double* tS; double* tH; int32_t* status;
};

// a2-a3 for `count` submatrices starting at g.j0 (largest dimension max_n); A in FP64 (fp64_A) or FP32.
nolsm_status launch_prepare(const PrepArgs& g, int count, int max_n, bool fp64_A, void* Acache, cudaStream_t st);
// The same with the FP32 factor and iterative refinement of Q (A in FP32), followed by the FP64
// preparation of the submatrices it flagged.
nolsm_status launch_prepare_mixed(const PrepArgs& g, int count, int max_n, float* Acache, cudaStream_t st);
// After the tensor-core inverse (launch_ns_inverse): the centre columns of T_J(S)^-1 refined with X =
// T_J(S)^-1 in g.L32, the Gershgorin interval of A_J, then the FP64 preparation of the flagged submatrices.
nolsm_status launch_ns_qrefine(const PrepArgs& g, int count, int max_n, int max_b, float* Acache, cudaStream_t st);
// Largest submatrix dimension the FP64 preparation takes.
int prepare_fp64_max_n();
nolsm_status launch_sym_finish(const SymArgs& g, int count, int max_n, int max_b, cudaStream_t st);

}  // namespace nolsm
