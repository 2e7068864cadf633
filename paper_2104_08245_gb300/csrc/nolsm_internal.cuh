// Internal declarations of the NOLSM GB300 library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nolsm.h"

namespace nolsm {


// Per-submatrix status codes written by kernels (values of nolsm_status).
enum : int32_t { kSubOk = 0, kSubNotSpd = NOLSM_ERR_NOT_SPD, kSubNotConv = NOLSM_ERR_NOT_CONVERGED,
                 kSubNonFinite = NOLSM_ERR_NONFINITE, kSubTimeout = NOLSM_ERR_TIMEOUT };

void set_error(const char* fmt, ...);

#define NOLSM_CUDA_TRY(expr)                                                                     \
  do {                                                                                           \
    cudaError_t _e = (expr);                                                                     \
    if (_e != cudaSuccess) {                                                                     \
      ::nolsm::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e));     \
      return _e == cudaErrorMemoryAllocation ? NOLSM_ERR_OOM : NOLSM_ERR_CUDA;                   \
    }                                                                                            \
  } while (0)

#define NOLSM_LAUNCH_CHECK() NOLSM_CUDA_TRY(cudaGetLastError())

#define NOLSM_TRY(expr)                 \
  do {                                  \
    nolsm_status _s = (expr);           \
    if (_s != NOLSM_OK) return _s;      \
  } while (0)

// Device buffer owned by the plan.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

// Geometry-dependent data of one precision class, computed once per plan (a1-a3 and the bounds).
struct Prepared {
  bool fp64 = false;          // true: A held in FP64 (plain path); false: FP32 (tensor-core paths)
  DevBuf A;                   // A_J = T_J(S)^-1 T_J(H0), n_J x n_J row-major at a_off[J]
  std::vector<uint8_t> done;  // host flag per submatrix: prepared
  // tensor-core preparations: a lower estimate of cond(T_J(S)), (max_i L_ii / min_i L_ii)^2 from the FP32
  // Cholesky factor, max_i S_ii (T_J(S)^-1)_ii from the inverse square root (float per submatrix, device
  // and host copies; huge when the FP32 preparation failed)
  DevBuf cond;
  std::vector<float> h_cond;
};

// Above this estimate the overlap is too ill-conditioned for the mode: A_J = T_J(S)^-1 T_J(H0) is then far
// from normal (its eigenvectors are T_J(S)-orthogonal, with condition number about sqrt(cond)), and the
// low-precision products' rounding, amplified by it, keeps the sign from the mode's accuracy (or from
// converging at all); such a submatrix is prepared and solved on the FP64 path instead. The FP32 mode
// (1e-6 target) takes cond <= 10, the other modes (1e-4) cond <= 30; the synthetic water overlaps have
// 1.06 to 1.3.
inline float cond_max(int precision) { return precision == NOLSM_FP32 ? 10.0f : 30.0f; }

}  // namespace nolsm

struct nolsm_plan {
  nolsm_system sys{};
  int32_t n_mol = 0;
  int64_t d_nnzb = 0, d_nvals = 0;
  int32_t max_n = 0, min_n = 0, max_b = 0;
  double sum_n3 = 0.0;
  int64_t bytes = 0;

  // integer maps (device)
  nolsm::DevBuf s_blk_off, h_blk_off;       // int64 [nnzb+1]
  nolsm::DevBuf nb_ptr, nb_idx, nb_off;     // int32
  nolsm::DevBuf sub_n, sub_c0;              // int32 [n_mol]
  nolsm::DevBuf sub_b;                      // int32 [n_mol]: centre columns of each submatrix (b_J; a group's
                                            // members' functions in a grouped plan)
  nolsm::DevBuf d_blk_off;                  // int64 [d_nnzb+1]
  nolsm::DevBuf d_slot;                     // int32 [d_nnzb]: slot of block (nb_idx[p], J) in D
  nolsm::DevBuf a_off, c_off;               // int64 [n_mol+1]: offsets of n^2 and n*b arrays
  nolsm::DevBuf flag;                       // int32 scratch flag

  // grouped plans (nolsm_build_grouped): the submatrices are groups of molecules; n_mol counts the groups,
  // sys.n_mol the molecules; D keeps the per-molecule pattern (d_slot, d_blk_off, d_nnzb of that plan)
  bool grouped = false;
  nolsm::DevBuf m_nb_ptr, m_nb_idx;         // int32: the per-molecule plan's N(J)
  nolsm::DevBuf g_of, g_col;                // int32 [molecules]: group of J, offset of J's columns in it
  nolsm::DevBuf g_row;                      // int32 [molecule pairs]: offset of the rows of I in T_G, G of J

  // elements generated on the device from the geometry (nolsm_plan_set_elements) instead of read
  bool gen = false;
  nolsm_element_model model{};
  nolsm::DevBuf onsite_off;                 // int64 [n_mol+1]: offsets of each molecule's on-site energies

  // host copies
  std::vector<int32_t> h_sub_n, h_nbf, h_nb_ptr;   // h_nbf: per molecule of the input system
  std::vector<int32_t> h_sub_b;                    // per submatrix
  std::vector<int64_t> h_a_off, h_c_off;

  // geometry caches shared by all precisions (device), n_J x b_J row-major at c_off[J]
  nolsm::DevBuf Q;        // centre columns of T_J(S)^-1 (FP64)
  nolsm::DevBuf Sc, Hc;   // centre columns of T_J(S), T_J(H0) (FP64)
  nolsm::DevBuf lam;      // float64 [2*n_mol]: Gershgorin interval of A_J
  nolsm::DevBuf prep_status;  // int32 [n_mol]: kSubOk or kSubNotSpd from the factorisation
  nolsm::Prepared prep64, prep32, prep_sym, prep_ns;
  nolsm::DevBuf Lsym;               // float32, FP32 factors of every submatrix at a_off (symmetric form)
  nolsm::DevBuf Wc;                 // float64, W_c = L^-1 E_c at c_off (symmetric form)

  // bound sources other than Gershgorin (bounds.cu)
  nolsm::DevBuf lam_p;              // float64 [2*n_mol]: power-iteration interval
  std::vector<uint8_t> pow_done;    // host flag per submatrix: lam_p computed (for pow_cls)
  int pow_cls = -1;
  nolsm::DevBuf onsite;             // float64 [2*n_mol]: sum and sum of squares of diag(H0_II)
  bool onsite_done = false;
  nolsm::DevBuf feat;               // float32 [n_mol*7]: features of the last features() call
  nolsm::DevBuf mlp_y;              // float32 [n_mol*3]: network outputs
  nolsm::DevBuf lam_m;              // float64 [2*n_mol]: learned interval
  nolsm::DevBuf budget;             // int32 [n_mol]: learned step budget
  nolsm::DevBuf rerun;              // int32 [n_mol + 1]: failed submatrices, then their count
  nolsm::DevBuf ill_list;           // int32 [n_mol]: submatrices a tensor-core solve hands to the FP64 path
  const nolsm_mlp* mlp = nullptr;   // network used by NOLSM_BOUND_MLP (caller-owned)

  // per-mu results
  nolsm::DevBuf Dc;                 // centre columns of T_J(D), FP64, at c_off[J]
  nolsm::DevBuf t_S, t_H;           // float64 [n_mol]
  nolsm::DevBuf iters, status;      // int32 [n_mol]
  nolsm::DevBuf rsteps;             // int32 [n_mol]: steps taken in the refinement format
  nolsm::DevBuf nbelow;             // int32 [n_mol]: eigenvalues below mu, (n - Tr sign) / 2 of the last solve
  nolsm::DevBuf nb_lo, nb_hi;       // int32 [n_mol]: the same at the ends of find_mu's bracket (-1: unknown)
  nolsm::DevBuf active;             // int32 [n_mol]: find_mu's submatrices with an eigenvalue in the bracket
  bool bisect_first = true;         // the next bisection point is the first (solves every submatrix)
  bool bisect_listed = false;       // the last point solved the work list (else the whole range)
  int32_t bisect_count = -1;        // submatrices the last point solved (-1: no point since the last side)
  double bisect_trace = 0.0;        // Tr(DS) of the last point
  nolsm::DevBuf sums;               // float64 [4]
  nolsm::DevBuf counter;            // int32 work counters of persistent kernels
  int64_t solved_begin = 0, solved_end = 0;
  int solved_cls = -1;              // preparation class of the last solve (kPrepFP64, kPrepMixed, kPrepSym)
  bool have_solution = false;
  nolsm::DevBuf Wd;                 // centre columns of T_J(W) (energy-weighted), FP64, at c_off[J]
  nolsm::DevBuf tW;                 // float64 [n_mol]: t_S of T_J(W)

  // workspaces
  nolsm::DevBuf ws_dense;           // gathered T_J(S), T_J(H0) of one preparation chunk (FP64)
  nolsm::DevBuf ws_l32;             // FP32 factors of one preparation chunk (low-precision paths)
  nolsm::DevBuf ws_refine;          // q as FP32 pairs and FP32 corrections of Q for one chunk
  nolsm::DevBuf prep_order;         // submatrices of one chunk, largest first (mixed preparation)
  nolsm::DevBuf ws_ysym;            // L^-1 T_J(H0) of one preparation chunk (symmetric form)
  nolsm::DevBuf ws_ns;              // per-CTA Newton-Schulz buffers (FP64 path)
  void* tc = nullptr;               // tensor-core path state (tc_path.cu)

  // tracing: accumulated stats and the events that time one ABI call's phases
  nolsm_stats stats{};
  cudaEvent_t ev[8] = {};
  bool ev_ok = false;
  std::vector<cudaEvent_t> pev;     // preparation chunks: before gather, after gather, after factorisation
  size_t pev_used = 0;
  std::vector<cudaEvent_t> tev;     // preparation chunks: around the tensor-core inverse kernel
  size_t tev_used = 0;

  ~nolsm_plan();
};

namespace nolsm {

nolsm_status dev_alloc(nolsm_plan* plan, DevBuf& b, size_t bytes);
void dev_free(nolsm_plan* plan, DevBuf& b);

// plan construction (plan_kernels.cu)
nolsm_status build_plan_device(nolsm_plan* plan, cudaStream_t st);

// per-geometry preparation and per-mu solve of the FP64 path (fp64_path.cu)
// Preparation classes: FP64 A (plain FP64 path), FP32 A = T_J(S)^-1 T_J(H0) (tensor-core paths), FP32
// symmetric form M = L^-1 T_J(H0) L^-T (E4M3, or any tensor-core mode on request).
// A fourth class holds FP32 A prepared by the tensor-core inverse square root (Eqs. inv1-inv3).
enum : int { kPrepFP64 = 0, kPrepMixed = 1, kPrepSym = 2, kPrepNS = 3 };
inline int prep_class(const nolsm_options& o) {
  if (o.precision == NOLSM_FP64) return kPrepFP64;
  if (o.precision == NOLSM_FP8E4M3 || o.symmetric_form) return kPrepSym;
  return o.inverse == NOLSM_INVERSE_NEWTON_SCHULZ ? kPrepNS : kPrepMixed;
}
inline Prepared& prepared(nolsm_plan* plan, int cls);
nolsm_status prepare(nolsm_plan* plan, int64_t j0, int64_t j1, int cls, cudaStream_t st);
// a4 scale of submatrix J at mu: alpha = max(hi - mu, mu - lo) of the bound source's interval, but not
// below 1/1.7 of the same from the Gershgorin interval [lg, hg], which contains the spectrum. Every
// eigenvalue of X_0 then lies in [-1.7, 1.7] inside (-sqrt(3), sqrt(3)), where the Newton-Schulz map
// keeps its sign and converges, whatever the learned or estimated interval says.
__host__ __device__ inline double scale_alpha(const double* lam, const double* lam_g, int J, double mu) {
  const double a = fmax(lam[2 * J + 1] - mu, mu - lam[2 * J]);
  const double ag = fmax(lam_g[2 * J + 1] - mu, mu - lam_g[2 * J]);
  return fmax(a, ag * (1.0 / 1.7));
}

// Scale source and work list of one solve: lam = interval per submatrix (Gershgorin, power or learned),
// budget = per-submatrix step cap (nullable); list/count = solve only list[0, count) instead of [j0, j1).
struct SolveSpec {
  const double* lam = nullptr;
  const int32_t* budget = nullptr;
  const int32_t* list = nullptr;
  int32_t count = 0;
};
nolsm_status solve_fp64(nolsm_plan* plan, double mu, const nolsm_options& o, int64_t j0, int64_t j1,
                        const SolveSpec& spec, cudaStream_t st);

nolsm_status ensure_results(nolsm_plan* plan);

// Times phases of one ABI call: mark(i) records event i on the stream; after the stream has been
// synchronised, elapsed(i, j) is the device time between marks i and j in ms (0 if unavailable).
void mark(nolsm_plan* plan, int i, cudaStream_t st);
double elapsed(nolsm_plan* plan, int i, int j);
// The same for the preparation's per-chunk events: pmark records the next one; after a synchronisation
// prep_times adds the gather and factorisation times to the stats and starts over.
void pmark(nolsm_plan* plan, cudaStream_t st);
// the same pairs around the tensor-core inverse kernel (prep_times adds them to ms_prep_tensor)
void tmark(nolsm_plan* plan, cudaStream_t st);
void prep_times(nolsm_plan* plan);

// shared epilogue: sum the per-submatrix traces of [j0, j1) (fp64_path.cu)
// (the work counters cover list[0, count) when list is set: the submatrices the call solved)
nolsm_status reduce_traces(nolsm_plan* plan, int64_t j0, int64_t j1, int terms_main, cudaStream_t st, double* tS,
                           double* tH, int32_t* first_bad_status, const int32_t* list = nullptr, int32_t count = 0);
// write-back of centre columns (default: those of T_J(D)) into the merged pattern
nolsm_status scatter(nolsm_plan* plan, double* D_vals, int64_t j0, int64_t j1, cudaStream_t st,
                     const double* src = nullptr);
// the same for a grouped plan: each member's columns of T_G(D) on the rows of its own N(J) (grouped.cu)
nolsm_status scatter_grouped(nolsm_plan* plan, double* D_vals, int64_t j0, int64_t j1, cudaStream_t st,
                             const double* src);
// centre columns of the energy-weighted T_J(W) at the plan's solution (energy_weighted.cu)
nolsm_status energy_weighted(nolsm_plan* plan, cudaStream_t st, double* W_vals, double* trace_WS);

}  // namespace nolsm

inline nolsm::Prepared& nolsm::prepared(nolsm_plan* plan, int cls) {
  return cls == kPrepFP64 ? plan->prep64
         : cls == kPrepSym ? plan->prep_sym
         : cls == kPrepNS  ? plan->prep_ns
                           : plan->prep32;
}
