/*
 * nolsm.h -- C ABI of the GB300 (sm_103a) hot path of the non-orthogonalised local submatrix method
 * (NOLSM), arXiv:2104.08245.
 *
 * The method approximates the density matrix of Eq. purification,
 *     D = 1/2 (I - sign(S^-1 H0 - mu I)) S^-1,
 * molecule by molecule: for each molecule J it builds dense submatrices T_J(S), T_J(H0) over the rows
 * where S or H0 is non-zero in J's columns (merged pattern, Sec. "The Non-Orthogonal Local Submatrix
 * Method"), evaluates Eq. purification_submatrix on them with the Newton-Schulz sign iteration
 * (Eq. NS1, NS2) after spectral rescaling, and writes the centre molecule's columns back into the
 * sparse D (Sec. "The Submatrix Method", step (iii)). mu is set by bisection so that Tr(DS) equals
 * the number of occupied orbitals (Sec. "Simulation Details").
 *
 * Conventions shared by every call:
 *  - Pointers marked (device) are CUDA device pointers owned by the caller; the library never frees
 *    them. Pointers marked (host) are ordinary host memory.
 *  - Work is enqueued on the caller's stream (NULL = legacy default stream). Calls that return host
 *    scalars synchronise that stream before returning.
 *  - Errors come back as nolsm_status codes; no call aborts, throws across the ABI or prints. After an
 *    error, nolsm_last_error() gives a one-line message (per thread). A CUDA error that corrupted the
 *    context is reported as NOLSM_ERR_CUDA and the plan must then be destroyed.
 *  - Per-submatrix outcomes (not SPD, not converged, non-finite) are reported in the optional device
 *    array `status` and summarised in the return code (the first such error by submatrix index wins).
 *  - Every device-side loop is bounded (iteration caps); no kernel waits without a limit.
 *  - One submatrix per molecule, indexed by the molecule index J = 0 .. n_mol-1.
 */
#ifndef NOLSM_H
#define NOLSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* nolsm_stream_t; /* a cudaStream_t */

typedef enum {
  NOLSM_OK = 0,
  NOLSM_ERR_ARG = 1,           /* invalid argument or malformed block-CSR input */
  NOLSM_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  NOLSM_ERR_OOM = 3,           /* device allocation failed */
  NOLSM_ERR_NOT_SPD = 4,       /* a Cholesky pivot of some T_J(S) was <= 0 */
  NOLSM_ERR_NOT_CONVERGED = 5, /* some sign iteration hit max_iter or missed tol_accept */
  NOLSM_ERR_NONFINITE = 6,     /* NaN/Inf met in some submatrix */
  NOLSM_ERR_NO_PLATEAU = 7,    /* find_mu: bracket narrowed below tol_mu with |Tr(DS)-N| > tol_n */
  NOLSM_ERR_UNSUPPORTED = 8,   /* option combination or size this build does not handle */
  NOLSM_ERR_NO_SOLUTION = 9,   /* scatter_density called before any solve_batch */
  NOLSM_ERR_TIMEOUT = 10       /* a bounded device-side wait gave up (the kernel returned early) */
} nolsm_status;

/* Arithmetic of the sign-iteration products (a5/a6). The trace sums are FP64 in every mode. The overlap
 * factorisation is FP64 in NOLSM_FP64; the tensor-core modes factor T_J(S) in FP32, form A_J with FP32
 * solves, and refine the centre columns of T_J(S)^-1 with a double-FP32 residual (about 48 bits) to about
 * 1e-12 relative; a submatrix whose refinement does not contract, or whose overlap is too ill-conditioned
 * for the FP32 factor, is prepared again with the FP64 factorisation.
 *   NOLSM_FP64       every step in FP64 on the CUDA cores (the plain reference path).
 *   NOLSM_FP32       every Newton-Schulz product as a three-term split of FP16 tensor-core products
 *                    (hi*hi + hi*lo + lo*hi, FP32 accumulation): about 22 significant bits.
 *   NOLSM_BF16       Newton-Schulz products as single BF16 tensor-core products (FP32 accumulation)
 *                    until tol_ns, then refine_steps steps in the NOLSM_FP32 arithmetic.
 *   NOLSM_BF16X3     three-term split BF16 products throughout (about 16 significant bits), then
 *                    refine_steps steps in the NOLSM_FP32 arithmetic.
 *   NOLSM_FP8E4M3    single E4M3 products (kind::f8f6f4, FP32 accumulation) on the symmetric form
 *                    (symmetric_form is implied), every operand scaled by 2^7, until the defect
 *                    reaches 0.1 (about twice the floor that E4M3 rounding of the iterate leaves) or
 *                    stops falling, then refine_steps (>= 1) steps in the NOLSM_FP32 arithmetic. The
 *                    E4M3 rounding of the iterates persists in D (max|dD| about 2e-3 on the synthetic
 *                    water systems); the traces stay within about 1e-6 relative.
 *   NOLSM_FP16       single FP16 tensor-core products (11 significant bits, FP32 accumulation) until
 *                    tol_ns, then refine_steps steps in the NOLSM_FP32 arithmetic: the cost of NOLSM_BF16
 *                    with three more bits per product. */
typedef enum {
  NOLSM_FP64 = 0,
  NOLSM_FP32 = 1,
  NOLSM_BF16 = 2,
  NOLSM_BF16X3 = 3,
  NOLSM_FP8E4M3 = 4,
  NOLSM_FP16 = 5
} nolsm_precision;

/* Source of the spectral scale alpha_J(mu) >= rho(A_J - mu I) applied before the sign iteration. */
typedef enum {
  NOLSM_BOUND_GERSHGORIN = 0, /* Gershgorin interval of A_J = T_J(S)^-1 T_J(H0) */
  NOLSM_BOUND_POWER = 1,      /* power-iteration estimates of the extreme eigenvalues, widened */
  NOLSM_BOUND_MLP = 2         /* the learned predictor (nolsm_mlp_*); fallback: power iteration */
} nolsm_bound_source;

/* Sparse input. S and H0 are symmetric; each is stored block-CSR over molecules: block row I lists,
 * in strictly ascending order, the molecules J with a stored block (I, J); block (I, J) holds
 * nbf[I] x nbf[J] float64 values row-major; blocks are concatenated in CSR order. The two patterns
 * may differ (their union is the merged pattern); each must be structurally symmetric. All arrays
 * are device memory owned by the caller and must stay valid and unchanged until the plan built from
 * them is destroyed. s_vals and h_vals may be NULL when the plan's elements are generated on the device
 * from the geometry (nolsm_plan_set_elements): the patterns alone are then the metadata. */
typedef struct {
  int32_t n_mol;
  const int32_t* nbf;       /* (device) [n_mol], basis functions per molecule, 1..64 */
  int64_t s_nnzb;
  const int32_t* s_row_ptr; /* (device) [n_mol+1] */
  const int32_t* s_col_idx; /* (device) [s_nnzb] */
  const double* s_vals;     /* (device) [sum over blocks of nbf[I]*nbf[J]] */
  int64_t h_nnzb;
  const int32_t* h_row_ptr; /* (device) [n_mol+1] */
  const int32_t* h_col_idx; /* (device) [h_nnzb] */
  const double* h_vals;     /* (device) */
} nolsm_system;

typedef struct {
  int32_t precision;     /* nolsm_precision */
  int32_t refine_steps;  /* steps after the low-precision phase (ignored by FP64); while the last of
                            them still lowers the defect without reaching tol_accept, the iteration
                            goes on (up to max_iter) */
  int32_t max_iter;      /* cap on Newton-Schulz steps per submatrix (all phases) */
  double tol_ns;         /* the low-precision (or FP64) phase ends after the step whose defect
                            ||I - X_k^2||_F / sqrt(n) is <= tol_ns */
  double tol_accept;     /* the final X must have defect <= tol_accept, else NOT_CONVERGED */
  double tol_n;          /* find_mu: accept |Tr(DS) - N_occ| <= tol_n * N_occ */
  double tol_mu;         /* find_mu: stop when the bracket is narrower than this (Ha) */
  int32_t max_bisect;    /* find_mu: cap on evaluations */
  int32_t bound_source;  /* nolsm_bound_source */
  int64_t sub_begin;     /* solve only submatrices [sub_begin, sub_end) (streaming); */
  int64_t sub_end;       /* sub_end <= 0 means n_mol */
  int32_t symmetric_form;/* tensor-core modes: iterate on M = L^-1 T_J(H0) L^-T (T_J(S) = L L^T), which has
                            the spectrum of A_J and symmetric iterates, and finish with T_J(D) =
                            L^-T 1/2 (I - sign(M - mu I)) L^-1 (Eq. purification_submatrix); always used by
                            NOLSM_FP8E4M3 (every operand is then loaded in the K-major layout) */
  int32_t inverse;       /* tensor-core modes, standard form: how A_J = T_J(S)^-1 T_J(H0) is prepared.
                            NOLSM_INVERSE_CHOLESKY: FP32 Cholesky factor and FP32 solves.
                            NOLSM_INVERSE_NEWTON_SCHULZ: the coupled Newton-Schulz iteration for the inverse
                            square root of Sec. "Efficient Iterative Matrix Function Solvers on GPU Tensor
                            Cores" (Eqs. inv1-inv3) on the tensor cores (three-term FP16 split products),
                            T_J(S)^-1 = Z^2 / c and A_J = T_J(S)^-1 T_J(H0) as two more products; the step whose
                            ||I - Z_k Y_k||_F / sqrt(n) <= 1e-3 is the last. Either way the centre columns of
                            T_J(S)^-1 are refined to about 1e-12 with a double-FP32 residual, and a submatrix
                            that fails is prepared again with the FP64 factorisation. Ignored by NOLSM_FP64 and
                            the symmetric form (which keep the Cholesky factor). */
  int64_t wait_ns;       /* tensor-core sign kernel: limit of each device-side wait of one warp role on another
                            (a product's operands, its accumulator, the next descriptor), in ns; <= 0: 2 s. A
                            wait that runs out ends the kernel early: the submatrices in flight and those not
                            yet taken report NOLSM_ERR_TIMEOUT (a small limit makes that happen on purpose) */
} nolsm_options;

enum { NOLSM_INVERSE_CHOLESKY = 0, NOLSM_INVERSE_NEWTON_SCHULZ = 1 };

/* Defaults for a precision: FP64 tol_ns 1e-9, tol_accept 1e-7, max_iter 100; low-precision modes
 * tol_ns 1e-2, refine_steps 2 (FP8: 3), tol_accept 1e-4; tol_n 1e-5 (relative), tol_mu 1e-10,
 * max_bisect 100, Gershgorin bounds, all submatrices. */
void nolsm_options_default(nolsm_options* opts, int32_t precision);

/* A plan owns all its device workspaces. They come from the device's default stream-ordered memory pool
 * (cudaMallocAsync), whose release threshold the library raises once per device so that freed pages
 * stay in the pool for the next plan (a plan per geometry then maps no new pages); allocations and
 * releases complete before the calls return. If an allocation fails, the pool is trimmed and the
 * allocation retried once. */
typedef struct nolsm_plan nolsm_plan; /* opaque */

typedef struct {
  int32_t n_mol;       /* = number of submatrices */
  int64_t d_nnzb;      /* blocks of D in the merged pattern */
  int64_t d_nvals;     /* float64 values of D */
  int32_t max_n;       /* largest submatrix dimension n_J */
  int32_t min_n;       /* smallest n_J */
  double sum_n3;       /* sum over J of n_J^3 (work metric) */
  int64_t device_bytes;/* device memory currently held by the plan */
  int64_t nb_entries;  /* entries of nb_idx / nb_off (nolsm_plan_get_maps): d_nnzb, or for a grouped plan the
                          total length of its groups' row lists */
  int32_t grouped;     /* 1 for a plan from nolsm_build_grouped (n_mol then counts its groups) */
} nolsm_plan_info;

/* a0: submatrix construction plan (Sec. "The Non-Orthogonal Local Submatrix Method", merged pattern;
 * Sec. "The Submatrix Method", step (i); molecule-coalesced columns, Sec. "Simulation Details").
 * Builds, on the device, N(J) = {I : block (I,J) stored in S or in H0} in ascending order, the local
 * offsets of each molecule inside T_J, n_J, the offset of J's own columns, the slot of every block
 * (I, J) in the merged pattern (used by the write-back) and the grouping of submatrices by size.
 * Checks the input (sorted, in range, structurally symmetric); returns NOLSM_ERR_ARG if malformed.
 * On success *out owns device memory until nolsm_plan_destroy. Synchronises the stream. */
nolsm_status nolsm_build_submatrices(const nolsm_system* sys, nolsm_stream_t stream, nolsm_plan** out);

nolsm_status nolsm_plan_query(const nolsm_plan* plan, nolsm_plan_info* info);

/* Matrix elements generated on the device (Sec. "Minimization of Communication": only the submatrices' row
 * indices, species and positions reach the GPU, and the elements of the submatrices are computed there). The
 * plan's block patterns say which blocks exist; their values come from the synthetic water-like model of
 * this library's benchmarks (the paper's GFN-xTB element formulas are not part of this work): for molecules
 * I != J with a stored block and minimum-image vector d from I to J, r = |d|, every entry (a, c) is
 *   S_IJ[a][c] = exp(-s_exp r^2) / sqrt(b_I b_J) * (1 + aniso (u_a - u_c)),
 *   H_IJ[a][c] = hop exp(-r / hop_len) / sqrt(b_I b_J) * (1 + aniso (w_a - w_c)),
 * with u_a = (d / r) . dirs[0][a], w_a = (d / r) . dirs[1][a] (only when aniso != 0); the diagonal blocks are
 * S_II = identity and H_II = diag(onsite of I). Computed in FP64 (the paper uses FP32 for its special-function
 * units; here the FP64 path's 1e-9 parity needs the elements to FP64 rounding).
 *   pos (device, [n_mol][3], Angstrom), cell (host, 3 periodic edges), onsite (device, [sum of nbf]: the
 *   on-site energies of each molecule's functions, molecules in order), dirs (device, [2][64][3], read only
 *   when aniso != 0; may be NULL otherwise). The arrays must stay valid until the plan is destroyed.
 * After this call every preparation generates T_J(S), T_J(H0) (and the centre columns) from the model instead
 * of reading s_vals / h_vals; geometry caches prepared before are discarded. NOLSM_ERR_ARG on NULL pointers
 * or non-positive cell edges. */
typedef struct {
  const double* pos;
  double cell[3];
  const double* onsite;
  double s_exp;
  double hop, hop_len;
  double aniso;
  const double* dirs;
} nolsm_element_model;

nolsm_status nolsm_plan_set_elements(nolsm_plan* plan, const nolsm_element_model* model);

/* Copies the plan's integer maps into caller device buffers (any pointer may be NULL):
 * nb_ptr [n_mol+1], nb_idx [nb_entries], nb_off [nb_entries], sub_n [n_mol], sub_c0 [n_mol],
 * d_blk_off [d_nnzb+1] (int64 element offsets of the D blocks). The merged pattern of D is
 * block row I = nb_idx[nb_ptr[I] .. nb_ptr[I+1]) of a per-molecule plan. For a grouped plan the first five
 * describe its groups (rows of T_G in order, members first) and d_blk_off the per-molecule pattern of D. */
nolsm_status nolsm_plan_get_maps(const nolsm_plan* plan, int32_t* nb_ptr, int32_t* nb_idx, int32_t* nb_off,
                                 int32_t* sub_n, int32_t* sub_c0, int64_t* d_blk_off, nolsm_stream_t stream);

/* The geometry caches of a1-a3 for the options' range and preparation (precision, symmetric_form,
 * inverse), prepared first if needed, copied to caller device buffers (either may be NULL): A (float32,
 * or float64 for NOLSM_FP64; A_J = T_J(S)^-1 T_J(H0) row-major n_J x n_J at element offset a_off[J], the
 * symmetric form's M_J = L^-1 T_J(H0) L^-T instead) and Q (float64, the centre columns of T_J(S)^-1, n_J x
 * b_J row-major at c_off[J]), where a_off and c_off are the exclusive prefix sums of n_J^2 and n_J b_J over
 * J = 0 .. n_mol-1 (only the range's entries are written). prep_status (device int32 [n_mol], may be NULL):
 * NOLSM_OK or NOLSM_ERR_NOT_SPD per submatrix. cond_est (device float [n_mol], may be NULL; tensor-core modes
 * with the standard form only, else left untouched): a lower estimate of cond(T_J(S)), (max_i L_ii /
 * min_i L_ii)^2 of the FP32 Cholesky factor or max_i S_ii (T_J(S)^-1)_ii after the inverse square root (about
 * 3.4e38 where the FP32 preparation failed). A tensor-core solve hands every submatrix whose estimate exceeds
 * 10 (NOLSM_FP32) or 30 (the other tensor-core modes) to the FP64 path before its own solve, and after it
 * every submatrix that failed the low-precision accept test or turned non-finite; nolsm_stats.ill_conditioned
 * counts them. Only submatrices of at most 775 rows (the FP64 factorisation's shared-memory panel) are
 * handed over; larger ones above the limit stay in the requested mode and nolsm_stats.ill_conditioned_kept
 * counts them. Synchronises the stream. */
nolsm_status nolsm_plan_get_prepared(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream, void* A,
                                     double* Q, int32_t* prep_status, float* cond_est);

/* Merged submatrices on the device (Sec. "Submatrix Combination Heuristics"): a new plan whose submatrices
 * are groups of molecules, e.g. the groups of nolsm_combine_submatrices. group_of (host, [n_mol] of the
 * per-molecule plan mp): a label per molecule, molecules with equal labels forming one group (any labels in
 * 0 .. n_mol-1; groups are numbered in the order of their smallest member). The submatrix of group G has the
 * rows of N(G), the union of its members' N(J): the members first (ascending), then the other molecules
 * (ascending); its centre columns are the members' functions (sub_c0 = 0, width the sum of their b_J).
 * Everything that works on submatrices then works on the groups (nolsm_solve_batch, nolsm_find_mu with its
 * options' range counting groups, bound sources, nolsm_energy_weighted); nolsm_scatter_density writes member
 * J's columns of T_G(D) on the rows of its own N(J), so that D keeps mp's pattern (d_blk_off, d_nvals). The
 * new plan shares mp's input arrays (and its element model, if set) and owns its own maps; mp may be
 * destroyed afterwards. Host work O(sum over groups of |N(G)| log |N(G)|); synchronises the stream.
 * NOLSM_ERR_ARG for a label outside 0 .. n_mol-1 or a grouped mp; NOLSM_ERR_UNSUPPORTED when a group has more
 * than 64 centre columns (the preparation's column tiles; split such a group). */
nolsm_status nolsm_build_grouped(const nolsm_plan* mp, const int32_t* group_of, nolsm_stream_t stream, nolsm_plan** out);

/* a1-a7: every submatrix J in [sub_begin, sub_end) at chemical potential mu:
 *   T_J(S), T_J(H0) gathered (a1); T_J(S) = L L^T in FP64 (a2); A_J = T_J(S)^-1 T_J(H0) (a3);
 *   X_0 = (A_J - mu I)/alpha_J (a4, Sec. rescaling before Eq. NS1); X <- 1/2 X (3I - X^2) (a5/a6,
 *   Eq. NS1) until the defect test passes; centre columns of
 *   T_J(D) = 1/2 (I - X) T_J(S)^-1 (a7, Eq. purification_submatrix) and the partial traces
 *   t_S(J) = sum_{j centre, i} T_J(D)_ij T_J(S)_ij and t_H(J) likewise with H0 (Eq. e_elec).
 * Steps a1-a3 depend only on the geometry and run once per plan and precision class; later calls
 * at other mu reuse them. Outputs (any may be NULL):
 *   trace_DS, trace_DH (host): FP64 sums of t_S, t_H over the range;
 *   sub_t_S, sub_t_H (device, [n_mol] float64): per-submatrix partial traces (range entries written);
 *   iters (device, [n_mol] int32): Newton-Schulz steps taken; status (device, [n_mol] int32):
 *   per-submatrix nolsm_status. The centre columns are kept in the plan for nolsm_scatter_density.
 * Synchronises the stream. */
nolsm_status nolsm_solve_batch(nolsm_plan* plan, double mu, const nolsm_options* opts, nolsm_stream_t stream,
                               double* trace_DS, double* trace_DH, double* sub_t_S, double* sub_t_H,
                               int32_t* iters, int32_t* status);

/* a8: write-back (Sec. "The Submatrix Method", step (iii)): block (I, J) of D, for I in N(J), is set
 * to the rows of I in the centre columns of T_J(D) from the most recent nolsm_solve_batch. D_vals
 * (device, float64 [d_nvals]) is laid out in the merged pattern with offsets d_blk_off (see
 * nolsm_plan_get_maps); blocks of submatrices outside the last solved range are left untouched. */
nolsm_status nolsm_scatter_density(nolsm_plan* plan, double* D_vals, nolsm_stream_t stream);

/* Energy-weighted density matrix (NOLSM section: W = D H0 D, for the Pulay forces; submatrix form
 * T_J(W) = T_J(D) T_J(H0) T_J(D)) for the submatrices of the most recent solve (nolsm_solve_batch,
 * nolsm_bisect_point or nolsm_find_mu), at the solution the plan holds. The centre columns are
 * evaluated as W_c = A_J D_c with A_J = T_J(S)^-1 T_J(H0): the projector 1/2 (I - sign(A_J - mu I)) commutes
 * with A_J and is idempotent, so T_J(D) T_J(H0) T_J(D) = A_J T_J(D). The FP64 path multiplies in FP64; the
 * tensor-core paths multiply their FP32 A_J by D_c rounded to FP32 with FP32 accumulation.
 *   W_vals (device, float64 [d_nvals], may be NULL): block (I, J) of W, for I in N(J), set to the rows of I
 *     in the centre columns of T_J(W), laid out like D (nolsm_scatter_density); blocks of submatrices
 *     outside the last solved range are left untouched.
 *   trace_WS (host, may be NULL): sum over J of sum_{j centre, i} T_J(W)_ij T_J(S)_ij, the submatrix
 *     approximation of Tr(W S) = Tr(D H0) (Eq. e_elec) for the full matrices.
 * NOLSM_ERR_NO_SOLUTION before any solve; NOLSM_ERR_UNSUPPORTED when the last solve used the symmetric
 * form (NOLSM_FP8E4M3 or symmetric_form = 1), which does not keep A_J. Synchronises the stream. */
nolsm_status nolsm_energy_weighted(nolsm_plan* plan, nolsm_stream_t stream, double* W_vals, double* trace_WS);

/* Submatrix combination heuristic (Sec. "Submatrix Combination Heuristics", Eq. combination_criterion),
 * a host-side planning step: no device work and no CUDA call (the paper runs it once on a CPU node and
 * reuses the result). Submatrices i, j of dimensions n_i, n_j with n_c rows in common merge into one of
 * n_i + n_j - n_c rows iff (n_i + n_j - n_c)^3 < n_i^3 + n_j^3. Start: one submatrix per molecule J with rows
 * N(J); a group's candidates are the groups owning a molecule among its rows; a sweep lists every ordered
 * pair (i, j) passing the criterion with its level n_j - n_c and gain n_i^3 + n_j^3 - (n_i + n_j - n_c)^3,
 * takes the pairs by level ascending, gain descending, i, j ascending, and merges a pair when neither
 * group merged earlier in that sweep; sweeps repeat until one merges nothing. Dimensions count basis
 * functions; the cubes are exact 128-bit integers, so the result does not depend on `threads`.
 *   n_mol; nbf (host, [n_mol], >= 1); nb_ptr (host, [n_mol+1]), nb_idx (host, [nb_ptr[n_mol]]): N(J) of
 *     every J, strictly ascending, J in N(J), the relation symmetric (as nolsm_plan_get_maps returns it);
 *   threads: host threads that list the candidate pairs (<= 0: the hardware's count, at most 64).
 *   group_of (host, [n_mol]): each molecule's group, named by its smallest member; n_groups (host);
 *   metrics (host, [4], may be NULL): sum of n^3 before and after, sum of n^2 before and after (the
 *     cubic work metric and the quadratic element metric); sweeps (host, may be NULL).
 * NOLSM_ERR_ARG on a NULL pointer or a malformed pattern (nothing written). */
nolsm_status nolsm_combine_submatrices(int32_t n_mol, const int32_t* nbf, const int32_t* nb_ptr, const int32_t* nb_idx,
                                       int32_t threads, int32_t* group_of, int32_t* n_groups, double* metrics,
                                       int32_t* sweeps);

/* a9: chemical potential by bisection (Sec. "Simulation Details"): f(mu) = Tr(DS) - n_occ with
 * Tr(DS) over the options' range (a point solves only the submatrices with an eigenvalue left in the
 * bracket, see nolsm_bisect_point); mu = (lo+hi)/2; f < 0 raises lo, otherwise
 * hi is lowered; stops at the first |f| <= tol_n * n_occ (NOLSM_OK), when hi - lo <= tol_mu
 * (NOLSM_ERR_NO_PLATEAU) or after max_bisect evaluations (NOLSM_ERR_NO_PLATEAU). If lo >= hi the
 * bracket is the union of the Gershgorin intervals of all A_J in the range (prepared first). The plan
 * keeps the solution at the returned mu for nolsm_scatter_density. mu_history (host, may be NULL) receives up
 * to max_bisect evaluated mu values. */
nolsm_status nolsm_find_mu(nolsm_plan* plan, double n_occ, double lo, double hi, const nolsm_options* opts,
                           nolsm_stream_t stream, double* mu_out, double* trace_DS_out, int32_t* steps_out,
                           double* mu_history);

/* The bisection of nolsm_find_mu one point at a time, for callers that drive it themselves (several
 * ranks summing Tr(DS) per point). Each point solves only the submatrices that can change inside the
 * bracket: a submatrix whose count of eigenvalues below mu, (n - Tr sign(A_J - mu I)) / 2, is the same
 * at both ends of the bracket has no eigenvalue inside, so its centre columns and traces from its last
 * solve hold for every mu in the bracket.
 * nolsm_bisect_begin: starts a bisection over the options' range; bracket_contains_spectrum = 1 when
 *   the bracket holds every eigenvalue of every submatrix of the range (then the counts at its ends are
 *   0 and n; a Gershgorin bracket from nolsm_spectral_bracket does), 0 when unknown.
 * nolsm_bisect_point: one point mu (inside the current bracket): solves the submatrices that can change
 *   (all of them at the first point) and returns Tr(DS) over the range (host) and how many submatrices
 *   it solved (host, may be NULL). The plan keeps the solution for nolsm_scatter_density.
 * nolsm_bisect_side: after a point, records that it becomes the bracket's lower end (raises_lo = 1, when
 *   Tr(DS) summed over all ranks is below n_occ) or its upper end (0). */
nolsm_status nolsm_bisect_begin(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream,
                                int32_t bracket_contains_spectrum);
nolsm_status nolsm_bisect_point(nolsm_plan* plan, double mu, const nolsm_options* opts, nolsm_stream_t stream,
                                double* trace_DS, int32_t* solved);
nolsm_status nolsm_bisect_side(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream, int32_t raises_lo);

/* The bisection rule itself (Sec. "Simulation Details": mu by bisection for charge neutrality) as host
 * arithmetic only: no CUDA call, no plan, callable without a GPU. nolsm_find_mu and callers that sum
 * Tr(DS) over several ranks take every decision through these two calls, so all of them visit the same
 * points.
 * nolsm_bisection_start: bracket [lo, hi] (host scalars, lo < hi) for n_occ occupied orbitals; sets
 *   mu = (lo + hi) / 2, steps = 0, state = NOLSM_BISECT_EVALUATE. NOLSM_ERR_ARG on non-finite input or
 *   lo >= hi.
 * nolsm_bisection_update: after the point at b->mu with the total Tr(DS) there (summed over every rank's
 *   submatrices): steps += 1, f = trace_DS - n_occ; |f| <= tol_n |n_occ| accepts mu (state
 *   NOLSM_BISECT_ACCEPTED); otherwise mu becomes the bracket's lower end when f < 0 (*raises_lo = 1),
 *   else its upper end (*raises_lo = 0; pass it to nolsm_bisect_side), and the bisection stops (state
 *   NOLSM_BISECT_NO_PLATEAU) when hi - lo <= tol_mu or steps >= max_bisect (100 when <= 0), or goes on
 *   at the new midpoint (state NOLSM_BISECT_EVALUATE, mu updated). raises_lo (host) may be NULL. */
enum { NOLSM_BISECT_ACCEPTED = 0, NOLSM_BISECT_EVALUATE = 1, NOLSM_BISECT_NO_PLATEAU = 2 };
typedef struct {
  double lo, hi;      /* current bracket */
  double mu;          /* the point to evaluate next (EVALUATE) or the last one evaluated */
  double n_occ;       /* target Tr(DS) */
  double trace_DS;    /* total Tr(DS) at the last evaluated point */
  int32_t steps;      /* points evaluated */
  int32_t state;      /* NOLSM_BISECT_* */
} nolsm_bisection;

nolsm_status nolsm_bisection_start(nolsm_bisection* b, double n_occ, double lo, double hi);
nolsm_status nolsm_bisection_update(nolsm_bisection* b, double trace_DS, const nolsm_options* opts,
                                    int32_t* raises_lo);

/* The union [lo, hi] of the Gershgorin intervals of A_J = T_J(S)^-1 T_J(H0) over the options' range
 * of submatrices (prepares a1-a3 for the range first): a bracket of every submatrix eigenvalue, used
 * as the default bisection bracket (Sec. "Simulation Details" gives no bracket). lo, hi: host. */
nolsm_status nolsm_spectral_bracket(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream, double* lo,
                                    double* hi);

/* Accumulated per-phase device times (CUDA events on the caller's stream) and work counters of a
 * plan since it was built or last reset; no paper counterpart (the paper times the whole method and
 * counts 2 n^3 per product, Sec. "FLOPs in the NOLSM method"). */
typedef struct {
  double ms_plan;              /* a0 */
  double ms_prepare;           /* a1-a3: gather, FP64 Cholesky, solves, bounds */
  double ms_sign;              /* a4-a7: the sign-iteration kernel (all solve_batch calls) */
  double ms_reduce;            /* trace sums */
  double ms_scatter;           /* a8 */
  int64_t solves;              /* nolsm_solve_batch calls */
  int64_t sub_solves;          /* submatrices solved, summed over calls */
  int64_t ns_steps;            /* Newton-Schulz steps, summed over submatrices and calls */
  double flops_paper;          /* 4 n^3 per Newton-Schulz step on the unpadded n (2 n^3 per product) */
  double flops_tensor;         /* tensor-core flops the products need (x3 for split steps), unpadded n */
  double flops_tensor_padded;  /* same on the padded tile shapes the kernel executes */
  double flops_fp64;           /* FP64 flops of the factorisation and solves (a2, a3) */
  int64_t launches;            /* kernels launched for this plan */
  int64_t reruns;              /* submatrices solved again after failing the convergence test under
                                  learned or power-iteration bounds */
  double ms_gather;            /* a1 alone (part of ms_prepare) */
  double ms_factor;            /* a2-a3 factorisation and solve kernels alone (part of ms_prepare) */
  double flops_fp32;           /* FP32 flops of the low-precision paths' factorisation and solves */
  int64_t factor_launches;     /* preparation chunks (one factorisation kernel launch each) */
  double ms_energy_weighted;   /* the centre columns of T_J(W) (nolsm_energy_weighted), kernel alone */
  double ms_prep_tensor;       /* the tensor-core inverse-square-root kernel alone (part of ms_factor) */
  double flops_prep_tensor;    /* its products, 2 n^3 each on the unpadded n (the paper's count) */
  double flops_prep_tensor_issued; /* the same x3 (three-term split products) */
  int64_t ill_conditioned;     /* submatrices of tensor-core solves that were solved on the FP64 path: overlap
                                  too ill-conditioned for the mode, or the low-precision solve failed */
  int64_t ill_conditioned_kept; /* submatrices whose overlap is too ill-conditioned for the mode but larger
                                  than the FP64 path takes (n > 775): solved in the requested mode, whose
                                  accuracy target then does not hold for them */
} nolsm_stats;

nolsm_status nolsm_plan_stats(const nolsm_plan* plan, nolsm_stats* stats);
nolsm_status nolsm_plan_stats_reset(nolsm_plan* plan);

void nolsm_plan_destroy(nolsm_plan* plan);

/* ---------------------------------------------------------------------------------------------
 * a4 bound sources and a10, the learned bound predictor. No counterpart in the paper, which only
 * requires a rescaling before the sign iteration (Sec. "Linear-Scaling Electronic Structure
 * Calculations", after Eq. NS2) and runs a fixed number of steps (Sec. "Efficient Iterative Matrix
 * Function Solvers on GPU Tensor Cores").
 *
 * Bound sources (nolsm_options.bound_source) for the scale alpha_J(mu) = max(hi - mu, mu - lo):
 *   NOLSM_BOUND_GERSHGORIN  the Gershgorin interval of A_J (always safe);
 *   NOLSM_BOUND_POWER       [lo, hi] from 30 steps of two shifted power iterations on A_J (A_J - lo_G I
 *                           and hi_G I - A_J), widened by 5 % of the width, clipped to Gershgorin;
 *   NOLSM_BOUND_MLP         the plan's network (nolsm_plan_set_mlp) predicts (lo, hi, steps / 16) from the
 *                           features below (trained on the power interval, which is already widened); the
 *                           interval, widened by 1 % of its width and clipped to Gershgorin, sets alpha,
 *                           and ceil(1.5 * steps) + 3 caps the submatrix's Newton-Schulz steps.
 * In every source alpha is at least 1/1.7 of the Gershgorin alpha, so every eigenvalue of X_0 lies in
 * [-1.7, 1.7], where the Newton-Schulz map keeps its sign.
 * Every submatrix whose sign iteration fails the convergence test (or turns non-finite) under MLP
 * bounds is solved again with power bounds, and under power bounds again with the Gershgorin interval,
 * within the same nolsm_solve_batch call: no submatrix is accepted unconverged (stats.reruns counts).
 *
 * Features of submatrix J (float32, 7 per submatrix, in this order): n_J / 100, Gershgorin lo and hi
 * of A_J, |N(J)| / 32, mean and standard deviation of diag T_J(H0), mu.
 * Network: h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), y = h2 W3 + b3, width 128, FP32; parameters in
 * one float32 array of nolsm_mlp_param_count() values: W1 [7][128], b1 [128], W2 [128][128], b2 [128],
 * W3 [128][3], b3 [3] (weights [fan_in][fan_out] row-major). Loss 1/(2B) sum (y - t)^2; Adam.
 * --------------------------------------------------------------------------------------------- */
typedef struct nolsm_mlp nolsm_mlp; /* opaque; owns its parameters, Adam state and workspaces */

int32_t nolsm_mlp_param_count(void);

/* Glorot-uniform weights from SplitMix64(seed, parameter index), zero biases, Adam state zero. */
nolsm_status nolsm_mlp_create(uint64_t seed, nolsm_stream_t stream, nolsm_mlp** out);
void nolsm_mlp_destroy(nolsm_mlp* mlp);

/* Parameters to / from host memory (nolsm_mlp_param_count() floats); set also resets the Adam state. */
nolsm_status nolsm_mlp_get_params(const nolsm_mlp* mlp, float* host_params);
nolsm_status nolsm_mlp_set_params(nolsm_mlp* mlp, const float* host_params);

/* y [B][3] = network(x [B][7]); x, y device float32. */
nolsm_status nolsm_mlp_forward(nolsm_mlp* mlp, int32_t B, const float* x, float* y, nolsm_stream_t stream);

/* Gradient of the loss over the batch (x [B][7], targets t [B][3], device) by the backward pass; kept for
 * nolsm_mlp_adam_step and copied to grad_host (nullable, param_count floats); loss (nullable, host). */
nolsm_status nolsm_mlp_gradient(nolsm_mlp* mlp, int32_t B, const float* x, const float* t, nolsm_stream_t stream,
                                float* grad_host, double* loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the last gradient. */
nolsm_status nolsm_mlp_adam_step(nolsm_mlp* mlp, float lr, nolsm_stream_t stream);

/* Minibatch Adam training on N samples (x [N][7], t [N][3], device): epochs passes of ceil(N / batch)
 * steps, sample order (r * 7919 + epoch * 104729) mod N. epoch_loss (host, nullable, [epochs]) receives
 * the mean minibatch loss of each epoch. */
nolsm_status nolsm_mlp_train(nolsm_mlp* mlp, int32_t N, const float* x, const float* t, int32_t epochs,
                             int32_t batch, float lr, nolsm_stream_t stream, double* epoch_loss);

/* The network NOLSM_BOUND_MLP uses in this plan's solves (NULL: none); it must outlive that use. */
nolsm_status nolsm_plan_set_mlp(nolsm_plan* plan, const nolsm_mlp* mlp);

/* Features (device, float32 [n_mol][7]) of the submatrices in the options' range at mu (prepares a1-a3
 * for the range first). Synchronises the stream. */
nolsm_status nolsm_features(nolsm_plan* plan, double mu, const nolsm_options* opts, nolsm_stream_t stream,
                            float* feat);

/* Power-iteration interval (device, float64 [2*n_mol], nullable) of the submatrices in the options' range
 * (prepares a1-a3 first; cached in the plan). Synchronises the stream. */
nolsm_status nolsm_power_bounds(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream, double* lam);

/* Training samples the method produces for the learned predictor, for the options' range at mu:
 * x = features (device float32 [n_mol][7]); t = (power-iteration lo, hi, Newton-Schulz steps / 16 of a
 * solve at mu with power bounds) (device float32 [n_mol][3]). Runs that solve. Synchronises the stream. */
nolsm_status nolsm_training_data(nolsm_plan* plan, double mu, const nolsm_options* opts, nolsm_stream_t stream,
                                 float* x, float* t);

/* Allocation-free sign iteration. No counterpart in the paper.
 *
 * For callers that cannot call cudaMalloc when they need a result: a host application or MD engine
 * that owns all device memory through its own pool (a stray cudaMalloc would bypass its accounting or
 * fail against its reservation), or code with a fixed device-memory budget that must not allocate
 * while it runs. It runs the same tensor-core kernel as nolsm_solve_batch (a4-a7: scale, Newton-Schulz
 * sign iteration with the defect test and refinement, centre columns of D and the partial traces) on
 * inputs the caller already holds, using scratch that lives in a static device array inside the
 * library (about 4.8 MB; every GPU that loads the library keeps it until the process exits).
 *
 * Inputs (device, caller-owned) for submatrix i in [0, count):
 *   sub_n[i] dimension n_i (1..192), nbf[i] number b_i of centre columns,
 *   a_off[i] element offset of A_i in A, c_off[i] element offset of the n_i x b_i arrays,
 *   A    FP32, A_i = T(S)^-1 T(H0) row-major n_i x n_i,
 *   Q    FP64, the centre columns of T(S)^-1 (n_i x b_i row-major),
 *   Sc, Hc FP64, the centre columns of T(S) and T(H0),
 *   lam  FP64 [2*count], an interval [lam[2i], lam[2i+1]] that contains the spectrum of A_i,
 *   mu, opts (precision NOLSM_FP32, NOLSM_BF16X3 or NOLSM_BF16; tolerances, caps; range fields unused).
 * Outputs (device, caller-owned): Dc (n_i x b_i at c_off[i], the centre columns of T(D)), t_S[i], t_H[i],
 *   iters[i], status[i] (per-submatrix nolsm_status).
 * Limits: 1 <= count <= 4096 and every n_i <= 192, else NOLSM_ERR_UNSUPPORTED with a message. To check
 * the dimensions the call copies sub_n to the host and synchronises the stream (work enqueued on it
 * earlier completes first); then it enqueues the solve and returns without waiting: results are ready
 * when the stream reaches that point. Every status[i] is first set to NOLSM_ERR_TIMEOUT on the stream and
 * overwritten by the kernel when it finishes submatrix i, so a submatrix left undone after a device-side
 * wait gave up reads as timed out.
 * The first call on a device looks up the device address of the static array; make that first call
 * before any stream capture. All calls share the one array (the call resets its counters on the stream
 * first), so calls that overlap on the GPU, from different streams or host threads on one device, race:
 * the caller must serialise them. */
nolsm_status nolsm_sign_noalloc(int32_t count, const int32_t* sub_n, const int32_t* nbf, const int64_t* a_off,
                                const int64_t* c_off, const float* A, const double* Q, const double* Sc,
                                const double* Hc, const double* lam, double mu, const nolsm_options* opts,
                                nolsm_stream_t stream, double* Dc, double* t_S, double* t_H, int32_t* iters,
                                int32_t* status);
/* Launch shape of the tensor-core kernel (no counterpart in the paper, which drives library GEMMs). The kernel
 * comes in two shapes: 0 (384 threads, two epilogue groups, output tiles of 128 rows x up to 256 columns) and
 * 1 (512 threads, three epilogue groups, 128 x up to 192, a register split between warpgroups). Each solve
 * (kernel 0: sign iteration) or preparation chunk (kernel 1: inverse square root) splits its submatrices,
 * largest first, into two buckets, n above 192 (bucket 1) and the rest (bucket 0), and launches them once
 * together when both take the same shape, else once each. The first time a process
 * meets a (kernel, precision, bucket), both shapes run on that bucket's largest submatrices (32 per slot
 * of every SM), timed with CUDA events on the caller's stream, and the faster is kept for the life of the
 * process; the timed runs' results are computed again by the bucket's launch. Setting the environment
 * variable NOLSM_TC_SHAPE to "0" or "1" fixes the shape instead (read at every call); E4M3 and the reruns of
 * failed submatrices always take shape 0. Returns the shape chosen so far for (kernel, precision, bucket), or
 * -1 when none has been measured yet. Host only; thread-safe. */
int32_t nolsm_tc_shape(int32_t kernel, int32_t precision, int32_t bucket);

const char* nolsm_status_str(nolsm_status s);
const char* nolsm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NOLSM_H */
