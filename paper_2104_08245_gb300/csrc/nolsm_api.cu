// C ABI entry points (include/nolsm.h): argument checks, plan lifecycle, dispatch by precision, the
// host side of the mu bisection, and error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "nolsm_internal.cuh"
#include "bounds.cuh"
#include "prep.cuh"
#include "tc_path.cuh"

namespace nolsm {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// Workspaces come from the device's default stream-ordered memory pool, which keeps freed memory
// (release threshold raised once per device) so that a plan built per geometry reuses the previous
// plan's pages instead of mapping new ones. Allocation and release are made complete before they
// return, like cudaMalloc and cudaFree, so buffers may be used on any stream.
static void pool_keep_freed_memory() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done[dev] = true;
}

nolsm_status dev_alloc(nolsm_plan* plan, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  pool_keep_freed_memory();
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, 0);
  if (e == cudaErrorMemoryAllocation) {   // give the pool's kept pages back to the device and retry once
    cudaGetLastError();
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      cudaDeviceSynchronize();
      cudaMemPoolTrimTo(pool, 0);
    }
    e = cudaMallocAsync(&p, bytes, 0);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? NOLSM_ERR_OOM : NOLSM_ERR_CUDA;
  }
  b.p = p;
  b.bytes = bytes;
  plan->bytes += (int64_t)bytes;
  return NOLSM_OK;
}

void dev_free(nolsm_plan* plan, DevBuf& b) {
  if (b.p) {
    cudaDeviceSynchronize();   // no work still using the buffer, whatever stream it runs on
    cudaFreeAsync(b.p, 0);
    cudaStreamSynchronize(0);
    plan->bytes -= (int64_t)b.bytes;
  }
  b.p = nullptr;
  b.bytes = 0;
}

void mark(nolsm_plan* plan, int i, cudaStream_t st) {
  if (plan->ev_ok) cudaEventRecord(plan->ev[i], st);
}

void pmark(nolsm_plan* plan, cudaStream_t st) {
  if (!plan->ev_ok) return;
  if (plan->pev_used == plan->pev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    plan->pev.push_back(e);
  }
  cudaEventRecord(plan->pev[plan->pev_used++], st);
}

void tmark(nolsm_plan* plan, cudaStream_t st) {
  if (!plan->ev_ok) return;
  if (plan->tev_used == plan->tev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    plan->tev.push_back(e);
  }
  cudaEventRecord(plan->tev[plan->tev_used++], st);
}

void prep_times(nolsm_plan* plan) {
  for (size_t k = 0; k + 1 < plan->tev_used; k += 2) {
    float a = 0.0f;
    if (cudaEventElapsedTime(&a, plan->tev[k], plan->tev[k + 1]) == cudaSuccess) plan->stats.ms_prep_tensor += a;
    else cudaGetLastError();
  }
  plan->tev_used = 0;
  for (size_t k = 0; k + 2 < plan->pev_used; k += 3) {
    float a = 0.0f, b = 0.0f;
    if (cudaEventElapsedTime(&a, plan->pev[k], plan->pev[k + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&b, plan->pev[k + 1], plan->pev[k + 2]) == cudaSuccess) {
      plan->stats.ms_gather += a;
      plan->stats.ms_factor += b;
    } else {
      cudaGetLastError();
    }
  }
  plan->pev_used = 0;
}

double elapsed(nolsm_plan* plan, int i, int j) {
  if (!plan->ev_ok) return 0.0;
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, plan->ev[i], plan->ev[j]) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return (double)ms;
}

}  // namespace nolsm

using namespace nolsm;

nolsm_plan::~nolsm_plan() {
  DevBuf* all[] = {&s_blk_off, &h_blk_off, &nb_ptr, &nb_idx, &nb_off, &sub_n, &sub_c0, &d_blk_off, &d_slot,
                   &a_off, &c_off, &flag, &Q, &Sc, &Hc, &lam, &prep_status, &prep64.A, &prep32.A, &prep_sym.A, &prep_ns.A, &Lsym, &Wc, &Dc,
                   &t_S, &t_H, &iters, &status, &rsteps, &nbelow, &nb_lo, &nb_hi, &active, &sums, &counter, &ws_dense, &ws_l32, &ws_refine, &prep_order, &ws_ns,
                   &lam_p, &onsite, &feat, &mlp_y, &lam_m, &budget, &rerun, &ws_ysym, &Wd, &tW,
                   &prep32.cond, &prep_ns.cond, &ill_list, &onsite_off,
                   &sub_b, &m_nb_ptr, &m_nb_idx, &g_of, &g_col, &g_row};
  for (DevBuf* b : all) dev_free(this, *b);
  tc_release(this);
  if (ev_ok)
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  for (cudaEvent_t e : pev) cudaEventDestroy(e);
  for (cudaEvent_t e : tev) cudaEventDestroy(e);
}

extern "C" {

void nolsm_options_default(nolsm_options* o, int32_t precision) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = precision;
  const bool fp64 = precision == NOLSM_FP64;
  o->refine_steps = fp64 ? 0 : (precision == NOLSM_FP8E4M3 ? 3 : 2);
  o->max_iter = 100;
  o->tol_ns = fp64 ? 1e-9 : 1e-2;
  o->tol_accept = fp64 ? 1e-7 : 1e-4;
  o->tol_n = 1e-5;
  o->tol_mu = 1e-10;
  o->max_bisect = 100;
  o->bound_source = NOLSM_BOUND_GERSHGORIN;
  o->sub_begin = 0;
  o->sub_end = 0;
}

int32_t nolsm_tc_shape(int32_t kernel, int32_t precision, int32_t bucket) {
  return tc_shape_choice(kernel, precision, bucket);
}

const char* nolsm_status_str(nolsm_status s) {
  switch (s) {
    case NOLSM_OK: return "ok";
    case NOLSM_ERR_ARG: return "invalid argument";
    case NOLSM_ERR_CUDA: return "CUDA error";
    case NOLSM_ERR_OOM: return "out of device memory";
    case NOLSM_ERR_NOT_SPD: return "overlap submatrix not positive definite";
    case NOLSM_ERR_NOT_CONVERGED: return "sign iteration did not converge";
    case NOLSM_ERR_NONFINITE: return "non-finite value";
    case NOLSM_ERR_NO_PLATEAU: return "bisection found no mu with the requested electron count";
    case NOLSM_ERR_UNSUPPORTED: return "unsupported option or size";
    case NOLSM_ERR_NO_SOLUTION: return "no solution to write back";
    case NOLSM_ERR_TIMEOUT: return "device-side wait timed out";
  }
  return "unknown status";
}

const char* nolsm_last_error(void) { return g_err; }

nolsm_status nolsm_build_submatrices(const nolsm_system* sys, nolsm_stream_t stream, nolsm_plan** out) {
  if (!out) { set_error("nolsm_build_submatrices: out is NULL"); return NOLSM_ERR_ARG; }
  *out = nullptr;
  if (!sys || sys->n_mol <= 0 || !sys->nbf || !sys->s_row_ptr || !sys->h_row_ptr ||
      sys->s_nnzb <= 0 || sys->h_nnzb <= 0 || !sys->s_col_idx || !sys->h_col_idx ||
      sys->s_nnzb > INT32_MAX || sys->h_nnzb > INT32_MAX) {
    set_error("nolsm_build_submatrices: missing or inconsistent system arrays");
    return NOLSM_ERR_ARG;
  }
  nolsm_plan* plan = new (std::nothrow) nolsm_plan();
  if (!plan) { set_error("host allocation failed"); return NOLSM_ERR_OOM; }
  plan->sys = *sys;
  plan->n_mol = sys->n_mol;
  plan->ev_ok = true;
  for (cudaEvent_t& e : plan->ev)
    if (cudaEventCreate(&e) != cudaSuccess) plan->ev_ok = false;
  if (!plan->ev_ok) cudaGetLastError();
  mark(plan, 0, (cudaStream_t)stream);
  nolsm_status s = build_plan_device(plan, (cudaStream_t)stream);
  if (s != NOLSM_OK) {
    delete plan;
    return s;
  }
  mark(plan, 1, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  plan->stats.ms_plan += elapsed(plan, 0, 1);
  *out = plan;
  return NOLSM_OK;
}

nolsm_status nolsm_plan_query(const nolsm_plan* plan, nolsm_plan_info* info) {
  if (!plan || !info) { set_error("nolsm_plan_query: NULL argument"); return NOLSM_ERR_ARG; }
  info->n_mol = plan->n_mol;
  info->d_nnzb = plan->d_nnzb;
  info->d_nvals = plan->d_nvals;
  info->max_n = plan->max_n;
  info->min_n = plan->min_n;
  info->sum_n3 = plan->sum_n3;
  info->device_bytes = plan->bytes;
  info->nb_entries = plan->h_nb_ptr.empty() ? 0 : plan->h_nb_ptr.back();
  info->grouped = plan->grouped ? 1 : 0;
  return NOLSM_OK;
}

nolsm_status nolsm_plan_set_elements(nolsm_plan* plan, const nolsm_element_model* m) {
  if (!plan || !m || !m->pos || !m->onsite || (m->aniso != 0.0 && !m->dirs) ||
      !(m->cell[0] > 0.0 && m->cell[1] > 0.0 && m->cell[2] > 0.0) || !std::isfinite(m->s_exp) ||
      !std::isfinite(m->hop) || !(m->hop_len > 0.0) || !std::isfinite(m->aniso)) {
    set_error("nolsm_plan_set_elements: NULL array or invalid model parameter");
    return NOLSM_ERR_ARG;
  }
  const int32_t n = plan->sys.n_mol;   // molecules of the input system
  std::vector<int64_t> off((size_t)n + 1, 0);
  for (int32_t I = 0; I < n; ++I) off[(size_t)I + 1] = off[(size_t)I] + plan->h_nbf[(size_t)I];
  if (!plan->onsite_off.p) NOLSM_TRY(dev_alloc(plan, plan->onsite_off, sizeof(int64_t) * off.size()));
  NOLSM_CUDA_TRY(cudaMemcpy(plan->onsite_off.p, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice));
  plan->model = *m;
  plan->gen = true;
  // the geometry caches were prepared from other elements (or none): prepare again
  for (Prepared* P : {&plan->prep64, &plan->prep32, &plan->prep_sym, &plan->prep_ns}) P->done.assign(P->done.size(), 0);
  plan->pow_done.assign(plan->pow_done.size(), 0);
  plan->onsite_done = false;
  plan->have_solution = false;
  return NOLSM_OK;
}

nolsm_status nolsm_plan_get_maps(const nolsm_plan* plan, int32_t* nb_ptr, int32_t* nb_idx, int32_t* nb_off,
                                 int32_t* sub_n, int32_t* sub_c0, int64_t* d_blk_off, nolsm_stream_t stream) {
  if (!plan) { set_error("nolsm_plan_get_maps: NULL plan"); return NOLSM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)plan->n_mol, m = (size_t)plan->d_nnzb, q = (size_t)plan->h_nb_ptr[n];
  if (nb_ptr) NOLSM_CUDA_TRY(cudaMemcpyAsync(nb_ptr, plan->nb_ptr.p, 4 * (n + 1), cudaMemcpyDeviceToDevice, st));
  if (nb_idx) NOLSM_CUDA_TRY(cudaMemcpyAsync(nb_idx, plan->nb_idx.p, 4 * q, cudaMemcpyDeviceToDevice, st));
  if (nb_off) NOLSM_CUDA_TRY(cudaMemcpyAsync(nb_off, plan->nb_off.p, 4 * q, cudaMemcpyDeviceToDevice, st));
  if (sub_n) NOLSM_CUDA_TRY(cudaMemcpyAsync(sub_n, plan->sub_n.p, 4 * n, cudaMemcpyDeviceToDevice, st));
  if (sub_c0) NOLSM_CUDA_TRY(cudaMemcpyAsync(sub_c0, plan->sub_c0.p, 4 * n, cudaMemcpyDeviceToDevice, st));
  if (d_blk_off) NOLSM_CUDA_TRY(cudaMemcpyAsync(d_blk_off, plan->d_blk_off.p, 8 * (m + 1), cudaMemcpyDeviceToDevice, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  return NOLSM_OK;
}

static nolsm_status check_options(const nolsm_plan* plan, const nolsm_options* o, int64_t* j0, int64_t* j1) {
  if (!o) { set_error("options are NULL"); return NOLSM_ERR_ARG; }
  if (o->precision < NOLSM_FP64 || o->precision > NOLSM_FP16 || o->max_iter < 1 || o->max_iter > 10000 ||
      o->refine_steps < 0 || o->refine_steps > 100 || !(o->tol_ns > 0) || !(o->tol_accept > 0) ||
      o->bound_source < 0 || o->bound_source > NOLSM_BOUND_MLP || o->inverse < NOLSM_INVERSE_CHOLESKY ||
      o->inverse > NOLSM_INVERSE_NEWTON_SCHULZ) {
    set_error("invalid options (precision %d, max_iter %d, refine %d, tol_ns %g, tol_accept %g, bound %d)",
              o->precision, o->max_iter, o->refine_steps, o->tol_ns, o->tol_accept, o->bound_source);
    return NOLSM_ERR_ARG;
  }
  *j0 = o->sub_begin;
  *j1 = o->sub_end <= 0 ? plan->n_mol : o->sub_end;
  if (*j0 < 0 || *j0 >= *j1 || *j1 > plan->n_mol) {
    set_error("invalid submatrix range [%lld, %lld) of %d", (long long)*j0, (long long)*j1, plan->n_mol);
    return NOLSM_ERR_ARG;
  }
  return NOLSM_OK;
}

// Scale source of one solve: the Gershgorin interval, the power-iteration interval (cached per plan) or
// the learned interval and step budget (features at mu, then the plan's network).
static nolsm_status bound_spec(nolsm_plan* plan, int source, double mu, const nolsm_options& o, int cls, int64_t j0,
                               int64_t j1, cudaStream_t st, SolveSpec* spec) {
  *spec = SolveSpec{};
  spec->lam = plan->lam.as<double>();
  if (source == NOLSM_BOUND_POWER) {
    NOLSM_TRY(power_bounds(plan, cls, j0, j1, nullptr, 0, st));
    spec->lam = plan->lam_p.as<double>();
  } else if (source == NOLSM_BOUND_MLP) {
    NOLSM_TRY(features(plan, mu, j0, j1, st));
    NOLSM_TRY(mlp_bounds(plan, j0, j1, o.max_iter, st));
    spec->lam = plan->lam_m.as<double>();
    spec->budget = plan->budget.as<int32_t>();
  }
  return NOLSM_OK;
}

// Submatrices of a tensor-core solve that go to the FP64 path instead (host list): FP64 preparation of them
// (in runs of consecutive indices; cached like any preparation), then the FP64 sign iteration on their list.
static nolsm_status solve_on_fp64(nolsm_plan* plan, double mu, const nolsm_options& o, int64_t j0, int64_t j1,
                                  std::vector<int32_t>& subs, cudaStream_t st) {
  if (subs.empty()) return NOLSM_OK;
  std::sort(subs.begin(), subs.end());
  for (size_t a = 0; a < subs.size();) {
    size_t b = a + 1;
    while (b < subs.size() && subs[b] == subs[b - 1] + 1) ++b;
    NOLSM_TRY(prepare(plan, subs[a], (int64_t)subs[b - 1] + 1, kPrepFP64, st));
    a = b;
  }
  if (!plan->ill_list.p) NOLSM_TRY(dev_alloc(plan, plan->ill_list, sizeof(int32_t) * (size_t)plan->n_mol));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->ill_list.p, subs.data(), sizeof(int32_t) * subs.size(), cudaMemcpyHostToDevice, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));   // subs is a host vector
  nolsm_options o64;
  nolsm_options_default(&o64, NOLSM_FP64);
  o64.max_iter = std::max(o.max_iter, o64.max_iter);
  SolveSpec fs;
  fs.list = plan->ill_list.as<int32_t>();
  fs.count = (int32_t)subs.size();
  NOLSM_TRY(solve_fp64(plan, mu, o64, j0, j1, fs, st));
  plan->stats.ill_conditioned += (int64_t)subs.size();
  return NOLSM_OK;
}

// Before a tensor-core solve's own kernel: the submatrices of the work (the list, else the range) whose
// overlap is too ill-conditioned for the mode (cond estimate above cond_max; the sign kernel skips them).
static nolsm_status ill_conditioned_list(nolsm_plan* plan, const nolsm_options& o, int cls, int64_t j0, int64_t j1,
                                         const int32_t* list, int32_t count, cudaStream_t st, std::vector<int32_t>* out) {
  out->clear();
  const Prepared& P = prepared(plan, cls);
  if (!P.cond.p || P.h_cond.empty()) return NOLSM_OK;
  const float lim = cond_max(o.precision);
  const int max_n = prepare_fp64_max_n();   // larger submatrices stay on the tensor path
  auto take = [&](int32_t J) {
    if (P.h_cond[(size_t)J] <= lim) return;
    if (plan->h_sub_n[(size_t)J] <= max_n)
      out->push_back(J);
    else
      plan->stats.ill_conditioned_kept += 1;
  };
  if (list) {
    std::vector<int32_t> cand((size_t)count);
    NOLSM_CUDA_TRY(cudaMemcpyAsync(cand.data(), list, sizeof(int32_t) * (size_t)count, cudaMemcpyDeviceToHost, st));
    NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int32_t J : cand) take(J);
  } else {
    for (int64_t J = j0; J < j1; ++J) take((int32_t)J);
  }
  return NOLSM_OK;
}

// After a tensor-core solve (and its bound-source reruns): the submatrices of the range that failed the accept
// test or turned non-finite and that the FP64 path can take (a wait that gave up stays reported as such).
static nolsm_status failed_fp64_list(nolsm_plan* plan, int64_t j0, int64_t j1, cudaStream_t st, std::vector<int32_t>* out) {
  out->clear();
  std::vector<int32_t> stv((size_t)(j1 - j0)), ps((size_t)(j1 - j0));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(stv.data(), plan->status.as<int32_t>() + j0, sizeof(int32_t) * stv.size(),
                                 cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(ps.data(), plan->prep_status.as<int32_t>() + j0, sizeof(int32_t) * ps.size(),
                                 cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  const int max_n = prepare_fp64_max_n();
  for (int64_t J = j0; J < j1; ++J) {
    const int32_t s = stv[(size_t)(J - j0)];
    if (s != kSubNotConv && s != kSubNonFinite) continue;
    if (ps[(size_t)(J - j0)] == kSubNotSpd) continue;   // an indefinite overlap stays reported
    if (plan->h_sub_n[(size_t)J] <= max_n) out->push_back((int32_t)J);
  }
  return NOLSM_OK;
}

// The solve of nolsm_solve_batch, restricted to the device list[0, count) of submatrices of the range
// when `list` is set (the others keep their previous results; the trace sums cover the whole range).
static nolsm_status solve_impl(nolsm_plan* plan, double mu, const nolsm_options* opts, cudaStream_t st,
                               const int32_t* list, int32_t count, double* trace_DS, double* trace_DH,
                               double* sub_t_S, double* sub_t_H, int32_t* iters, int32_t* status) {
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  NOLSM_TRY(ensure_results(plan));
  const bool fp64 = opts->precision == NOLSM_FP64;
  const int cls = prep_class(*opts);
  mark(plan, 0, st);
  NOLSM_TRY(prepare(plan, j0, j1, cls, st));
  int level = opts->bound_source;
  SolveSpec spec;
  NOLSM_TRY(bound_spec(plan, level, mu, *opts, cls, j0, j1, st, &spec));
  if (list) {
    spec.list = list;
    spec.count = count;
  }
  mark(plan, 1, st);
  std::vector<int32_t> handed;
  if (!fp64 && cls != kPrepSym) NOLSM_TRY(ill_conditioned_list(plan, *opts, cls, j0, j1, list, count, st, &handed));
  NOLSM_TRY(fp64 ? solve_fp64(plan, mu, *opts, j0, j1, spec, st) : solve_tc(plan, mu, *opts, j0, j1, spec, st));
  NOLSM_TRY(solve_on_fp64(plan, mu, *opts, j0, j1, handed, st));
  // submatrices that failed the convergence test under learned bounds are solved again with power
  // bounds, under power bounds with the Gershgorin interval
  while (level > NOLSM_BOUND_GERSHGORIN) {
    int32_t count = 0;
    NOLSM_TRY(failed_list(plan, j0, j1, st, &count));
    if (count == 0) break;
    level -= 1;
    SolveSpec rs;
    rs.list = plan->rerun.as<int32_t>();
    rs.count = count;
    if (level == NOLSM_BOUND_POWER) {
      NOLSM_TRY(power_bounds(plan, cls, 0, 0, rs.list, count, st));
      rs.lam = plan->lam_p.as<double>();
    } else {
      rs.lam = plan->lam.as<double>();
    }
    NOLSM_TRY(fp64 ? solve_fp64(plan, mu, *opts, j0, j1, rs, st) : solve_tc(plan, mu, *opts, j0, j1, rs, st));
    plan->stats.reruns += count;
  }
  // no submatrix is accepted unconverged: what the low-precision solve left failed goes to the FP64 path
  if (!fp64 && cls != kPrepSym) {
    NOLSM_TRY(failed_fp64_list(plan, j0, j1, st, &handed));
    NOLSM_TRY(solve_on_fp64(plan, mu, *opts, j0, j1, handed, st));
  }
  mark(plan, 2, st);
  double tS = 0, tH = 0;
  int32_t bad = 0;
  NOLSM_TRY(reduce_traces(plan, j0, j1, fp64 ? 1 : main_terms(opts->precision), st, &tS, &tH, &bad, list, count));
  mark(plan, 3, st);
  const size_t cnt = (size_t)(j1 - j0);
  if (sub_t_S) NOLSM_CUDA_TRY(cudaMemcpyAsync(sub_t_S + j0, plan->t_S.as<double>() + j0, 8 * cnt, cudaMemcpyDeviceToDevice, st));
  if (sub_t_H) NOLSM_CUDA_TRY(cudaMemcpyAsync(sub_t_H + j0, plan->t_H.as<double>() + j0, 8 * cnt, cudaMemcpyDeviceToDevice, st));
  if (iters) NOLSM_CUDA_TRY(cudaMemcpyAsync(iters + j0, plan->iters.as<int32_t>() + j0, 4 * cnt, cudaMemcpyDeviceToDevice, st));
  if (status) NOLSM_CUDA_TRY(cudaMemcpyAsync(status + j0, plan->status.as<int32_t>() + j0, 4 * cnt, cudaMemcpyDeviceToDevice, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  plan->stats.ms_prepare += elapsed(plan, 0, 1);
  prep_times(plan);
  plan->stats.ms_sign += elapsed(plan, 1, 2);
  plan->stats.ms_reduce += elapsed(plan, 2, 3);
  plan->stats.solves += 1;
  plan->stats.sub_solves += list ? count : j1 - j0;
  if (trace_DS) *trace_DS = tS;
  if (trace_DH) *trace_DH = tH;
  plan->solved_begin = j0;
  plan->solved_end = j1;
  plan->solved_cls = cls;
  plan->have_solution = true;
  if (bad != 0) {
    set_error("nolsm_solve_batch: a submatrix reported '%s'", nolsm_status_str((nolsm_status)bad));
    return (nolsm_status)bad;
  }
  return NOLSM_OK;
}

nolsm_status nolsm_solve_batch(nolsm_plan* plan, double mu, const nolsm_options* opts, nolsm_stream_t stream,
                               double* trace_DS, double* trace_DH, double* sub_t_S, double* sub_t_H,
                               int32_t* iters, int32_t* status) {
  if (!plan) { set_error("nolsm_solve_batch: NULL plan"); return NOLSM_ERR_ARG; }
  if (!std::isfinite(mu)) { set_error("nolsm_solve_batch: mu is not finite"); return NOLSM_ERR_ARG; }
  return solve_impl(plan, mu, opts, (cudaStream_t)stream, nullptr, 0, trace_DS, trace_DH, sub_t_S, sub_t_H, iters,
                    status);
}

static nolsm_status ensure_dev(nolsm_plan* plan, DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return NOLSM_OK;
  dev_free(plan, b);
  return dev_alloc(plan, b, bytes);
}

// a9 support. n_below(J, mu) = (n - Tr sign(A_J - mu I)) / 2 counts the eigenvalues of submatrix J below mu;
// where it is equal at both ends of the bracket, no eigenvalue of J lies inside, T_J(D) is the same for
// every mu in the bracket, and J needs no further solve: its centre columns and traces stay valid.
__global__ void k_bracket_init(int32_t j0, int32_t j1, const int32_t* __restrict__ sub_n, int known,
                               int32_t* __restrict__ nb_lo, int32_t* __restrict__ nb_hi) {
  for (int32_t J = j0 + blockIdx.x * blockDim.x + threadIdx.x; J < j1; J += gridDim.x * blockDim.x) {
    nb_lo[J] = known ? 0 : -1;            // the default bracket contains every submatrix's spectrum
    nb_hi[J] = known ? sub_n[J] : -1;
  }
}

__global__ void k_active_list(int32_t j0, int32_t j1, const int32_t* __restrict__ nb_lo,
                              const int32_t* __restrict__ nb_hi, int32_t* __restrict__ list, int32_t* __restrict__ count) {
  for (int32_t J = j0 + blockIdx.x * blockDim.x + threadIdx.x; J < j1; J += gridDim.x * blockDim.x)
    if (nb_lo[J] < 0 || nb_hi[J] < 0 || nb_lo[J] != nb_hi[J]) list[atomicAdd(count, 1)] = J;
}

__global__ void k_bracket_update(int32_t j0, int32_t j1, const int32_t* __restrict__ list, int32_t count,
                                 const int32_t* __restrict__ nbelow, int32_t* __restrict__ nb_side) {
  const int32_t m = list ? count : j1 - j0;
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    const int32_t J = list ? list[e] : j0 + e;
    nb_side[J] = nbelow[J];
  }
}

nolsm_status nolsm_scatter_density(nolsm_plan* plan, double* D_vals, nolsm_stream_t stream) {
  if (!plan || !D_vals) { set_error("nolsm_scatter_density: NULL argument"); return NOLSM_ERR_ARG; }
  if (!plan->have_solution) { set_error("nolsm_scatter_density: no solve yet"); return NOLSM_ERR_NO_SOLUTION; }
  mark(plan, 4, (cudaStream_t)stream);
  NOLSM_TRY(scatter(plan, D_vals, plan->solved_begin, plan->solved_end, (cudaStream_t)stream));
  mark(plan, 5, (cudaStream_t)stream);
  NOLSM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  plan->stats.ms_scatter += elapsed(plan, 4, 5);
  return NOLSM_OK;
}

nolsm_status nolsm_plan_get_prepared(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream, void* A,
                                     double* Q, int32_t* prep_status, float* cond_est) {
  if (!plan) { set_error("nolsm_plan_get_prepared: NULL plan"); return NOLSM_ERR_ARG; }
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  cudaStream_t st = (cudaStream_t)stream;
  NOLSM_TRY(ensure_results(plan));
  const int cls = prep_class(*opts);
  NOLSM_TRY(prepare(plan, j0, j1, cls, st));
  prep_times(plan);
  const Prepared& P = prepared(plan, cls);
  const size_t esz = P.fp64 ? sizeof(double) : sizeof(float);
  const int64_t a0 = plan->h_a_off[j0], a1 = plan->h_a_off[j1], c0 = plan->h_c_off[j0], c1 = plan->h_c_off[j1];
  if (A)
    NOLSM_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(A) + esz * a0, static_cast<const char*>(P.A.p) + esz * a0,
                                   esz * (size_t)(a1 - a0), cudaMemcpyDeviceToDevice, st));
  if (Q)
    NOLSM_CUDA_TRY(cudaMemcpyAsync(Q + c0, plan->Q.as<double>() + c0, sizeof(double) * (size_t)(c1 - c0),
                                   cudaMemcpyDeviceToDevice, st));
  if (prep_status)
    NOLSM_CUDA_TRY(cudaMemcpyAsync(prep_status + j0, plan->prep_status.as<int32_t>() + j0,
                                   sizeof(int32_t) * (size_t)(j1 - j0), cudaMemcpyDeviceToDevice, st));
  if (cond_est && P.cond.p)
    NOLSM_CUDA_TRY(cudaMemcpyAsync(cond_est + j0, P.cond.as<float>() + j0, sizeof(float) * (size_t)(j1 - j0),
                                   cudaMemcpyDeviceToDevice, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  return NOLSM_OK;
}

nolsm_status nolsm_spectral_bracket(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream, double* lo,
                                    double* hi) {
  if (!plan || !lo || !hi) { set_error("nolsm_spectral_bracket: NULL argument"); return NOLSM_ERR_ARG; }
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  cudaStream_t st = (cudaStream_t)stream;
  NOLSM_TRY(ensure_results(plan));
  mark(plan, 0, st);
  NOLSM_TRY(prepare(plan, j0, j1, prep_class(*opts), st));
  mark(plan, 1, st);
  std::vector<double> lam((size_t)(2 * (j1 - j0)));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(lam.data(), plan->lam.as<double>() + 2 * j0, sizeof(double) * lam.size(),
                                 cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  plan->stats.ms_prepare += elapsed(plan, 0, 1);
  prep_times(plan);
  std::vector<int32_t> pst((size_t)(j1 - j0));
  NOLSM_CUDA_TRY(cudaMemcpy(pst.data(), plan->prep_status.as<int32_t>() + j0, sizeof(int32_t) * pst.size(),
                            cudaMemcpyDeviceToHost));
  double a = INFINITY, b = -INFINITY;
  for (size_t k = 0; k < pst.size(); ++k) {
    if (pst[k] != kSubOk) continue;
    a = std::min(a, lam[2 * k]);
    b = std::max(b, lam[2 * k + 1]);
  }
  if (!(a < b) || !std::isfinite(a) || !std::isfinite(b)) {
    set_error("nolsm_spectral_bracket: no submatrix with a usable spectrum in the range");
    return NOLSM_ERR_NOT_SPD;
  }
  *lo = a;
  *hi = b;
  return NOLSM_OK;
}

// The bisection's per-point state lives in the plan: counts of eigenvalues below mu at the bracket's
// ends (nb_lo, nb_hi; -1 unknown), the count of the last point (nbelow) and its work list.
nolsm_status nolsm_bisect_begin(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream,
                                int32_t bracket_contains_spectrum) {
  if (!plan || !opts) { set_error("nolsm_bisect_begin: NULL argument"); return NOLSM_ERR_ARG; }
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  cudaStream_t st = (cudaStream_t)stream;
  NOLSM_TRY(ensure_results(plan));
  const size_t nm = (size_t)plan->n_mol;
  NOLSM_TRY(ensure_dev(plan, plan->nb_lo, sizeof(int32_t) * nm));
  NOLSM_TRY(ensure_dev(plan, plan->nb_hi, sizeof(int32_t) * nm));
  NOLSM_TRY(ensure_dev(plan, plan->active, sizeof(int32_t) * (nm + 1)));
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (j1 - j0 + 255) / 256));
  k_bracket_init<<<blocks, 256, 0, st>>>((int32_t)j0, (int32_t)j1, plan->sub_n.as<int32_t>(),
                                         bracket_contains_spectrum ? 1 : 0, plan->nb_lo.as<int32_t>(),
                                         plan->nb_hi.as<int32_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  plan->bisect_first = true;
  plan->bisect_count = -1;
  return NOLSM_OK;
}

nolsm_status nolsm_bisect_point(nolsm_plan* plan, double mu, const nolsm_options* opts, nolsm_stream_t stream,
                                double* trace_DS, int32_t* solved) {
  if (!plan || !opts || !std::isfinite(mu)) { set_error("nolsm_bisect_point: invalid argument"); return NOLSM_ERR_ARG; }
  if (!plan->nb_lo.p) { set_error("nolsm_bisect_point: no nolsm_bisect_begin"); return NOLSM_ERR_ARG; }
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nm = (size_t)plan->n_mol;
  int32_t* act = plan->active.as<int32_t>();
  const int32_t* list = nullptr;
  int32_t count = (int32_t)(j1 - j0);
  if (!plan->bisect_first) {   // the submatrices with an eigenvalue in the bracket (all at the first point)
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (j1 - j0 + 255) / 256));
    NOLSM_CUDA_TRY(cudaMemsetAsync(act + nm, 0, sizeof(int32_t), st));
    k_active_list<<<blocks, 256, 0, st>>>((int32_t)j0, (int32_t)j1, plan->nb_lo.as<int32_t>(), plan->nb_hi.as<int32_t>(),
                                          act, act + nm);
    NOLSM_LAUNCH_CHECK();
    NOLSM_CUDA_TRY(cudaMemcpyAsync(&count, act + nm, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
    list = act;
  }
  plan->bisect_first = false;
  plan->bisect_count = count;
  plan->bisect_listed = list != nullptr;
  if (solved) *solved = count;
  if (count == 0) {   // no submatrix changes inside the bracket: Tr(DS) is the last point's
    if (trace_DS) *trace_DS = plan->bisect_trace;
    return NOLSM_OK;
  }
  double t = 0.0;
  nolsm_status s = solve_impl(plan, mu, opts, st, list, count, &t, nullptr, nullptr, nullptr, nullptr, nullptr);
  plan->bisect_trace = t;
  if (trace_DS) *trace_DS = t;
  return s;
}

nolsm_status nolsm_bisect_side(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream, int32_t raises_lo) {
  if (!plan || !opts) { set_error("nolsm_bisect_side: NULL argument"); return NOLSM_ERR_ARG; }
  if (plan->bisect_count < 0) { set_error("nolsm_bisect_side: no nolsm_bisect_point"); return NOLSM_ERR_ARG; }
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->bisect_count > 0) {
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (j1 - j0 + 255) / 256));
    k_bracket_update<<<blocks, 256, 0, st>>>((int32_t)j0, (int32_t)j1,
                                             plan->bisect_listed ? plan->active.as<int32_t>() : nullptr,
                                             plan->bisect_count, plan->nbelow.as<int32_t>(),
                                             raises_lo ? plan->nb_lo.as<int32_t>() : plan->nb_hi.as<int32_t>());
    NOLSM_LAUNCH_CHECK();
    NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  plan->bisect_count = -1;
  return NOLSM_OK;
}

nolsm_status nolsm_bisection_start(nolsm_bisection* b, double n_occ, double lo, double hi) {
  if (!b || !std::isfinite(n_occ) || !std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi)) {
    set_error("nolsm_bisection_start: invalid bracket [%g, %g] or n_occ %g", lo, hi, n_occ);
    return NOLSM_ERR_ARG;
  }
  b->lo = lo;
  b->hi = hi;
  b->mu = 0.5 * (lo + hi);
  b->n_occ = n_occ;
  b->trace_DS = 0.0;
  b->steps = 0;
  b->state = NOLSM_BISECT_EVALUATE;
  return NOLSM_OK;
}

nolsm_status nolsm_bisection_update(nolsm_bisection* b, double trace_DS, const nolsm_options* opts,
                                    int32_t* raises_lo) {
  if (!b || !opts || b->state != NOLSM_BISECT_EVALUATE || !std::isfinite(trace_DS)) {
    set_error("nolsm_bisection_update: no point to decide on, or a non-finite Tr(DS)");
    return NOLSM_ERR_ARG;
  }
  b->steps += 1;
  b->trace_DS = trace_DS;
  const double f = trace_DS - b->n_occ;
  if (std::fabs(f) <= opts->tol_n * std::fabs(b->n_occ)) {
    b->state = NOLSM_BISECT_ACCEPTED;
    return NOLSM_OK;
  }
  const int below = f < 0.0 ? 1 : 0;
  if (raises_lo) *raises_lo = below;
  if (below) b->lo = b->mu; else b->hi = b->mu;
  const int cap = opts->max_bisect > 0 ? opts->max_bisect : 100;
  if (b->hi - b->lo <= opts->tol_mu || b->steps >= cap) {
    b->state = NOLSM_BISECT_NO_PLATEAU;
    return NOLSM_OK;
  }
  b->mu = 0.5 * (b->lo + b->hi);
  return NOLSM_OK;
}

nolsm_status nolsm_find_mu(nolsm_plan* plan, double n_occ, double lo, double hi, const nolsm_options* opts,
                           nolsm_stream_t stream, double* mu_out, double* trace_DS_out, int32_t* steps_out,
                           double* mu_history) {
  if (!plan || !opts || !std::isfinite(lo) || !std::isfinite(hi) || !std::isfinite(n_occ)) {
    set_error("nolsm_find_mu: invalid arguments");
    return NOLSM_ERR_ARG;
  }
  const bool default_bracket = !(lo < hi);
  if (default_bracket) {
    NOLSM_TRY(nolsm_spectral_bracket(plan, opts, stream, &lo, &hi));
  }
  NOLSM_TRY(nolsm_bisect_begin(plan, opts, stream, default_bracket ? 1 : 0));
  nolsm_bisection b;
  NOLSM_TRY(nolsm_bisection_start(&b, n_occ, lo, hi));
  nolsm_status result = NOLSM_OK;
  double mu = b.mu;
  while (b.state == NOLSM_BISECT_EVALUATE) {
    mu = b.mu;
    double t = 0.0;
    nolsm_status s = nolsm_bisect_point(plan, mu, opts, stream, &t, nullptr);
    if (mu_history) mu_history[b.steps] = mu;
    if (s != NOLSM_OK) {   // the point itself failed: report it at that mu
      b.steps += 1;
      b.trace_DS = t;
      result = s;
      break;
    }
    int32_t raises_lo = 0;
    NOLSM_TRY(nolsm_bisection_update(&b, t, opts, &raises_lo));
    if (b.state != NOLSM_BISECT_ACCEPTED) NOLSM_TRY(nolsm_bisect_side(plan, opts, stream, raises_lo));
  }
  if (result == NOLSM_OK && b.state == NOLSM_BISECT_NO_PLATEAU) result = NOLSM_ERR_NO_PLATEAU;
  if (mu_out) *mu_out = mu;
  if (trace_DS_out) *trace_DS_out = b.trace_DS;
  if (steps_out) *steps_out = b.steps;
  if (result == NOLSM_ERR_NO_PLATEAU)
    set_error("nolsm_find_mu: stopped after %d evaluations at mu=%.12g with Tr(DS)=%.9f, target %.9f", b.steps, mu,
              b.trace_DS, n_occ);
  return result;
}

nolsm_status nolsm_plan_set_mlp(nolsm_plan* plan, const nolsm_mlp* mlp) {
  if (!plan) { set_error("nolsm_plan_set_mlp: NULL plan"); return NOLSM_ERR_ARG; }
  plan->mlp = mlp;
  return NOLSM_OK;
}

nolsm_status nolsm_features(nolsm_plan* plan, double mu, const nolsm_options* opts, nolsm_stream_t stream, float* feat) {
  if (!plan || !feat || !std::isfinite(mu)) { set_error("nolsm_features: invalid argument"); return NOLSM_ERR_ARG; }
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  cudaStream_t st = (cudaStream_t)stream;
  NOLSM_TRY(ensure_results(plan));
  NOLSM_TRY(prepare(plan, j0, j1, prep_class(*opts), st));
  NOLSM_TRY(features(plan, mu, j0, j1, st));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(feat + j0 * kFeatures, plan->feat.as<float>() + j0 * kFeatures,
                                 sizeof(float) * kFeatures * (size_t)(j1 - j0), cudaMemcpyDeviceToDevice, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  return NOLSM_OK;
}

nolsm_status nolsm_power_bounds(nolsm_plan* plan, const nolsm_options* opts, nolsm_stream_t stream, double* lam) {
  if (!plan) { set_error("nolsm_power_bounds: NULL plan"); return NOLSM_ERR_ARG; }
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  cudaStream_t st = (cudaStream_t)stream;
  NOLSM_TRY(ensure_results(plan));
  const int cls = prep_class(*opts);
  NOLSM_TRY(prepare(plan, j0, j1, cls, st));
  NOLSM_TRY(power_bounds(plan, cls, j0, j1, nullptr, 0, st));
  if (lam)
    NOLSM_CUDA_TRY(cudaMemcpyAsync(lam + 2 * j0, plan->lam_p.as<double>() + 2 * j0, sizeof(double) * 2 * (size_t)(j1 - j0),
                                   cudaMemcpyDeviceToDevice, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  return NOLSM_OK;
}

nolsm_status nolsm_training_data(nolsm_plan* plan, double mu, const nolsm_options* opts, nolsm_stream_t stream,
                                 float* x, float* t) {
  if (!plan || !x || !t || !std::isfinite(mu)) { set_error("nolsm_training_data: invalid argument"); return NOLSM_ERR_ARG; }
  int64_t j0, j1;
  NOLSM_TRY(check_options(plan, opts, &j0, &j1));
  nolsm_options o = *opts;
  o.bound_source = NOLSM_BOUND_POWER;
  NOLSM_TRY(nolsm_power_bounds(plan, &o, stream, nullptr));
  NOLSM_TRY(nolsm_features(plan, mu, &o, stream, x));
  NOLSM_TRY(nolsm_solve_batch(plan, mu, &o, stream, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr));
  cudaStream_t st = (cudaStream_t)stream;
  NOLSM_TRY(training_targets(plan, j0, j1, t, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  return NOLSM_OK;
}

nolsm_status nolsm_plan_stats(const nolsm_plan* plan, nolsm_stats* stats) {
  if (!plan || !stats) { set_error("nolsm_plan_stats: NULL argument"); return NOLSM_ERR_ARG; }
  *stats = plan->stats;
  return NOLSM_OK;
}

nolsm_status nolsm_plan_stats_reset(nolsm_plan* plan) {
  if (!plan) { set_error("nolsm_plan_stats_reset: NULL plan"); return NOLSM_ERR_ARG; }
  plan->stats = nolsm_stats{};
  return NOLSM_OK;
}

void nolsm_plan_destroy(nolsm_plan* plan) { delete plan; }

}  // extern "C"
