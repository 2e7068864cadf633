// Merged submatrices (Sec. "Submatrix Combination Heuristics"): a plan whose submatrices are groups of
// molecules. The submatrix of group G covers N(G), the union of its members' N(J), with the members' rows
// first (members ascending) and the other molecules of N(G) after them (ascending), so that the centre
// columns of T_G, the functions of all members, are the first b_G = sum of the members' b_J columns and
// every kernel of the per-molecule path runs on T_G unchanged (centre offset 0, centre width b_G). Eq.
// purification_submatrix on T_G gives T_G(D); member J's columns of it are written back on the rows of its
// own N(J), so that D keeps the merged pattern of S and H0 of the per-molecule plan. Tr(DS) of the groups
// equals that of the written-back D: a row outside N(J) has S_ij = 0 in J's columns.
#include <algorithm>
#include <new>
#include <vector>

#include "nolsm_internal.cuh"

namespace nolsm {

namespace {

constexpr int32_t kMaxCentre = 64;   // centre columns the preparation's column tiles hold

// one warp per molecule pair p = (J, I in N(J)) of the per-molecule pattern: block (I, J) of D <- rows of I
// and columns of J in the centre columns of T_G(D), G the group of J
__global__ void __launch_bounds__(256) k_scatter_grouped(int32_t n_mol, int64_t p_count, const int32_t* __restrict__ nbf,
                                                         const int32_t* __restrict__ m_nb_ptr,
                                                         const int32_t* __restrict__ m_nb_idx,
                                                         const int32_t* __restrict__ d_slot,
                                                         const int64_t* __restrict__ d_blk_off,
                                                         const int32_t* __restrict__ g_of, const int32_t* __restrict__ g_col,
                                                         const int32_t* __restrict__ g_row, const int32_t* __restrict__ sub_b,
                                                         const int64_t* __restrict__ c_off, int32_t j0, int32_t j1,
                                                         const double* __restrict__ Dc, double* __restrict__ D) {
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (p >= p_count) return;
  int lo = 0, hi = n_mol;   // owner J of pair p: m_nb_ptr[J] <= p < m_nb_ptr[J + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)m_nb_ptr[mid] <= p) lo = mid; else hi = mid;
  }
  const int J = lo;
  const int G = g_of[J];
  if (G < j0 || G >= j1) return;   // the group was not in the last solved range
  const int I = m_nb_idx[p];
  const int bI = nbf[I], bJ = nbf[J], bG = sub_b[G];
  const double* src = Dc + c_off[G] + (int64_t)g_row[p] * bG + g_col[J];
  double* dst = D + d_blk_off[d_slot[p]];
  for (int e = lane; e < bI * bJ; e += 32) {
    const int r = e / bJ, c = e - r * bJ;
    dst[e] = src[(int64_t)r * bG + c];
  }
}

template <typename T>
nolsm_status upload(nolsm_plan* plan, DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
  NOLSM_TRY(dev_alloc(plan, b, sizeof(T) * std::max<size_t>(v.size(), 1)));
  if (!v.empty()) NOLSM_CUDA_TRY(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return NOLSM_OK;
}

nolsm_status copy_dev(nolsm_plan* plan, DevBuf& dst, const DevBuf& src, cudaStream_t st) {
  NOLSM_TRY(dev_alloc(plan, dst, src.bytes));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(dst.p, src.p, src.bytes, cudaMemcpyDeviceToDevice, st));
  return NOLSM_OK;
}

}  // namespace

nolsm_status scatter_grouped(nolsm_plan* plan, double* D, int64_t j0, int64_t j1, cudaStream_t st, const double* src) {
  const int64_t pairs = plan->d_nnzb;
  if (pairs <= 0) return NOLSM_OK;
  k_scatter_grouped<<<(unsigned)((pairs * 32 + 255) / 256), 256, 0, st>>>(
      plan->sys.n_mol, pairs, plan->sys.nbf, plan->m_nb_ptr.as<int32_t>(), plan->m_nb_idx.as<int32_t>(),
      plan->d_slot.as<int32_t>(), plan->d_blk_off.as<int64_t>(), plan->g_of.as<int32_t>(), plan->g_col.as<int32_t>(),
      plan->g_row.as<int32_t>(), plan->sub_b.as<int32_t>(), plan->c_off.as<int64_t>(), (int32_t)j0, (int32_t)j1,
      src ? src : plan->Dc.as<double>(), D);
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 1;
  return NOLSM_OK;
}

}  // namespace nolsm

using namespace nolsm;

extern "C" nolsm_status nolsm_build_grouped(const nolsm_plan* mp, const int32_t* group_of, nolsm_stream_t stream,
                                            nolsm_plan** out) {
  if (!out) { set_error("nolsm_build_grouped: out is NULL"); return NOLSM_ERR_ARG; }
  *out = nullptr;
  if (!mp || !group_of) { set_error("nolsm_build_grouped: NULL argument"); return NOLSM_ERR_ARG; }
  if (mp->grouped) { set_error("nolsm_build_grouped: the plan is grouped already"); return NOLSM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = mp->n_mol;
  const int64_t m = mp->d_nnzb;
  std::vector<int32_t> nb_idx((size_t)m), nb_off((size_t)m);
  NOLSM_CUDA_TRY(cudaMemcpyAsync(nb_idx.data(), mp->nb_idx.p, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(nb_off.data(), mp->nb_off.p, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  const std::vector<int32_t>& nbf = mp->h_nbf;
  const std::vector<int32_t>& ptr = mp->h_nb_ptr;

  // groups in order of their smallest member; members ascending
  std::vector<int32_t> gidx((size_t)n, -1), label_to((size_t)n, -1);
  std::vector<std::vector<int32_t>> members;
  for (int32_t J = 0; J < n; ++J) {
    const int32_t l = group_of[J];
    if (l < 0 || l >= n) {
      set_error("nolsm_build_grouped: group_of[%d] = %d is not a molecule index", J, l);
      return NOLSM_ERR_ARG;
    }
    if (label_to[(size_t)l] < 0) {
      label_to[(size_t)l] = (int32_t)members.size();
      members.emplace_back();
    }
    gidx[(size_t)J] = label_to[(size_t)l];
    members[(size_t)gidx[(size_t)J]].push_back(J);
  }
  const int32_t G = (int32_t)members.size();

  // rows of every group: members, then the rest of the union of their N(J); offsets of every molecule in it
  std::vector<int32_t> gnb_ptr((size_t)G + 1, 0), gnb_idx, gnb_off, gsub_n((size_t)G), gsub_b((size_t)G),
      g_col((size_t)n), g_row((size_t)m);
  std::vector<int32_t> pos((size_t)n, -1), stamp((size_t)n, -1);
  for (int32_t g = 0; g < G; ++g) {
    std::vector<int32_t> rest;
    for (int32_t J : members[(size_t)g]) stamp[(size_t)J] = g;
    for (int32_t J : members[(size_t)g])
      for (int32_t p = ptr[(size_t)J]; p < ptr[(size_t)J + 1]; ++p) {
        const int32_t I = nb_idx[(size_t)p];
        if (stamp[(size_t)I] != g) {
          stamp[(size_t)I] = g;
          rest.push_back(I);
        }
      }
    std::sort(rest.begin(), rest.end());
    int32_t off = 0, b = 0;
    auto add = [&](int32_t I) {
      pos[(size_t)I] = off;
      gnb_idx.push_back(I);
      gnb_off.push_back(off);
      off += nbf[(size_t)I];
    };
    for (int32_t J : members[(size_t)g]) {
      add(J);
      b += nbf[(size_t)J];
    }
    for (int32_t I : rest) add(I);
    gnb_ptr[(size_t)g + 1] = (int32_t)gnb_idx.size();
    gsub_n[(size_t)g] = off;
    gsub_b[(size_t)g] = b;
    for (int32_t J : members[(size_t)g]) {
      g_col[(size_t)J] = pos[(size_t)J];
      for (int32_t p = ptr[(size_t)J]; p < ptr[(size_t)J + 1]; ++p) g_row[(size_t)p] = pos[(size_t)nb_idx[(size_t)p]];
    }
  }
  for (int32_t g = 0; g < G; ++g)
    if (gsub_b[(size_t)g] > kMaxCentre) {
      set_error("nolsm_build_grouped: group %d has %d centre columns (its members' functions); a submatrix takes "
                "at most %d", g, gsub_b[(size_t)g], kMaxCentre);
      return NOLSM_ERR_UNSUPPORTED;
    }
  std::vector<int64_t> a_off((size_t)G + 1, 0), c_off((size_t)G + 1, 0);
  for (int32_t g = 0; g < G; ++g) {
    const int64_t ng = gsub_n[(size_t)g];
    a_off[(size_t)g + 1] = a_off[(size_t)g] + ng * ng;
    c_off[(size_t)g + 1] = c_off[(size_t)g] + ng * gsub_b[(size_t)g];
  }

  nolsm_plan* plan = new (std::nothrow) nolsm_plan();
  if (!plan) { set_error("host allocation failed"); return NOLSM_ERR_OOM; }
  plan->sys = mp->sys;
  plan->n_mol = G;
  plan->grouped = true;
  plan->ev_ok = true;
  for (cudaEvent_t& e : plan->ev)
    if (cudaEventCreate(&e) != cudaSuccess) plan->ev_ok = false;
  if (!plan->ev_ok) cudaGetLastError();
  auto fail = [&](nolsm_status s) {
    delete plan;
    return s;
  };
#define GR_TRY(expr)                           \
  do {                                         \
    nolsm_status _s = (expr);                  \
    if (_s != NOLSM_OK) return fail(_s);       \
  } while (0)
  std::vector<int32_t> zeros((size_t)G, 0);
  GR_TRY(upload(plan, plan->nb_ptr, gnb_ptr, st));
  GR_TRY(upload(plan, plan->nb_idx, gnb_idx, st));
  GR_TRY(upload(plan, plan->nb_off, gnb_off, st));
  GR_TRY(upload(plan, plan->sub_n, gsub_n, st));
  GR_TRY(upload(plan, plan->sub_c0, zeros, st));
  GR_TRY(upload(plan, plan->sub_b, gsub_b, st));
  GR_TRY(upload(plan, plan->a_off, a_off, st));
  GR_TRY(upload(plan, plan->c_off, c_off, st));
  GR_TRY(upload(plan, plan->g_of, gidx, st));
  GR_TRY(upload(plan, plan->g_col, g_col, st));
  GR_TRY(upload(plan, plan->g_row, g_row, st));
  GR_TRY(copy_dev(plan, plan->s_blk_off, mp->s_blk_off, st));
  GR_TRY(copy_dev(plan, plan->h_blk_off, mp->h_blk_off, st));
  GR_TRY(copy_dev(plan, plan->d_slot, mp->d_slot, st));
  GR_TRY(copy_dev(plan, plan->d_blk_off, mp->d_blk_off, st));
  GR_TRY(copy_dev(plan, plan->m_nb_ptr, mp->nb_ptr, st));
  GR_TRY(copy_dev(plan, plan->m_nb_idx, mp->nb_idx, st));
  GR_TRY(dev_alloc(plan, plan->flag, sizeof(int32_t)));
  if (mp->gen) {   // elements generated from the geometry, as in the per-molecule plan
    GR_TRY(copy_dev(plan, plan->onsite_off, mp->onsite_off, st));
    plan->gen = true;
    plan->model = mp->model;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    set_error("nolsm_build_grouped: copying the maps failed");
    return fail(NOLSM_ERR_CUDA);
  }
#undef GR_TRY
  plan->d_nnzb = mp->d_nnzb;
  plan->d_nvals = mp->d_nvals;
  plan->h_sub_n = gsub_n;
  plan->h_sub_b = gsub_b;
  plan->h_nbf = mp->h_nbf;
  plan->h_nb_ptr = gnb_ptr;
  plan->h_a_off = a_off;
  plan->h_c_off = c_off;
  plan->max_n = 0;
  plan->min_n = INT32_MAX;
  plan->max_b = 0;
  plan->sum_n3 = 0.0;
  for (int32_t g = 0; g < G; ++g) {
    plan->max_n = std::max(plan->max_n, gsub_n[(size_t)g]);
    plan->min_n = std::min(plan->min_n, gsub_n[(size_t)g]);
    plan->max_b = std::max(plan->max_b, gsub_b[(size_t)g]);
    plan->sum_n3 += (double)gsub_n[(size_t)g] * gsub_n[(size_t)g] * gsub_n[(size_t)g];
  }
  *out = plan;
  return NOLSM_OK;
}
