// Submatrix combination heuristic (Sec. "Submatrix Combination Heuristics", Eq. combination_criterion):
// a host-side planning step, as in the paper (there it runs once on a CPU node and its result serves many
// steps). No device code and no CUDA call.
//
// Submatrices i, j of dimensions n_i, n_j with n_c rows in common merge into one of n_i + n_j - n_c rows
// if and only if (n_i + n_j - n_c)^3 < n_i^3 + n_j^3. Start: one submatrix per molecule with rows N(J).
// A group's candidates are the groups owning a molecule among its rows. One sweep lists every ordered
// pair (i, j) that passes the criterion with its level n_j - n_c (the rows j would add to i) and gain
// n_i^3 + n_j^3 - (n_i + n_j - n_c)^3, takes the pairs by level ascending, gain descending, then i and j
// ascending, and merges a pair when neither group has merged earlier in the same sweep (the merged group
// keeps the smaller id, which is always its smallest member). Sweeps repeat until one merges nothing.
// Dimensions count basis functions; cubes are exact 128-bit integers, so the result is unique and
// independent of the number of threads that build the pair lists.
#include <algorithm>
#include <thread>
#include <vector>

#include "nolsm_internal.cuh"

namespace nolsm {
namespace {

typedef __int128 i128;

struct Pair {
  int64_t level;
  i128 gain;
  int32_t i, j;
  int64_t n_i, n_j, common;
};

bool before(const Pair& a, const Pair& b) {
  if (a.level != b.level) return a.level < b.level;
  if (a.gain != b.gain) return a.gain > b.gain;
  if (a.i != b.i) return a.i < b.i;
  return a.j < b.j;
}

inline i128 cube(int64_t n) { return (i128)n * n * n; }

struct Groups {
  const int32_t* nbf;
  std::vector<std::vector<int32_t>> rows, members;
  std::vector<int64_t> dim;
  std::vector<int32_t> group_of;

  // basis functions of the rows two groups share (both row lists ascending)
  int64_t common(int32_t i, int32_t j) const {
    const std::vector<int32_t>& a = rows[i];
    const std::vector<int32_t>& b = rows[j];
    size_t p = 0, q = 0;
    int64_t c = 0;
    while (p < a.size() && q < b.size()) {
      if (a[p] < b[q]) ++p;
      else if (b[q] < a[p]) ++q;
      else { c += nbf[a[p]]; ++p; ++q; }
    }
    return c;
  }

  void list_pairs(const std::vector<int32_t>& live, size_t first, size_t stride, std::vector<Pair>& out) const {
    std::vector<int32_t> cand;
    for (size_t k = first; k < live.size(); k += stride) {
      const int32_t i = live[k];
      cand.clear();
      for (int32_t m : rows[i])
        if (group_of[m] != i) cand.push_back(group_of[m]);
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      for (int32_t j : cand) {
        const int64_t n_i = dim[i], n_j = dim[j], c = common(i, j);
        const i128 lhs = cube(n_i + n_j - c), rhs = cube(n_i) + cube(n_j);
        if (lhs < rhs) out.push_back(Pair{n_j - c, rhs - lhs, i, j, n_i, n_j, c});
      }
    }
  }
};

}  // namespace
}  // namespace nolsm

using namespace nolsm;

nolsm_status nolsm_combine_submatrices(int32_t n_mol, const int32_t* nbf, const int32_t* nb_ptr, const int32_t* nb_idx,
                                       int32_t threads, int32_t* group_of, int32_t* n_groups, double* metrics,
                                       int32_t* sweeps) {
  if (n_mol < 0 || (n_mol > 0 && (!nbf || !nb_ptr || !nb_idx || !group_of)) || !n_groups) {
    set_error("nolsm_combine_submatrices: NULL argument or negative n_mol");
    return NOLSM_ERR_ARG;
  }
  // the input: N(J) ascending and in range, J in N(J), the relation symmetric, nbf >= 1
  if (n_mol > 0 && nb_ptr[0] != 0) { set_error("nolsm_combine_submatrices: nb_ptr[0] != 0"); return NOLSM_ERR_ARG; }
  for (int32_t J = 0; J < n_mol; ++J) {
    if (nbf[J] < 1) { set_error("nolsm_combine_submatrices: nbf[%d] < 1", J); return NOLSM_ERR_ARG; }
    if (nb_ptr[J + 1] < nb_ptr[J]) { set_error("nolsm_combine_submatrices: nb_ptr decreases at %d", J); return NOLSM_ERR_ARG; }
    bool self = false;
    for (int32_t p = nb_ptr[J]; p < nb_ptr[J + 1]; ++p) {
      const int32_t I = nb_idx[p];
      if (I < 0 || I >= n_mol || (p > nb_ptr[J] && nb_idx[p - 1] >= I)) {
        set_error("nolsm_combine_submatrices: N(%d) not ascending or out of range", J);
        return NOLSM_ERR_ARG;
      }
      self |= I == J;
    }
    if (!self) { set_error("nolsm_combine_submatrices: %d not in N(%d)", J, J); return NOLSM_ERR_ARG; }
  }
  for (int32_t J = 0; J < n_mol; ++J)
    for (int32_t p = nb_ptr[J]; p < nb_ptr[J + 1]; ++p) {
      const int32_t I = nb_idx[p];
      if (!std::binary_search(nb_idx + nb_ptr[I], nb_idx + nb_ptr[I + 1], J)) {
        set_error("nolsm_combine_submatrices: pattern not symmetric (%d in N(%d), not %d in N(%d))", I, J, J, I);
        return NOLSM_ERR_ARG;
      }
    }

  Groups g;
  g.nbf = nbf;
  g.rows.resize(n_mol);
  g.members.resize(n_mol);
  g.dim.resize(n_mol);
  g.group_of.resize(n_mol);
  double n3_0 = 0.0, n2_0 = 0.0;
  for (int32_t J = 0; J < n_mol; ++J) {
    g.rows[J].assign(nb_idx + nb_ptr[J], nb_idx + nb_ptr[J + 1]);
    g.members[J].assign(1, J);
    g.group_of[J] = J;
    int64_t d = 0;
    for (int32_t I : g.rows[J]) d += nbf[I];
    g.dim[J] = d;
    n3_0 += (double)cube(d);
    n2_0 += (double)d * (double)d;
  }
  std::vector<char> alive(n_mol, 1), touched(n_mol, 0);
  int nthreads = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
  nthreads = std::min(nthreads, 64);
  int32_t nsweeps = 0;
  std::vector<int32_t> live;
  while (true) {
    ++nsweeps;
    live.clear();
    for (int32_t J = 0; J < n_mol; ++J)
      if (alive[J]) live.push_back(J);
    const int nt = (int)std::max<size_t>(1, std::min<size_t>((size_t)nthreads, live.size() / 64));
    std::vector<std::vector<Pair>> parts(nt);
    if (nt == 1) {
      g.list_pairs(live, 0, 1, parts[0]);
    } else {
      std::vector<std::thread> pool;
      try {
        for (int t = 0; t < nt; ++t)
          pool.emplace_back([&g, &live, &parts, t, nt]() { g.list_pairs(live, (size_t)t, (size_t)nt, parts[t]); });
      } catch (...) {   // no threads to be had: the rest on this one
        for (auto& th : pool) th.join();
        for (int t = (int)pool.size(); t < nt; ++t) g.list_pairs(live, (size_t)t, (size_t)nt, parts[t]);
        pool.clear();
      }
      for (auto& th : pool) th.join();
    }
    std::vector<Pair> pairs;
    for (auto& p : parts) pairs.insert(pairs.end(), p.begin(), p.end());
    std::sort(pairs.begin(), pairs.end(), before);
    std::fill(touched.begin(), touched.end(), 0);
    int64_t merged = 0;
    for (const Pair& p : pairs) {
      if (touched[p.i] || touched[p.j]) continue;
      touched[p.i] = touched[p.j] = 1;
      const int32_t keep = std::min(p.i, p.j), gone = std::max(p.i, p.j);
      std::vector<int32_t> rows_u, mem_u;
      std::set_union(g.rows[p.i].begin(), g.rows[p.i].end(), g.rows[p.j].begin(), g.rows[p.j].end(),
                     std::back_inserter(rows_u));
      std::merge(g.members[p.i].begin(), g.members[p.i].end(), g.members[p.j].begin(), g.members[p.j].end(),
                 std::back_inserter(mem_u));
      g.rows[keep].swap(rows_u);
      g.members[keep].swap(mem_u);
      std::vector<int32_t>().swap(g.rows[gone]);
      std::vector<int32_t>().swap(g.members[gone]);
      for (int32_t m : g.members[keep]) g.group_of[m] = keep;
      g.dim[keep] = p.n_i + p.n_j - p.common;
      alive[gone] = 0;
      ++merged;
    }
    if (merged == 0) break;
  }
  double n3_1 = 0.0, n2_1 = 0.0;
  int32_t ng = 0;
  for (int32_t J = 0; J < n_mol; ++J) {
    group_of[J] = g.group_of[J];
    if (!alive[J]) continue;
    ++ng;
    n3_1 += (double)cube(g.dim[J]);
    n2_1 += (double)g.dim[J] * (double)g.dim[J];
  }
  *n_groups = ng;
  if (metrics) {
    metrics[0] = n3_0;
    metrics[1] = n3_1;
    metrics[2] = n2_0;
    metrics[3] = n2_1;
  }
  if (sweeps) *sweeps = nsweeps;
  return NOLSM_OK;
}
