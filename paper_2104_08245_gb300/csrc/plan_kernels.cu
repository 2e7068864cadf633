// a0: submatrix construction plan, built on the device (integer work, bit-exact).
//
// Merged pattern (Sec. "The Non-Orthogonal Local Submatrix Method"): row I belongs to the submatrix
// of column J when S_IJ != 0 or H0_IJ != 0; all columns of molecule J share one submatrix
// (Sec. "Simulation Details"). With structurally symmetric S and H0, the rows of column J are the
// columns of row J, so N(J) is the sorted union of block row J of S and block row J of H0.
#include <cstdio>

#include "nolsm_internal.cuh"

namespace nolsm {

namespace {

enum : int32_t {
  kBadRowPtr = 1,
  kBadCol = 2,
  kNotSymmetric = 4,
  kBadNbf = 8,
  kNoDiagonal = 16,
  kTooLarge = 32,
};

constexpr int kMaxNbf = 64;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---------------------------------------------------------------------------------- exclusive scan
// out[i] = sum_{k<i} in[k] for i in [0, n], so out[n] is the total. Three passes: tile sums, a scan of
// the tile sums in one block, and a per-tile rescan with the tile's offset.

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T w = lane < nw ? warp_tot[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T u = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += u;
    }
    if (lane < nw) warp_tot[lane] = wi - w;
    if (lane == nw - 1) *total = wi;
  }
  __syncthreads();
  T r = warp_tot[warp] + incl - v;
  __syncthreads();
  return r;
}

__global__ void k_tile_sums(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ tile_sums) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  block_exclusive_scan<int64_t>(s, wt, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_single(int64_t* __restrict__ v, int64_t n) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  int64_t carry = 0;
  for (int64_t b = 0; b < n; b += kScanTile) {
    const int64_t base = b + (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      loc[i] = base + i < n ? v[base + i] : 0;
      s += loc[i];
    }
    int64_t ex = block_exclusive_scan<int64_t>(s, wt, &tot) + carry;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      if (base + i < n) v[base + i] = ex;
      ex += loc[i];
    }
    carry += tot;
    __syncthreads();
  }
}

template <typename TO>
__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t n, const int64_t* __restrict__ tile_off,
                             TO* __restrict__ out) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t loc[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    loc[i] = base + i < n ? in[base + i] : 0;
    s += loc[i];
  }
  int64_t ex = block_exclusive_scan<int64_t>(s, wt, &tot) + tile_off[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = (TO)ex;
    ex += loc[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (TO)(tile_off[blockIdx.x] + tot);
}

// Exclusive scan of n int64 values into out[0..n]; tmp must hold ceil(n/kScanTile)+1 int64.
template <typename TO>
nolsm_status exclusive_scan(const int64_t* in, int64_t n, TO* out, int64_t* tmp, cudaStream_t st) {
  if (n == 0) {
    NOLSM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(TO), st));
    return NOLSM_OK;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp);
  NOLSM_LAUNCH_CHECK();
  k_scan_single<<<1, kScanThreads, 0, st>>>(tmp, tiles);
  NOLSM_LAUNCH_CHECK();
  k_scan_tiles<TO><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp, out);
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}

// ---------------------------------------------------------------------------------- validation

__device__ int find_sorted(const int32_t* __restrict__ a, int lo, int hi, int32_t key) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid;
  }
  return -1;
}

__global__ void k_validate(int32_t n_mol, const int32_t* __restrict__ nbf, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, int64_t nnzb, int32_t* flag) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_mol) return;
  int32_t bad = 0;
  if (nbf[I] < 1 || nbf[I] > kMaxNbf) bad |= kBadNbf;
  const int lo = rp[I], hi = rp[I + 1];
  if (I == 0 && lo != 0) bad |= kBadRowPtr;
  if (I == n_mol - 1 && (int64_t)hi != nnzb) bad |= kBadRowPtr;
  if (hi < lo || lo < 0 || (int64_t)hi > nnzb) {
    bad |= kBadRowPtr;
  } else {
    int32_t prev = -1;
    for (int p = lo; p < hi; ++p) {
      const int32_t J = ci[p];
      if (J < 0 || J >= n_mol || J <= prev) { bad |= kBadCol; break; }
      prev = J;
    }
  }
  if (bad) atomicOr(flag, bad);
}

// Structural symmetry: every stored block (I, J) has a stored (J, I). Runs only on validated input.
__global__ void k_symmetric(int32_t n_mol, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            int32_t* flag) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_mol) return;
  for (int p = rp[I]; p < rp[I + 1]; ++p) {
    const int32_t J = ci[p];
    if (find_sorted(ci, rp[J], rp[J + 1], I) < 0) { atomicOr(flag, kNotSymmetric); return; }
  }
}

// Element count of every stored block of a block-CSR matrix.
__global__ void k_block_sizes(int32_t n_mol, const int32_t* __restrict__ nbf, const int32_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, int64_t* __restrict__ sizes) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_mol) return;
  const int64_t bI = nbf[I];
  for (int p = rp[I]; p < rp[I + 1]; ++p) sizes[p] = bI * nbf[ci[p]];
}

// |N(J)|: size of the sorted union of block row J of S and of H0.
__global__ void k_nb_count(int32_t n_mol, const int32_t* __restrict__ srp, const int32_t* __restrict__ sci,
                           const int32_t* __restrict__ hrp, const int32_t* __restrict__ hci,
                           int64_t* __restrict__ count) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= n_mol) return;
  int a = srp[J], ae = srp[J + 1], b = hrp[J], be = hrp[J + 1];
  int64_t c = 0;
  while (a < ae || b < be) {
    const int32_t va = a < ae ? sci[a] : INT32_MAX;
    const int32_t vb = b < be ? hci[b] : INT32_MAX;
    if (va <= vb) ++a;
    if (vb <= va) ++b;
    ++c;
  }
  count[J] = c;
}

// N(J) in ascending order, local offsets, n_J and the offset of J's own columns.
__global__ void k_nb_fill(int32_t n_mol, const int32_t* __restrict__ nbf, const int32_t* __restrict__ srp,
                          const int32_t* __restrict__ sci, const int32_t* __restrict__ hrp,
                          const int32_t* __restrict__ hci, const int32_t* __restrict__ nb_ptr,
                          int32_t* __restrict__ nb_idx, int32_t* __restrict__ nb_off, int32_t* __restrict__ sub_n,
                          int32_t* __restrict__ sub_c0, int32_t max_n, int32_t* flag) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= n_mol) return;
  int a = srp[J], ae = srp[J + 1], b = hrp[J], be = hrp[J + 1];
  int q = nb_ptr[J];
  int32_t off = 0, c0 = -1;
  while (a < ae || b < be) {
    const int32_t va = a < ae ? sci[a] : INT32_MAX;
    const int32_t vb = b < be ? hci[b] : INT32_MAX;
    const int32_t I = va <= vb ? va : vb;
    if (va <= vb) ++a;
    if (vb <= va) ++b;
    if (I == J) c0 = off;
    nb_idx[q] = I;
    nb_off[q] = off;
    ++q;
    off += nbf[I];
  }
  sub_n[J] = off;
  sub_c0[J] = c0;
  if (c0 < 0) atomicOr(flag, kNoDiagonal);
  if (off > max_n) atomicOr(flag, kTooLarge);
}

// Per-submatrix sizes of the n^2 and n*b arrays.
__global__ void k_sub_sizes(int32_t n_mol, const int32_t* __restrict__ nbf, const int32_t* __restrict__ sub_n,
                            int64_t* __restrict__ n2, int64_t* __restrict__ nb) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= n_mol) return;
  const int64_t n = sub_n[J];
  n2[J] = n * n;
  nb[J] = n * nbf[J];
}

// For every J and every I in N(J): the slot of block (I, J) in block row I of the merged pattern.
__global__ void k_d_slot(int32_t n_mol, const int32_t* __restrict__ nb_ptr, const int32_t* __restrict__ nb_idx,
                         int32_t* __restrict__ d_slot, int32_t* flag) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= n_mol) return;
  for (int p = nb_ptr[J]; p < nb_ptr[J + 1]; ++p) {
    const int32_t I = nb_idx[p];
    const int q = find_sorted(nb_idx, nb_ptr[I], nb_ptr[I + 1], J);
    d_slot[p] = q;
    if (q < 0) atomicOr(flag, kNotSymmetric);
  }
}

nolsm_status check_flag(nolsm_plan* plan, cudaStream_t st, const char* what) {
  int32_t f = 0;
  NOLSM_CUDA_TRY(cudaMemcpyAsync(&f, plan->flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  if (f) {
    set_error("%s: malformed input (flags 0x%x: %s%s%s%s%s%s)", what, f, (f & kBadRowPtr) ? "row_ptr " : "",
              (f & kBadCol) ? "col_idx-unsorted-or-out-of-range " : "", (f & kNotSymmetric) ? "not-symmetric " : "",
              (f & kBadNbf) ? "nbf-out-of-range " : "", (f & kNoDiagonal) ? "no-diagonal-block " : "",
              (f & kTooLarge) ? "submatrix-too-large " : "");
    return NOLSM_ERR_ARG;
  }
  return NOLSM_OK;
}

}  // namespace

constexpr int32_t kMaxSubN = 4096;

nolsm_status build_plan_device(nolsm_plan* plan, cudaStream_t st) {
  const nolsm_system& s = plan->sys;
  const int32_t n = s.n_mol;
  const unsigned g = (unsigned)((n + 127) / 128);
  NOLSM_TRY(dev_alloc(plan, plan->flag, sizeof(int32_t)));
  NOLSM_CUDA_TRY(cudaMemsetAsync(plan->flag.p, 0, sizeof(int32_t), st));

  // validate both patterns
  k_validate<<<g, 128, 0, st>>>(n, s.nbf, s.s_row_ptr, s.s_col_idx, s.s_nnzb, plan->flag.as<int32_t>());
  NOLSM_LAUNCH_CHECK();
  k_validate<<<g, 128, 0, st>>>(n, s.nbf, s.h_row_ptr, s.h_col_idx, s.h_nnzb, plan->flag.as<int32_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_TRY(check_flag(plan, st, "nolsm_build_submatrices"));
  k_symmetric<<<g, 128, 0, st>>>(n, s.s_row_ptr, s.s_col_idx, plan->flag.as<int32_t>());
  NOLSM_LAUNCH_CHECK();
  k_symmetric<<<g, 128, 0, st>>>(n, s.h_row_ptr, s.h_col_idx, plan->flag.as<int32_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_TRY(check_flag(plan, st, "nolsm_build_submatrices"));

  // scratch for sizes and scans
  const int64_t big = std::max<int64_t>(std::max<int64_t>(s.s_nnzb, s.h_nnzb), n) + 1;
  DevBuf sizes, tmp, cnt;
  NOLSM_TRY(dev_alloc(plan, sizes, sizeof(int64_t) * (size_t)big));
  NOLSM_TRY(dev_alloc(plan, tmp, sizeof(int64_t) * (size_t)(big / kScanTile + 2)));
  NOLSM_TRY(dev_alloc(plan, cnt, sizeof(int64_t) * (size_t)(n + 1)));

  // element offsets of the S and H0 blocks
  NOLSM_TRY(dev_alloc(plan, plan->s_blk_off, sizeof(int64_t) * (size_t)(s.s_nnzb + 1)));
  NOLSM_TRY(dev_alloc(plan, plan->h_blk_off, sizeof(int64_t) * (size_t)(s.h_nnzb + 1)));
  k_block_sizes<<<g, 128, 0, st>>>(n, s.nbf, s.s_row_ptr, s.s_col_idx, sizes.as<int64_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_TRY(exclusive_scan<int64_t>(sizes.as<int64_t>(), s.s_nnzb, plan->s_blk_off.as<int64_t>(),
                                    tmp.as<int64_t>(), st));
  k_block_sizes<<<g, 128, 0, st>>>(n, s.nbf, s.h_row_ptr, s.h_col_idx, sizes.as<int64_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_TRY(exclusive_scan<int64_t>(sizes.as<int64_t>(), s.h_nnzb, plan->h_blk_off.as<int64_t>(),
                                    tmp.as<int64_t>(), st));

  // merged neighbourhoods
  NOLSM_TRY(dev_alloc(plan, plan->nb_ptr, sizeof(int32_t) * (size_t)(n + 1)));
  k_nb_count<<<g, 128, 0, st>>>(n, s.s_row_ptr, s.s_col_idx, s.h_row_ptr, s.h_col_idx, cnt.as<int64_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_TRY(exclusive_scan<int32_t>(cnt.as<int64_t>(), n, plan->nb_ptr.as<int32_t>(), tmp.as<int64_t>(), st));
  int32_t total = 0;
  NOLSM_CUDA_TRY(cudaMemcpyAsync(&total, plan->nb_ptr.as<int32_t>() + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  plan->d_nnzb = total;
  NOLSM_TRY(dev_alloc(plan, plan->nb_idx, sizeof(int32_t) * (size_t)std::max(total, 1)));
  NOLSM_TRY(dev_alloc(plan, plan->nb_off, sizeof(int32_t) * (size_t)std::max(total, 1)));
  NOLSM_TRY(dev_alloc(plan, plan->d_slot, sizeof(int32_t) * (size_t)std::max(total, 1)));
  NOLSM_TRY(dev_alloc(plan, plan->sub_n, sizeof(int32_t) * (size_t)n));
  NOLSM_TRY(dev_alloc(plan, plan->sub_c0, sizeof(int32_t) * (size_t)n));
  k_nb_fill<<<g, 128, 0, st>>>(n, s.nbf, s.s_row_ptr, s.s_col_idx, s.h_row_ptr, s.h_col_idx,
                               plan->nb_ptr.as<int32_t>(), plan->nb_idx.as<int32_t>(), plan->nb_off.as<int32_t>(),
                               plan->sub_n.as<int32_t>(), plan->sub_c0.as<int32_t>(), kMaxSubN,
                               plan->flag.as<int32_t>());
  NOLSM_LAUNCH_CHECK();
  k_d_slot<<<g, 128, 0, st>>>(n, plan->nb_ptr.as<int32_t>(), plan->nb_idx.as<int32_t>(), plan->d_slot.as<int32_t>(),
                              plan->flag.as<int32_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_TRY(check_flag(plan, st, "nolsm_build_submatrices"));

  // D block offsets: block row I of D is N(I)
  if ((int64_t)total + 1 > big) {
    dev_free(plan, sizes);
    NOLSM_TRY(dev_alloc(plan, sizes, sizeof(int64_t) * (size_t)(total + 1)));
    dev_free(plan, tmp);
    NOLSM_TRY(dev_alloc(plan, tmp, sizeof(int64_t) * (size_t)(total / kScanTile + 2)));
  }
  NOLSM_TRY(dev_alloc(plan, plan->d_blk_off, sizeof(int64_t) * (size_t)(total + 1)));
  k_block_sizes<<<g, 128, 0, st>>>(n, s.nbf, plan->nb_ptr.as<int32_t>(), plan->nb_idx.as<int32_t>(),
                                   sizes.as<int64_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_TRY(exclusive_scan<int64_t>(sizes.as<int64_t>(), total, plan->d_blk_off.as<int64_t>(), tmp.as<int64_t>(), st));

  // offsets of the per-submatrix n^2 and n*b arrays
  DevBuf nb_sz;
  NOLSM_TRY(dev_alloc(plan, nb_sz, sizeof(int64_t) * (size_t)(n + 1)));
  NOLSM_TRY(dev_alloc(plan, plan->a_off, sizeof(int64_t) * (size_t)(n + 1)));
  NOLSM_TRY(dev_alloc(plan, plan->c_off, sizeof(int64_t) * (size_t)(n + 1)));
  k_sub_sizes<<<g, 128, 0, st>>>(n, s.nbf, plan->sub_n.as<int32_t>(), cnt.as<int64_t>(), nb_sz.as<int64_t>());
  NOLSM_LAUNCH_CHECK();
  NOLSM_TRY(exclusive_scan<int64_t>(cnt.as<int64_t>(), n, plan->a_off.as<int64_t>(), tmp.as<int64_t>(), st));
  NOLSM_TRY(exclusive_scan<int64_t>(nb_sz.as<int64_t>(), n, plan->c_off.as<int64_t>(), tmp.as<int64_t>(), st));

  // host copies
  plan->h_sub_n.resize(n);
  plan->h_nbf.resize(n);
  plan->h_nb_ptr.resize(n + 1);
  plan->h_a_off.resize(n + 1);
  plan->h_c_off.resize(n + 1);
  NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->h_sub_n.data(), plan->sub_n.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->h_nbf.data(), s.nbf, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  NOLSM_TRY(dev_alloc(plan, plan->sub_b, sizeof(int32_t) * (size_t)n));   // one submatrix per molecule: b_J
  NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->sub_b.p, s.nbf, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->h_nb_ptr.data(), plan->nb_ptr.p, sizeof(int32_t) * (n + 1),
                                 cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->h_a_off.data(), plan->a_off.p, sizeof(int64_t) * (n + 1),
                                 cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->h_c_off.data(), plan->c_off.p, sizeof(int64_t) * (n + 1),
                                 cudaMemcpyDeviceToHost, st));
  int64_t dvals = 0;
  NOLSM_CUDA_TRY(cudaMemcpyAsync(&dvals, plan->d_blk_off.as<int64_t>() + total, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  plan->d_nvals = dvals;
  dev_free(plan, sizes);
  dev_free(plan, tmp);
  dev_free(plan, cnt);
  dev_free(plan, nb_sz);

  plan->stats.launches += 28;   // validation, block sizes, scans (3 kernels each), merge, slots
  plan->max_n = 0;
  plan->min_n = INT32_MAX;
  plan->max_b = 0;
  plan->sum_n3 = 0.0;
  for (int32_t J = 0; J < n; ++J) {
    const int32_t m = plan->h_sub_n[J];
    plan->max_n = std::max(plan->max_n, m);
    plan->min_n = std::min(plan->min_n, m);
    plan->max_b = std::max(plan->max_b, plan->h_nbf[J]);
    plan->h_sub_b.push_back(plan->h_nbf[J]);
    plan->sum_n3 += (double)m * m * m;
  }
  return NOLSM_OK;
}

}  // namespace nolsm
