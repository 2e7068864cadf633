// Energy-weighted density matrix of the submatrix method (NOLSM section: W = D H0 D, needed for the
// Pulay forces, and its submatrix form T_J(W) = T_J(D) T_J(H0) T_J(D)), centre columns only.
//
// With A_J = T_J(S)^-1 T_J(H0) and P = 1/2 (I - sign(A_J - mu I)), T_J(D) = P T_J(S)^-1. P is a function of
// A_J, so it commutes with A_J, and P^2 = P; hence
//   T_J(W) = P T_J(S)^-1 T_J(H0) P T_J(S)^-1 = P A_J P T_J(S)^-1 = A_J P T_J(S)^-1 = A_J T_J(D),
// and the centre columns are W_c = A_J D_c: one n x n by n x b product per submatrix on data the solve
// already holds (A_J from the preparation, D_c from the sign iteration), instead of the two n x n x n
// products of the definition. The kernel is bound by reading A_J from HBM (n^2 x 4 or 8 bytes per
// submatrix against n^2 b multiply-adds).
//
// Precision: the FP64 path multiplies its FP64 A_J by D_c in FP64. The tensor-core paths multiply the
// FP32 A_J their sign iteration starts from by D_c rounded to FP32, with FP32 accumulation; the error
// of W_c is then about ||A_J|| times the error of D_c plus sqrt(n) FP32 roundings of |A_J| |D_c|.
#include <algorithm>

#include "nolsm_internal.cuh"

namespace nolsm {
namespace {

constexpr int kEwThreads = 256;
constexpr int kEwWarps = kEwThreads / 32;
constexpr int kEwCols = 8;   // centre columns per pass (D_c staged in shared memory as [n][8])
constexpr int kEwRows = 4;   // rows of A_J per warp pass: 4 x 8 partial sums per lane
constexpr int kEwU = 8;      // k values per lane loaded ahead (rows of up to 256 elements in one chunk)

struct EwArgs {
  int32_t j0;
  const int32_t* sub_n;
  const int32_t* nbf;
  const int64_t* a_off;
  const int64_t* c_off;
  const double* Dc;   // centre columns of T_J(D), n x b row-major at c_off[J]
  const double* Sc;   // centre columns of T_J(S), same layout
  double* Wd;         // centre columns of T_J(W), same layout
  double* tW;         // [n_mol]: sum over centre columns j and rows i of T_J(W)_ij T_J(S)_ij
  const void* a_end;  // end of the A_J array (bound of the L2 prefetch)
};

// Asks the TMA unit to bring [p, p + bytes) into L2 (p and bytes multiples of 16; no completion to wait for).
__device__ __forceinline__ void prefetch_l2(uintptr_t p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void load8(const float* p, float (&v)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void load8(const double* p, double (&v)[8]) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const double2 a = *reinterpret_cast<const double2*>(p + 2 * h);
    v[2 * h] = a.x;
    v[2 * h + 1] = a.y;
  }
}

// Sum of v[L] over the 32 lanes of the warp, returned to lane L (a butterfly reduce-scatter: at each
// level a lane keeps the half of its values selected by one bit of its lane index and adds the
// partner's copy of that half).
template <typename T>
__device__ __forceinline__ T reduce_scatter32(T (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const T send = up ? v[j] : v[j + h];
      const T keep = up ? v[j + h] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0];
}

// One CTA per submatrix; one thread asks for all of A_J in L2 (bulk prefetch), then warps take 4 rows of
// A_J at a time, lanes stride over k (coalesced rows) and load up to 8 k values of each row ahead.
template <typename TA>
__global__ void __launch_bounds__(kEwThreads) k_energy_weighted(EwArgs g, const TA* __restrict__ A_all) {
  extern __shared__ __align__(16) unsigned char ew_smem[];
  TA* ds = reinterpret_cast<TA*>(ew_smem);   // [n][kEwCols]
  __shared__ double red[kEwWarps];
  const int J = g.j0 + (int)blockIdx.x;
  const int n = g.sub_n[J], b = g.nbf[J];
  const TA* __restrict__ A = A_all + g.a_off[J];
  const double* __restrict__ d = g.Dc + g.c_off[J];
  const double* __restrict__ S = g.Sc + g.c_off[J];
  double* __restrict__ W = g.Wd + g.c_off[J];
  const int tid = threadIdx.x, lane = tid & 31, wrp = tid >> 5;
  if (tid == 0) {
    // the whole of A_J into L2 at once, so that the warps' row loads below find it there: the start rounded
    // down and the end rounded down to 16 bytes stay inside the A array
    const uintptr_t lo = reinterpret_cast<uintptr_t>(A) & ~static_cast<uintptr_t>(15);
    const uintptr_t hi = min(reinterpret_cast<uintptr_t>(A + (size_t)n * n), reinterpret_cast<uintptr_t>(g.a_end)) &
                         ~static_cast<uintptr_t>(15);
    for (uintptr_t q = lo; q < hi; q += 32768) prefetch_l2(q, (uint32_t)min(static_cast<uintptr_t>(32768), hi - q));
  }
  double tw = 0.0;
  for (int c0 = 0; c0 < b; c0 += kEwCols) {
    const int cb = min(kEwCols, b - c0);
    __syncthreads();   // the previous pass has finished reading ds
    for (int e = tid; e < n * kEwCols; e += kEwThreads) {
      const int k = e >> 3, c = e & 7;
      ds[e] = c < cb ? (TA)d[(size_t)k * b + c0 + c] : (TA)0;
    }
    __syncthreads();
    for (int i0 = kEwRows * wrp; i0 < n; i0 += kEwRows * kEwWarps) {
      // rows past n read row n - 1 (in bounds); their sums are discarded
      const TA* __restrict__ arow[kEwRows];
#pragma unroll
      for (int r = 0; r < kEwRows; ++r) arow[r] = A + (size_t)min(i0 + r, n - 1) * n;
      TA acc[kEwRows * kEwCols];
#pragma unroll
      for (int v = 0; v < kEwRows * kEwCols; ++v) acc[v] = (TA)0;
      for (int kb = 0; kb < n; kb += 32 * kEwU) {
        // every load of the chunk is issued before the first multiply (kEwU x 4 loads in flight per lane)
        TA av[kEwU][kEwRows];
#pragma unroll
        for (int u = 0; u < kEwU; ++u) {
          const int k = kb + lane + 32 * u;
#pragma unroll
          for (int r = 0; r < kEwRows; ++r) av[u][r] = k < n ? arow[r][k] : (TA)0;
        }
#pragma unroll
        for (int u = 0; u < kEwU; ++u) {
          const int k = kb + lane + 32 * u;
          if (k < n) {
            TA dv[kEwCols];
            load8(ds + k * kEwCols, dv);
#pragma unroll
            for (int r = 0; r < kEwRows; ++r)
#pragma unroll
              for (int c = 0; c < kEwCols; ++c) acc[r * kEwCols + c] = fma(av[u][r], dv[c], acc[r * kEwCols + c]);
          }
        }
      }
      const TA sum = reduce_scatter32(acc, lane);
      const int i = i0 + (lane >> 3), c = lane & 7;
      if (i < n && c < cb) {
        const double w = (double)sum;
        W[(size_t)i * b + c0 + c] = w;
        tw += w * S[(size_t)i * b + c0 + c];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) tw += __shfl_down_sync(0xffffffffu, tw, o);
  if (lane == 0) red[wrp] = tw;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kEwWarps; ++w) s += red[w];
    g.tW[J] = s;
  }
}

// Sum of x[j0, j1) in a fixed order (one block).
__global__ void __launch_bounds__(256) k_sum_range(int32_t j0, int32_t j1, const double* __restrict__ x,
                                                   double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int J = j0 + threadIdx.x; J < j1; J += blockDim.x) s += x[J];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *out = t;
  }
}

template <typename TA>
nolsm_status launch_ew(const EwArgs& g, int count, int max_n, const TA* A, cudaStream_t st) {
  const size_t smem = sizeof(TA) * kEwCols * (size_t)std::max(max_n, 1);
  if (smem > 227u * 1024u) {
    set_error("nolsm_energy_weighted: submatrix dimension %d exceeds the shared-memory stage of D_c", max_n);
    return NOLSM_ERR_UNSUPPORTED;
  }
  if (smem > 48u * 1024u)
    NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_energy_weighted<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
  k_energy_weighted<TA><<<count, kEwThreads, smem, st>>>(g, A);
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}

}  // namespace

nolsm_status energy_weighted(nolsm_plan* plan, cudaStream_t st, double* W_vals, double* trace_WS) {
  const int64_t j0 = plan->solved_begin, j1 = plan->solved_end;
  const int cls = plan->solved_cls;
  if (cls == kPrepSym) {
    set_error("nolsm_energy_weighted: the last solve used the symmetric form, which keeps "
              "L^-1 T_J(H0) L^-T instead of T_J(S)^-1 T_J(H0)");
    return NOLSM_ERR_UNSUPPORTED;
  }
  const int32_t n_mol = plan->n_mol;
  if (!plan->Wd.p) {
    NOLSM_TRY(dev_alloc(plan, plan->Wd, sizeof(double) * (size_t)std::max<int64_t>(plan->h_c_off[n_mol], 1)));
    NOLSM_TRY(dev_alloc(plan, plan->tW, sizeof(double) * (size_t)std::max(n_mol, 1)));
  }
  int32_t max_n = 1;
  for (int64_t J = j0; J < j1; ++J) max_n = std::max(max_n, plan->h_sub_n[J]);
  EwArgs g;
  g.j0 = (int32_t)j0;
  g.sub_n = plan->sub_n.as<int32_t>();
  g.nbf = plan->sub_b.as<int32_t>();   // centre columns per submatrix
  g.a_off = plan->a_off.as<int64_t>();
  g.c_off = plan->c_off.as<int64_t>();
  g.Dc = plan->Dc.as<double>();
  g.Sc = plan->Sc.as<double>();
  g.Wd = plan->Wd.as<double>();
  g.tW = plan->tW.as<double>();
  const int count = (int)(j1 - j0);
  const Prepared& P = prepared(plan, cls);
  g.a_end = static_cast<const char*>(P.A.p) + (cls == kPrepFP64 ? sizeof(double) : sizeof(float)) * plan->h_a_off[n_mol];
  mark(plan, 6, st);
  if (count > 0) {
    if (cls == kPrepFP64) NOLSM_TRY(launch_ew<double>(g, count, max_n, P.A.as<double>(), st));
    else NOLSM_TRY(launch_ew<float>(g, count, max_n, P.A.as<float>(), st));
    plan->stats.launches += 1;
  }
  mark(plan, 7, st);
  if (W_vals) NOLSM_TRY(scatter(plan, W_vals, j0, j1, st, plan->Wd.as<double>()));
  double tw = 0.0;
  if (trace_WS && count > 0) {
    k_sum_range<<<1, 256, 0, st>>>((int32_t)j0, (int32_t)j1, plan->tW.as<double>(), plan->sums.as<double>());
    NOLSM_LAUNCH_CHECK();
    plan->stats.launches += 1;
    NOLSM_CUDA_TRY(cudaMemcpyAsync(&tw, plan->sums.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  plan->stats.ms_energy_weighted += elapsed(plan, 6, 7);
  if (trace_WS) *trace_WS = tw;
  return NOLSM_OK;
}

}  // namespace nolsm

using namespace nolsm;

nolsm_status nolsm_energy_weighted(nolsm_plan* plan, nolsm_stream_t stream, double* W_vals, double* trace_WS) {
  if (!plan) { set_error("nolsm_energy_weighted: NULL plan"); return NOLSM_ERR_ARG; }
  if (!plan->have_solution) { set_error("nolsm_energy_weighted: no solve yet"); return NOLSM_ERR_NO_SOLUTION; }
  return energy_weighted(plan, (cudaStream_t)stream, W_vals, trace_WS);
}
