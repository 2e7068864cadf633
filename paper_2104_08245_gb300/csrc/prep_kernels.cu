// a2-a3: the overlap factorisation T_J(S) = L L^T in FP64 and the solves that give
//   A_J = T_J(S)^-1 T_J(H0) = L^-T (L^-1 T_J(H0))            (Eq. purification_submatrix)
//   Q_J = T_J(S)^-1 [:, centre columns] = L^-T (L^-1 E_c)     (FP64 always)
// and the Gershgorin interval of A_J. One CTA (256 threads) per submatrix; the matrices stay in
// global memory (L2) and move through shared memory in 32-wide panels so that the arithmetic, not
// latency, bounds each phase: the Cholesky is right-looking with a 32-column panel, a panel solve and
// a tiled symmetric rank-32 update of the trailing matrix; the triangular solves are blocked by 32
// rows with one right-hand-side column per thread.
#include <algorithm>
#include <cmath>

#include "nolsm_internal.cuh"
#include "prep.cuh"

namespace nolsm {

namespace {

constexpr int NB = 32;
constexpr int kThreads = 256;

// ------------------------------------------------------------------------------------ Cholesky
// In place on the lower triangle of the n x n row-major S (upper triangle left as garbage).
// Returns false if a pivot is not positive (not SPD) or not finite.
__device__ bool cholesky_blocked(double* __restrict__ S, int n, double (*Ld)[NB + 1], double (*As)[65],
                                 double (*Bs)[65], int* s_bad) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    // (1) diagonal block, one warp, lane = row
    if (warp == 0) {
      for (int j = 0; j < kb; ++j)
        if (lane < kb) Ld[lane][j] = S[(size_t)(k0 + lane) * n + k0 + j];
      __syncwarp();
      for (int j = 0; j < kb; ++j) {
        if (lane == j) {
          const double d = Ld[j][j];
          if (!(d > 0.0) || !isfinite(d)) *s_bad = 1;
          Ld[j][j] = sqrt(fmax(d, 1e-300));
        }
        __syncwarp();
        if (lane > j && lane < kb) Ld[lane][j] /= Ld[j][j];
        __syncwarp();
        if (lane > j && lane < kb)
          for (int k = j + 1; k <= lane; ++k) Ld[lane][k] -= Ld[lane][j] * Ld[k][j];
        __syncwarp();
      }
      for (int j = 0; j < kb; ++j)
        if (lane < kb && j <= lane) S[(size_t)(k0 + lane) * n + k0 + j] = Ld[lane][j];
    }
    __syncthreads();
    if (*s_bad) return false;
    // (2) panel: rows below the block, x L_kk^T = s  (one thread per row)
    for (int i = k0 + kb + tid; i < n; i += kThreads) {
      double x[NB];
      double* Si = S + (size_t)i * n + k0;
#pragma unroll
      for (int j = 0; j < NB; ++j) x[j] = j < kb ? Si[j] : 0.0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < kb) {
          double v = x[j];
#pragma unroll
          for (int t = 0; t < j; ++t) v -= x[t] * Ld[j][t];
          x[j] = v / Ld[j][j];
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < kb) Si[j] = x[j];
    }
    __syncthreads();
    // (3) trailing update of the lower triangle, 64 x 64 tiles: S_ij -= sum_t P_it P_jt
    const int r0 = k0 + kb, m = n - r0;
    if (m <= 0) continue;
    const int T = (m + 63) / 64;
    const int tx = tid & 15, ty = tid >> 4;
    for (int tile = 0; tile < T * (T + 1) / 2; ++tile) {
      int ti = 0;
      while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
      const int tj = tile - ti * (ti + 1) / 2;
      const int bi = r0 + 64 * ti, bj = r0 + 64 * tj;
      for (int e = tid; e < 64 * NB; e += kThreads) {
        const int r = e >> 5, t = e & 31;
        As[t][r] = (bi + r < n && t < kb) ? S[(size_t)(bi + r) * n + k0 + t] : 0.0;
        Bs[t][r] = (bj + r < n && t < kb) ? S[(size_t)(bj + r) * n + k0 + t] : 0.0;
      }
      __syncthreads();
      double acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll 8
      for (int t = 0; t < NB; ++t) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[t][ty + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[t][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = bi + ty + 16 * a, j = bj + tx + 16 * b;
          if (i < n && j < n && j <= i) S[(size_t)i * n + j] -= acc[a][b];
        }
      __syncthreads();
    }
  }
  return true;
}

// ------------------------------------------------------------------------------------ triangular solves
// Column-per-thread blocked solves with the lower-triangular L (FP64, row-major, leading dim n),
// arithmetic in T. rhs(i, c) gives the right-hand side; X (leading dim ldx) receives the solution of
// L L^T X = B, columns [c0, c1) handled by this call (c - c0 < kThreads).
template <typename T, class Rhs>
__device__ void solve_llt(const double* __restrict__ L, int n, Rhs rhs, T* __restrict__ X, int ldx, int ncols,
                          T (*Lp)[NB + 1], T (*Ldg)[NB + 1]) {
  const int tid = threadIdx.x;
  for (int cb = 0; cb < ncols; cb += kThreads) {
    const int c = cb + tid;
    const bool act = c < ncols;
    // forward: L Y = B
    for (int r0 = 0; r0 < n; r0 += NB) {
      const int rb = min(NB, n - r0);
      T acc[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) acc[i] = (act && i < rb) ? rhs(r0 + i, c) : T(0);
      for (int q0 = 0; q0 < r0; q0 += NB) {
        for (int e = tid; e < NB * NB; e += kThreads) {
          const int i = e >> 5, t = e & 31;
          Lp[i][t] = i < rb ? (T)L[(size_t)(r0 + i) * n + q0 + t] : T(0);
        }
        __syncthreads();
        if (act) {
          T y[NB];
#pragma unroll
          for (int t = 0; t < NB; ++t) y[t] = X[(size_t)(q0 + t) * ldx + c];
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            T s = acc[i];
#pragma unroll
            for (int t = 0; t < NB; ++t) s -= Lp[i][t] * y[t];
            acc[i] = s;
          }
        }
        __syncthreads();
      }
      for (int e = tid; e < NB * NB; e += kThreads) {
        const int i = e >> 5, t = e & 31;
        Ldg[i][t] = (i < rb && t < rb) ? (T)L[(size_t)(r0 + i) * n + r0 + t] : T(0);
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i < rb) {
            T s = acc[i];
#pragma unroll
            for (int t = 0; t < i; ++t) s -= Ldg[i][t] * acc[t];
            acc[i] = s / Ldg[i][i];
            X[(size_t)(r0 + i) * ldx + c] = acc[i];
          }
        }
      }
      __syncthreads();
    }
    // backward: L^T X = Y, bottom block first
    const int nblk = (n + NB - 1) / NB;
    for (int rbk = nblk - 1; rbk >= 0; --rbk) {
      const int r0 = rbk * NB, rb = min(NB, n - r0);
      T acc[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) acc[i] = (act && i < rb) ? X[(size_t)(r0 + i) * ldx + c] : T(0);
      for (int q0 = r0 + NB; q0 < n; q0 += NB) {
        const int qb = min(NB, n - q0);
        for (int e = tid; e < NB * NB; e += kThreads) {
          const int t = e >> 5, i = e & 31;  // Lp[i][t] = L[q0+t][r0+i]
          Lp[i][t] = (t < qb && i < rb) ? (T)L[(size_t)(q0 + t) * n + r0 + i] : T(0);
        }
        __syncthreads();
        if (act) {
          T x[NB];
#pragma unroll
          for (int t = 0; t < NB; ++t) x[t] = t < qb ? X[(size_t)(q0 + t) * ldx + c] : T(0);
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            T s = acc[i];
#pragma unroll
            for (int t = 0; t < NB; ++t) s -= Lp[i][t] * x[t];
            acc[i] = s;
          }
        }
        __syncthreads();
      }
      for (int e = tid; e < NB * NB; e += kThreads) {
        const int i = e >> 5, t = e & 31;
        Ldg[i][t] = (i < rb && t < rb) ? (T)L[(size_t)(r0 + i) * n + r0 + t] : T(0);
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int ii = NB - 1; ii >= 0; --ii) {
          if (ii < rb) {
            T s = acc[ii];
#pragma unroll
            for (int t = ii + 1; t < NB; ++t)
              if (t < rb) s -= Ldg[t][ii] * acc[t];
            acc[ii] = s / Ldg[ii][ii];
            X[(size_t)(r0 + ii) * ldx + c] = acc[ii];
          }
        }
      }
      __syncthreads();
    }
  }
}

// The three phases use disjoint shared buffers carved from one allocation (under the 48 KB static limit).
constexpr size_t kCholBytes = sizeof(double) * (NB * (NB + 1) + 2 * NB * 65);
constexpr size_t kSolveBytes = 2 * sizeof(double) * NB * (NB + 1);

template <typename TA>
__global__ void __launch_bounds__(kThreads) k_prepare(PrepArgs g, TA* __restrict__ Acache) {
  __shared__ __align__(16) unsigned char raw[kCholBytes > kSolveBytes ? kCholBytes : kSolveBytes];
  double (*Ld)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(raw);
  double (*As)[65] = reinterpret_cast<double (*)[65]>(raw + sizeof(double) * NB * (NB + 1));
  double (*Bs)[65] = reinterpret_cast<double (*)[65]>(raw + sizeof(double) * (NB * (NB + 1) + NB * 65));
  TA (*Lp)[NB + 1] = reinterpret_cast<TA (*)[NB + 1]>(raw);
  TA (*Ldg)[NB + 1] = reinterpret_cast<TA (*)[NB + 1]>(raw + sizeof(TA) * NB * (NB + 1));
  double (*Lp64)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(raw);
  double (*Ldg64)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(raw + sizeof(double) * NB * (NB + 1));
  __shared__ int s_bad;
  __shared__ double rlo[kThreads], rhi[kThreads];
  const int J = g.j0 + blockIdx.x;
  const int n = g.sub_n[J];
  const int bJ = g.nbf[J];
  const int c0 = g.sub_c0[J];
  double* S = g.ws + (g.a_off[J] - g.a_base);
  const double* H = S + g.chunk_n2;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const bool ok = cholesky_blocked(S, n, Ld, As, Bs, &s_bad);
  if (threadIdx.x == 0) g.prep_status[J] = ok ? kSubOk : kSubNotSpd;
  if (!ok) return;   // uniform: every thread saw the same flag
  // A_J = L^-T L^-1 H in TA
  TA* A = Acache + g.a_off[J];
  solve_llt<TA>(S, n, [&](int i, int c) { return (TA)H[(size_t)i * n + c]; }, A, n, n, Lp, Ldg);
  __syncthreads();
  // Q_J = L^-T L^-1 E_c in FP64
  double* Q = g.Q + g.c_off[J];
  solve_llt<double>(S, n, [&](int i, int c) { return i == c0 + c ? 1.0 : 0.0; }, Q, bJ, bJ, Lp64, Ldg64);
  __syncthreads();
  // Gershgorin interval of A_J
  double lo = INFINITY, hi = -INFINITY;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    double r = 0.0;
    const TA* Ai = A + (size_t)i * n;
    for (int j = 0; j < n; ++j)
      if (j != i) r += fabs((double)Ai[j]);
    lo = fmin(lo, (double)Ai[i] - r);
    hi = fmax(hi, (double)Ai[i] + r);
  }
  rlo[threadIdx.x] = lo;
  rhi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      rlo[threadIdx.x] = fmin(rlo[threadIdx.x], rlo[threadIdx.x + s]);
      rhi[threadIdx.x] = fmax(rhi[threadIdx.x], rhi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    g.lam[2 * J] = rlo[0];
    g.lam[2 * J + 1] = rhi[0];
  }
}

}  // namespace

nolsm_status launch_prepare(const PrepArgs& g, int count, bool fp64_A, void* Acache, cudaStream_t st) {
  if (fp64_A)
    k_prepare<double><<<count, kThreads, 0, st>>>(g, static_cast<double*>(Acache));
  else
    k_prepare<float><<<count, kThreads, 0, st>>>(g, static_cast<float*>(Acache));
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}

}  // namespace nolsm
