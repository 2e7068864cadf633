// a2-a3: the overlap factorisation T_J(S) = L L^T in FP64 and the solves that give
//   A_J = T_J(S)^-1 T_J(H0) = L^-T (L^-1 T_J(H0))            (Eq. purification_submatrix)
//   Q_J = T_J(S)^-1 [:, centre columns] = L^-T (L^-1 E_c)     (FP64 always)
// and the Gershgorin interval of A_J. One CTA (128 threads) per submatrix, two CTAs per SM.
//
// FP64 runs at 2 lanes per clock per SM on this GPU (one full-warp FP64 instruction per 64 cycles per
// scheduler), so every FP64 instruction here is issued by full warps spread over all schedulers and no
// FP64 work is a dependent chain: the Cholesky factors a 32-column panel held in shared memory one
// column at a time in parallel over its rows, and builds the inverse X_r of the panel's diagonal block
// in the same sweep (column-oriented forward substitution on the identity). The triangular solves then
// apply X_r as a product instead of substituting row by row. X_r is kept, transposed, in the unused
// upper triangle of its diagonal block (its diagonal is 1/L_ii).
#include <algorithm>
#include <cmath>

#include "nolsm_internal.cuh"
#include "prep.cuh"

namespace nolsm {

namespace {

constexpr int NB = 32;
constexpr int kThreads = 128;   // two CTAs (two submatrices) per SM overlap each other's serial phases
constexpr int kMaxB = 64;

// X_r[a][t] for a, t < kb: lower-triangular inverse of the diagonal block starting at r0.
__device__ __forceinline__ double xinv(const double* S, int n, int r0, int a, int t) {
  if (t > a) return 0.0;
  if (t == a) return 1.0 / S[(size_t)(r0 + a) * n + r0 + a];
  return S[(size_t)(r0 + t) * n + r0 + a];  // stored transposed in the upper triangle
}

// ------------------------------------------------------------------------------------ Cholesky
// In place: the lower triangle of S receives L; the strict upper triangle of every diagonal block
// receives X_r^T. Returns false (uniformly) if a pivot is not positive or not finite.
__device__ bool cholesky(double* __restrict__ S, int n, double* __restrict__ Ps, double (*Xs)[NB + 1],
                         double* s_rinv /* [2] */, int* s_bad) {
  const int tid = threadIdx.x;
  constexpr int LDP = NB + 1;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0), mt = n - k0;
    for (int e = tid; e < mt * kb; e += kThreads) {
      const int i = e / kb, t = e - i * kb;
      Ps[i * LDP + t] = S[(size_t)(k0 + i) * n + k0 + t];
    }
    for (int e = tid; e < NB * NB; e += kThreads) Xs[e >> 5][e & 31] = ((e >> 5) == (e & 31)) ? 1.0 : 0.0;
    __syncthreads();
    // Column j: phase A scales column j-1 and row j-1 of X by r_{j-1} while thread 0 forms the pivot of
    // column j (FP32 rsqrt seed, two FP64 Newton steps); phase B updates the panel and X with the
    // unscaled column j times r_j^2.
    for (int j = 0; j <= kb; ++j) {
      if (j > 0) {
        const double rp = *s_rinv;
        for (int i = j + tid; i < mt; i += kThreads) Ps[i * LDP + j - 1] *= rp;
        if (tid < kb) Xs[j - 1][tid] *= rp;
      }
      if (tid == 0 && j < kb) {
        const double d = Ps[j * LDP + j];
        if (!(d > 0.0) || !isfinite(d)) *s_bad = 1;
        const double dd = fmax(d, 1e-300);
        double r = (double)rsqrtf((float)dd);
        r = r * fma(-0.5 * dd * r, r, 1.5);
        r = r * fma(-0.5 * dd * r, r, 1.5);
        Ps[j * LDP + j] = dd * r;
        s_rinv[1] = r;
      }
      __syncthreads();
      if (j == kb) break;
      const double r = s_rinv[1], r2 = r * r;
      if (tid == 0) s_rinv[0] = r;   // read by phase A of the next column (after the barrier below)
      const int w = kb - j - 1;
      if (w > 0) {
        // one thread per panel row: a single scaling, then plain DFMAs along the row
        for (int i = j + 1 + tid; i < mt; i += kThreads) {
          const double a = r2 * Ps[i * LDP + j];
          const int kend = i < kb ? i + 1 : kb;
          for (int k = j + 1; k < kend; ++k) Ps[i * LDP + k] = fma(-a, Ps[k * LDP + j], Ps[i * LDP + k]);
        }
        // X rows below j: X[i][c] -= L[i][j] X[j][c] for c <= j (both still unscaled by r_j)
        for (int e = tid; e < w * (j + 1); e += kThreads) {
          const int i = j + 1 + e / (j + 1), c = e % (j + 1);
          Xs[i][c] -= r2 * Ps[i * LDP + j] * Xs[j][c];
        }
      }
      __syncthreads();
    }
    if (*s_bad) return false;
    // write back L (panel) and X^T (upper triangle of the diagonal block)
    for (int e = tid; e < mt * kb; e += kThreads) {
      const int i = e / kb, t = e - i * kb;
      if (i >= kb || t <= i) S[(size_t)(k0 + i) * n + k0 + t] = Ps[i * LDP + t];
      else S[(size_t)(k0 + i) * n + k0 + t] = Xs[t][i];
    }
    // trailing update of the lower triangle, 32 x 32 tiles, 4 x 2 outputs per thread
    const int r0 = kb, m = mt - kb;   // panel-local first trailing row, trailing size
    if (m > 0) {
      const int T = (m + 31) / 32;
      const int tx = tid & 15, ty = tid >> 4;   // 16 x 8 threads, rows ty + 8a (a < 4), cols tx + 16b (b < 2)
      for (int tile = 0; tile < T * (T + 1) / 2; ++tile) {
        int ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
        const int tj = tile - ti * (ti + 1) / 2;
        const int bi = r0 + 32 * ti, bj = r0 + 32 * tj;
        double acc[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = 0.0;
        int ii[4], jj[2];
        bool vi[4], vj[2];
#pragma unroll
        for (int a = 0; a < 4; ++a) { ii[a] = bi + ty + 8 * a; vi[a] = ii[a] < mt; }
#pragma unroll
        for (int b = 0; b < 2; ++b) { jj[b] = bj + tx + 16 * b; vj[b] = jj[b] < mt; }
#pragma unroll 4
        for (int t = 0; t < kb; ++t) {
          double av[4], bv[2];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = vi[a] ? Ps[ii[a] * LDP + t] : 0.0;
#pragma unroll
          for (int b = 0; b < 2; ++b) bv[b] = vj[b] ? Ps[jj[b] * LDP + t] : 0.0;
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b)
            if (vi[a] && vj[b] && jj[b] <= ii[a]) S[(size_t)(k0 + ii[a]) * n + k0 + jj[b]] -= acc[a][b];
      }
    }
    __syncthreads();
  }
  return true;
}

// ------------------------------------------------------------------------------------ A = L^-T L^-1 H
// One right-hand-side column per thread (columns in batches of kThreads), blocked by 32 rows; L tiles are
// staged in shared memory in T, the diagonal blocks are applied through X_r.
template <typename T>
__device__ void solve_A(const double* __restrict__ S, const double* __restrict__ H, int n, T* __restrict__ X,
                        T (*Lp)[NB + 1], T (*Xf)[NB + 1]) {
  const int tid = threadIdx.x;
  const int nblk = (n + NB - 1) / NB;
  for (int cb = 0; cb < n; cb += kThreads) {
    const int c = cb + tid;
    const bool act = c < n;
    // forward: Y = L^-1 H
    for (int rbk = 0; rbk < nblk; ++rbk) {
      const int r0 = rbk * NB, rb = min(NB, n - r0);
      T acc[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) acc[i] = (act && i < rb) ? (T)H[(size_t)(r0 + i) * n + c] : T(0);
      for (int q0 = 0; q0 < r0; q0 += NB) {
        for (int e = tid; e < NB * NB; e += kThreads) {
          const int i = e >> 5, t = e & 31;
          Lp[i][t] = i < rb ? (T)S[(size_t)(r0 + i) * n + q0 + t] : T(0);
        }
        __syncthreads();
        if (act) {
          T y[NB];
#pragma unroll
          for (int t = 0; t < NB; ++t) y[t] = X[(size_t)(q0 + t) * n + c];
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
        const int a = e >> 5, t = e & 31;
        Xf[a][t] = (a < rb && t < rb) ? (T)xinv(S, n, r0, a, t) : T(0);
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int a = NB - 1; a >= 0; --a) {   // y = X_r acc (lower triangular: row a uses acc[0..a])
          T s = T(0);
#pragma unroll
          for (int t = 0; t <= a; ++t) s += Xf[a][t] * acc[t];
          if (a < rb) X[(size_t)(r0 + a) * n + c] = s;
          acc[a] = s;
        }
      }
      __syncthreads();
    }
    // backward: A = L^-T Y
    for (int rbk = nblk - 1; rbk >= 0; --rbk) {
      const int r0 = rbk * NB, rb = min(NB, n - r0);
      T acc[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) acc[i] = (act && i < rb) ? X[(size_t)(r0 + i) * n + c] : T(0);
      for (int q0 = r0 + NB; q0 < n; q0 += NB) {
        const int qb = min(NB, n - q0);
        for (int e = tid; e < NB * NB; e += kThreads) {
          const int t = e >> 5, i = e & 31;  // Lp[i][t] = L[q0+t][r0+i]
          Lp[i][t] = (t < qb && i < rb) ? (T)S[(size_t)(q0 + t) * n + r0 + i] : T(0);
        }
        __syncthreads();
        if (act) {
          T x[NB];
#pragma unroll
          for (int t = 0; t < NB; ++t) x[t] = t < qb ? X[(size_t)(q0 + t) * n + c] : T(0);
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
        const int a = e >> 5, t = e & 31;
        Xf[a][t] = (a < rb && t < rb) ? (T)xinv(S, n, r0, a, t) : T(0);
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int a = 0; a < NB; ++a) {   // x = X_r^T acc (upper triangular: row a uses acc[a..])
          T s = T(0);
#pragma unroll
          for (int t = a; t < NB; ++t) s += Xf[t][a] * acc[t];
          if (a < rb) X[(size_t)(r0 + a) * n + c] = s;
          acc[a] = s;
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------------------ Q = L^-T L^-1 E_c (FP64)
// Threads take (row, column) pairs so that every FP64 instruction is issued by full warps.
__device__ void solve_Q(const double* __restrict__ S, int n, int c0, int b, double* __restrict__ Q,
                        double (*Acc)[kMaxB + 1], double (*Xd)[NB + 1]) {
  const int tid = threadIdx.x;
  const int nblk = (n + NB - 1) / NB;
  for (int rbk = 0; rbk < nblk; ++rbk) {   // forward: W = L^-1 E
    const int r0 = rbk * NB, rb = min(NB, n - r0);
    for (int e = tid; e < rb * b; e += kThreads) {
      const int i = e / b, c = e - i * b;
      double s = (r0 + i == c0 + c) ? 1.0 : 0.0;
      const double* Li = S + (size_t)(r0 + i) * n;
      for (int q = 0; q < r0; ++q) s = fma(-Li[q], Q[(size_t)q * b + c], s);
      Acc[i][c] = s;
    }
    for (int e = tid; e < NB * NB; e += kThreads) {
      const int a = e >> 5, t = e & 31;
      Xd[a][t] = (a < rb && t < rb) ? xinv(S, n, r0, a, t) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < rb * b; e += kThreads) {
      const int a = e / b, c = e - a * b;
      double s = 0.0;
      for (int t = 0; t <= a; ++t) s = fma(Xd[a][t], Acc[t][c], s);
      Q[(size_t)(r0 + a) * b + c] = s;
    }
    __syncthreads();
  }
  for (int rbk = nblk - 1; rbk >= 0; --rbk) {   // backward: Q = L^-T W
    const int r0 = rbk * NB, rb = min(NB, n - r0);
    for (int e = tid; e < rb * b; e += kThreads) {
      const int i = e / b, c = e - i * b;
      double s = Q[(size_t)(r0 + i) * b + c];
      for (int q = r0 + rb; q < n; ++q) s = fma(-S[(size_t)q * n + r0 + i], Q[(size_t)q * b + c], s);
      Acc[i][c] = s;
    }
    for (int e = tid; e < NB * NB; e += kThreads) {
      const int a = e >> 5, t = e & 31;
      Xd[a][t] = (a < rb && t < rb) ? xinv(S, n, r0, a, t) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < rb * b; e += kThreads) {
      const int a = e / b, c = e - a * b;
      double s = 0.0;
      for (int t = a; t < rb; ++t) s = fma(Xd[t][a], Acc[t][c], s);
      Q[(size_t)(r0 + a) * b + c] = s;
    }
    __syncthreads();
  }
}

template <typename TA>
__global__ void __launch_bounds__(kThreads, 2) k_prepare(PrepArgs g, TA* __restrict__ Acache) {
  extern __shared__ double Ps[];   // factorisation panel: n x (NB+1) doubles
  __shared__ double Xs[NB][NB + 1];
  __shared__ __align__(16) unsigned char raw[sizeof(double) * NB * (kMaxB + 1)];
  __shared__ double s_rinv[2];
  __shared__ int s_bad;
  __shared__ float rlo[kThreads], rhi[kThreads];
  const int J = g.j0 + blockIdx.x;
  const int n = g.sub_n[J];
  const int bJ = g.nbf[J];
  const int c0 = g.sub_c0[J];
  double* S = g.ws + (g.a_off[J] - g.a_base);
  const double* H = S + g.chunk_n2;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const bool ok = cholesky(S, n, Ps, Xs, s_rinv, &s_bad);
  if (threadIdx.x == 0) g.prep_status[J] = ok ? kSubOk : kSubNotSpd;
  if (!ok) return;   // uniform: every thread read the flag after the same barrier
  // A_J in TA (shared memory reused: two T tiles)
  TA* A = Acache + g.a_off[J];
  TA (*Lp)[NB + 1] = reinterpret_cast<TA (*)[NB + 1]>(Ps);
  TA (*Xf)[NB + 1] = reinterpret_cast<TA (*)[NB + 1]>(Ps + NB * (NB + 1));
  solve_A<TA>(S, H, n, A, Lp, Xf);
  __syncthreads();
  // Q_J in FP64
  solve_Q(S, n, c0, bJ, g.Q + g.c_off[J], reinterpret_cast<double (*)[kMaxB + 1]>(raw), Xs);
  __syncthreads();
  // Gershgorin interval of A_J (in the arithmetic of A, widened by its rounding)
  float lo = INFINITY, hi = -INFINITY;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    float r = 0.0f;
    const TA* Ai = A + (size_t)i * n;
    for (int j = 0; j < n; ++j)
      if (j != i) r += fabsf((float)Ai[j]);
    lo = fminf(lo, (float)Ai[i] - r);
    hi = fmaxf(hi, (float)Ai[i] + r);
  }
  rlo[threadIdx.x] = lo;
  rhi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      rlo[threadIdx.x] = fminf(rlo[threadIdx.x], rlo[threadIdx.x + s]);
      rhi[threadIdx.x] = fmaxf(rhi[threadIdx.x], rhi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double w = 1e-5 * fmax(fabs((double)rlo[0]), fabs((double)rhi[0]));
    g.lam[2 * J] = (double)rlo[0] - w;
    g.lam[2 * J + 1] = (double)rhi[0] + w;
  }
}

}  // namespace

size_t prepare_smem_bytes(int max_n) { return sizeof(double) * (size_t)max_n * (NB + 1); }

nolsm_status launch_prepare(const PrepArgs& g, int count, int max_n, bool fp64_A, void* Acache, cudaStream_t st) {
  const size_t smem = prepare_smem_bytes(std::max(max_n, 2 * NB));
  if (smem > 200 * 1024) {
    set_error("submatrix dimension %d exceeds the factorisation panel's shared memory", max_n);
    return NOLSM_ERR_UNSUPPORTED;
  }
  if (fp64_A) {
    NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_prepare<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_prepare<double><<<count, kThreads, smem, st>>>(g, static_cast<double*>(Acache));
  } else {
    NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_prepare<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_prepare<float><<<count, kThreads, smem, st>>>(g, static_cast<float*>(Acache));
  }
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}

}  // namespace nolsm
