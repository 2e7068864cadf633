// a2-a3: the overlap factorisation T_J(S) = L L^T and the solves that give
//   A_J = T_J(S)^-1 T_J(H0) = L^-T (L^-1 T_J(H0))            (Eq. purification_submatrix)
//   Q_J = T_J(S)^-1 [:, centre columns] = L^-T (L^-1 E_c)     (to FP64 accuracy always)
// and the Gershgorin interval of A_J. One CTA (128 threads) per submatrix.
//
// Two preparations share the blocked algorithms below (templated on the factor's type):
//  - k_prepare (FP64 path, and fallback): L in FP64, factored in place; Q by FP64 solves.
//    FP64 runs at 2 lanes per clock per SM on this GPU (one full-warp FP64 instruction per 64 cycles per
//    scheduler), so every FP64 instruction here is issued by full warps spread over all schedulers and no
//    FP64 work is a dependent chain.
//  - k_prepare_mixed (low-precision paths): L in FP32 (the FP32 pipe is ~60x the FP64 one), A by FP32
//    solves as before, and Q by mixed-precision iterative refinement: q <- q + L^-T L^-1 (E_c - T_J(S) q)
//    with the residual in double-FP32 arithmetic (T_J(S) and q split into two FP32 words each, about 48
//    bits) and the correction solves in FP32, until the correction is below 1e-6 of q (the error then
//    contracts by the same factor per step, down to the residual's accuracy, about 1e-12 relative). A
//    submatrix whose FP32 factor fails or whose refinement does not contract is flagged and prepared
//    again by k_prepare (FP64 factor).
// The Cholesky factors a 32-column panel held in shared memory one column at a time in parallel over its
// rows, and builds the inverse X_r of the panel's diagonal block in the same sweep (column-oriented
// forward substitution on the identity). The triangular solves then apply X_r as a product instead of
// substituting row by row. X_r is kept, transposed, in the unused upper triangle of its diagonal block
// (its diagonal is 1/L_ii).
#include <algorithm>
#include <cmath>

#include "nolsm_internal.cuh"
#include "prep.cuh"

namespace nolsm {

namespace {

constexpr int NB = 32;
constexpr int kThreads = 128;   // several CTAs (submatrices) per SM overlap each other's serial phases
constexpr int kMaxB = 64;
constexpr int kRefineMax = 4;   // refinement steps of Q before a submatrix falls back to the FP64 factor
constexpr double kRefineTol = 1e-6;
constexpr double kNsOneStep = 1e-5;   // k_ns_qrefine: a first correction below this ends the refinement

// Row stride of panels and tiles in shared memory: FP64 rows padded by one element (bank spread),
// FP32 rows by four so that every row starts on a 16-byte boundary (vector loads).
template <typename T> struct Ld { static constexpr int v = NB + 1; };
template <> struct Ld<float> { static constexpr int v = NB + 4; };

// X_r[a][t] for a, t < kb: lower-triangular inverse of the diagonal block starting at r0.
template <typename T>
__device__ __forceinline__ T xinv(const T* S, int n, int r0, int a, int t) {
  if (t > a) return T(0);
  if (t == a) return T(1) / S[(size_t)(r0 + a) * n + r0 + a];
  return S[(size_t)(r0 + t) * n + r0 + a];  // stored transposed in the upper triangle
}

// Asynchronous 4-byte copy from global to shared memory; cp_async_wait_all waits for this thread's copies.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// The same for the FP32 factor, which stores X_r in the lower triangle of its diagonal blocks.
__device__ __forceinline__ float xinv32(const float* L, int n, int r0, int a, int t) {
  return t > a ? 0.0f : L[(size_t)(r0 + a) * n + r0 + t];
}

// ------------------------------------------------------------------------------------ Cholesky
// In place: the lower triangle of S receives L; the strict upper triangle of every diagonal block
// receives X_r^T. Returns false (uniformly) if a pivot is not positive or not finite.
template <typename T>
__device__ bool cholesky(T* __restrict__ S, int n, T* __restrict__ Ps, T (*Xs)[NB + 1], T* s_rinv /* [2] */,
                         int* s_bad) {
  const int tid = threadIdx.x;
  constexpr int LDP = Ld<T>::v;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0), mt = n - k0;
    if constexpr (sizeof(T) == 8) {
      for (int e = tid; e < mt * kb; e += kThreads) {
        const int i = e / kb, t = e - i * kb;
        Ps[i * LDP + t] = S[(size_t)(k0 + i) * n + k0 + t];
      }
    } else {
      // full 32-column rows, zero beyond kb (the trailing update reads whole 4-column groups)
      for (int e = tid; e < mt * NB; e += kThreads) {
        const int i = e / NB, t = e - i * NB;
        Ps[i * LDP + t] = t < kb ? S[(size_t)(k0 + i) * n + k0 + t] : T(0);
      }
    }
    for (int e = tid; e < NB * NB; e += kThreads) Xs[e >> 5][e & 31] = ((e >> 5) == (e & 31)) ? T(1) : T(0);
    __syncthreads();
    // Column j: phase A scales column j-1 and row j-1 of X by r_{j-1} while thread 0 forms the pivot of
    // column j (FP32 rsqrt seed, Newton steps in the factor's precision); phase B updates the panel and X
    // with the unscaled column j times r_j^2.
    for (int j = 0; j <= kb; ++j) {
      if (j > 0) {
        const T rp = *s_rinv;
        for (int i = j + tid; i < mt; i += kThreads) Ps[i * LDP + j - 1] *= rp;
        if (tid < kb) Xs[j - 1][tid] *= rp;
      }
      if (tid == 0 && j < kb) {
        const T d = Ps[j * LDP + j];
        if (!(d > T(0)) || !isfinite(d)) *s_bad = 1;
        if constexpr (sizeof(T) == 8) {
          const double dd = fmax(d, 1e-300);
          double r = (double)rsqrtf((float)dd);
          r = r * fma(-0.5 * dd * r, r, 1.5);
          r = r * fma(-0.5 * dd * r, r, 1.5);
          Ps[j * LDP + j] = dd * r;
          s_rinv[1] = r;
        } else {
          const float dd = fmaxf(d, 1e-30f);
          float r = rsqrtf(dd);
          r = r * fmaf(-0.5f * dd * r, r, 1.5f);
          Ps[j * LDP + j] = dd * r;
          s_rinv[1] = r;
        }
      }
      __syncthreads();
      if (j == kb) break;
      const T r = s_rinv[1], r2 = r * r;
      if (tid == 0) s_rinv[0] = r;   // read by phase A of the next column (after the barrier below)
      const int w = kb - j - 1;
      if (w > 0) {
        // one thread per panel row: a single scaling, then plain FMAs along the row
        for (int i = j + 1 + tid; i < mt; i += kThreads) {
          const T a = r2 * Ps[i * LDP + j];
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
    // write back L (panel) and X^T (upper triangle of the diagonal block); the FP32 factor keeps X_r
    // itself (diagonal 1/L_ii) in the lower triangle of the diagonal block, which no solve reads as L
    for (int e = tid; e < mt * kb; e += kThreads) {
      const int i = e / kb, t = e - i * kb;
      T v;
      if (i >= kb) v = Ps[i * LDP + t];
      else if (t > i) v = Xs[t][i];
      else v = sizeof(T) == 4 ? Xs[i][t] : Ps[i * LDP + t];
      S[(size_t)(k0 + i) * n + k0 + t] = v;
    }
    // trailing update of the lower triangle, 32 x 32 tiles, 4 x 2 outputs per thread
    const int r0 = kb, m = mt - kb;   // panel-local first trailing row, trailing size
    if (m > 0) {
      const int TT = (m + 31) / 32;
      const int tx = tid & 15, ty = tid >> 4;   // 16 x 8 threads, rows ty + 8a (a < 4), cols tx + 16b (b < 2)
      for (int tile = 0; tile < TT * (TT + 1) / 2; ++tile) {
        int ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
        const int tj = tile - ti * (ti + 1) / 2;
        const int bi = r0 + 32 * ti, bj = r0 + 32 * tj;
        T acc[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = T(0);
        int ii[4], jj[2];
        bool vi[4], vj[2];
#pragma unroll
        for (int a = 0; a < 4; ++a) { ii[a] = bi + ty + 8 * a; vi[a] = ii[a] < mt; }
#pragma unroll
        for (int b = 0; b < 2; ++b) { jj[b] = bj + tx + 16 * b; vj[b] = jj[b] < mt; }
        if constexpr (sizeof(T) == 8) {
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
        } else {
          const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int t = 0; t < kb; t += 4) {
            float4 av[4], bv[2];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = vi[a] ? *reinterpret_cast<const float4*>(&Ps[ii[a] * LDP + t]) : z4;
#pragma unroll
            for (int b = 0; b < 2; ++b) bv[b] = vj[b] ? *reinterpret_cast<const float4*>(&Ps[jj[b] * LDP + t]) : z4;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 2; ++b) {
                float s = acc[a][b];
                s = fmaf(av[a].x, bv[b].x, s);
                s = fmaf(av[a].y, bv[b].y, s);
                s = fmaf(av[a].z, bv[b].z, s);
                s = fmaf(av[a].w, bv[b].w, s);
                acc[a][b] = s;
              }
          }
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

// FP32 form for the mixed preparation with four block-wide barriers per 32-column panel instead of two
// per column: warp 0 factors the panel's 32 x 32 diagonal block in registers (lane i holds row i, the
// pivot column travels by shuffles) and inverts it (X_r = L_11^-1, row by row, each finished row
// broadcast); then every thread forms rows of L_21 = A_21 X_r^T; the trailing update is the tiled one above.
// Xs is [NB][NB + 4] (16-byte rows). Same results up to rounding order as cholesky<float>.
// S64 is the FP64 T_J(S): the first panel and the first trailing update read it (rounded to FP32) in
// place of S, so S needs no separate FP32 copy of T_J(S) before the factorisation.
__device__ bool cholesky32(float* __restrict__ S, const double* __restrict__ S64, int n, float* __restrict__ Ps,
                           float (*Xs)[NB + 4], int* s_bad) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int LDP = Ld<float>::v;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0), mt = n - k0;
    // panel rows by warp, lanes along the row, zero beyond kb; the copies are asynchronous, all in flight
    if (k0 == 0) {
#pragma unroll 4
      for (int i = warp; i < mt; i += kThreads / 32)
        Ps[i * LDP + lane] = lane < kb ? (float)S64[(size_t)i * n + lane] : 0.0f;
    } else {
      for (int i = warp; i < mt; i += kThreads / 32) {
        float* dst = Ps + i * LDP + lane;
        if (lane < kb) cp_async4(dst, S + (size_t)(k0 + i) * n + k0 + lane);
        else *dst = 0.0f;
      }
      cp_async_wait_all();
    }
    __syncthreads();
    if (warp == 0) {
      // factor the diagonal block in the panel itself: lane i owns row i (rows beyond kb idle)
      const bool live = lane < kb;
      bool bad = false;
      float myr = 1.0f;   // 1 / L_ii of this lane's row
      for (int j = 0; j < kb; ++j) {
        const float piv = Ps[j * LDP + j];
        bad = bad || !(piv > 0.0f) || !isfinite(piv);
        const float d = fmaxf(piv, 1e-30f);
        float r = rsqrtf(d);
        r = r * fmaf(-0.5f * d * r, r, 1.5f);
        __syncwarp();
        if (lane == j) {
          Ps[j * LDP + j] = d * r;
          myr = r;
        }
        if (live && lane > j) Ps[lane * LDP + j] *= r;
        __syncwarp();
        if (live && lane > j) {
          const float lij = Ps[lane * LDP + j];
          for (int k = j + 1; k <= lane; ++k) Ps[lane * LDP + k] = fmaf(-lij, Ps[k * LDP + j], Ps[lane * LDP + k]);
        }
        __syncwarp();
      }
      // X_r = L_11^-1: rows in order; lane i accumulates -sum_{k<i} L_ik X[k][j], then scales by 1/L_ii
      float x[NB];
#pragma unroll
      for (int k = 0; k < NB; ++k) x[k] = 0.0f;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (lane == i) {
#pragma unroll
          for (int j = 0; j <= i; ++j) x[j] = ((j == i) ? 1.0f + x[j] : x[j]) * myr;
        }
        const float lli = (live && lane > i) ? Ps[lane * LDP + i] : 0.0f;   // L[lane][i]
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          const float xij = __shfl_sync(0xffffffffu, x[j], i);
          if (lane > i) x[j] = fmaf(-lli, xij, x[j]);
        }
      }
      // Xs holds X_r transposed: Xs[k][i] = X_r[i][k] (zero above the diagonal of X_r)
#pragma unroll
      for (int k = 0; k < NB; ++k) Xs[k][lane] = (live && k <= lane) ? x[k] : 0.0f;
      if (__any_sync(0xffffffffu, bad && lane < kb)) {
        if (lane == 0) *s_bad = 1;
      }
    }
    __syncthreads();
    if (*s_bad) return false;
    // L_21 = A_21 X_r^T: row i of the panel below the diagonal block, one thread per row, eight outputs
    // at a time: out[j] = sum_{t <= j} A_21[i][t] X_r[j][t], X_r^T rows read as 16-byte vectors
    for (int i = kb + tid; i < mt; i += kThreads) {
      asm volatile("" ::: "memory");   // keeps the X_r loads in the loop (hoisting them all would spill)
      float* pi = Ps + i * LDP;
      float out[4][8];
#pragma unroll
      for (int jb = 0; jb < 4; ++jb) {
#pragma unroll
        for (int q = 0; q < 8; ++q) out[jb][q] = 0.0f;
#pragma unroll
        for (int t = 0; t < 8 * jb + 8; ++t) {
          const float rt = pi[t];
          const float4 x0 = *reinterpret_cast<const float4*>(&Xs[t][8 * jb]);
          const float4 x1 = *reinterpret_cast<const float4*>(&Xs[t][8 * jb + 4]);
          out[jb][0] = fmaf(rt, x0.x, out[jb][0]);
          out[jb][1] = fmaf(rt, x0.y, out[jb][1]);
          out[jb][2] = fmaf(rt, x0.z, out[jb][2]);
          out[jb][3] = fmaf(rt, x0.w, out[jb][3]);
          out[jb][4] = fmaf(rt, x1.x, out[jb][4]);
          out[jb][5] = fmaf(rt, x1.y, out[jb][5]);
          out[jb][6] = fmaf(rt, x1.z, out[jb][6]);
          out[jb][7] = fmaf(rt, x1.w, out[jb][7]);
        }
      }
#pragma unroll
      for (int jb = 0; jb < 4; ++jb) {
        *reinterpret_cast<float4*>(pi + 8 * jb) = make_float4(out[jb][0], out[jb][1], out[jb][2], out[jb][3]);
        *reinterpret_cast<float4*>(pi + 8 * jb + 4) = make_float4(out[jb][4], out[jb][5], out[jb][6], out[jb][7]);
      }
    }
    __syncthreads();
    // write back L (panel), X_r^T in the upper and X_r in the lower triangle of the diagonal block
    if (lane < kb) {
#pragma unroll 4
      for (int i = warp; i < mt; i += kThreads / 32) {
        float v;
        if (i >= kb) v = Ps[i * LDP + lane];
        else if (lane > i) v = Xs[i][lane];   // X_r^T[i][lane] = X_r[lane][i]
        else v = Xs[lane][i];                 // X_r[i][lane]
        S[(size_t)(k0 + i) * n + k0 + lane] = v;
      }
    }
    // trailing update of the lower triangle, 32 x 32 tiles, 4 x 2 outputs per thread
    const int r0 = kb, m = mt - kb;
    if (m > 0) {
      const int TT = (m + 31) / 32;
      const int tx = tid & 15, ty = tid >> 4;
      for (int tile = 0; tile < TT * (TT + 1) / 2; ++tile) {
        int ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
        const int tj = tile - ti * (ti + 1) / 2;
        const int bi = r0 + 32 * ti, bj = r0 + 32 * tj;
        float acc[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = 0.0f;
        int ii[4], jj[2];
        bool vi[4], vj[2];
#pragma unroll
        for (int a = 0; a < 4; ++a) { ii[a] = bi + ty + 8 * a; vi[a] = ii[a] < mt; }
#pragma unroll
        for (int b = 0; b < 2; ++b) { jj[b] = bj + tx + 16 * b; vj[b] = jj[b] < mt; }
        // the elements to update, loaded before the products so that their latency overlaps them
        float sv[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b)
            sv[a][b] = !(vi[a] && vj[b] && jj[b] <= ii[a]) ? 0.0f
                       : k0 == 0 ? (float)S64[(size_t)ii[a] * n + jj[b]]
                                 : S[(size_t)(k0 + ii[a]) * n + k0 + jj[b]];
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int t = 0; t < kb; t += 4) {
          float4 av[4], bv[2];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = vi[a] ? *reinterpret_cast<const float4*>(&Ps[ii[a] * LDP + t]) : z4;
#pragma unroll
          for (int b = 0; b < 2; ++b) bv[b] = vj[b] ? *reinterpret_cast<const float4*>(&Ps[jj[b] * LDP + t]) : z4;
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
              float s2 = acc[a][b];
              s2 = fmaf(av[a].x, bv[b].x, s2);
              s2 = fmaf(av[a].y, bv[b].y, s2);
              s2 = fmaf(av[a].z, bv[b].z, s2);
              s2 = fmaf(av[a].w, bv[b].w, s2);
              acc[a][b] = s2;
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b)
            if (vi[a] && vj[b] && jj[b] <= ii[a]) S[(size_t)(k0 + ii[a]) * n + k0 + jj[b]] = sv[a][b] - acc[a][b];
      }
    }
    __syncthreads();
  }
  return true;
}

// ------------------------------------------------------------------------------------ A = L^-T L^-1 H
// s - sum_t row[t] y[t] over one 32-wide block (row in shared memory; FP32 rows are 16-byte aligned)
template <typename T>
__device__ __forceinline__ T row_dot_sub(const T* row, const T (&y)[NB], T s) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int t = 0; t < NB; t += 4) {
      const float4 l = *reinterpret_cast<const float4*>(row + t);
      s -= l.x * y[t];
      s -= l.y * y[t + 1];
      s -= l.z * y[t + 2];
      s -= l.w * y[t + 3];
    }
  } else {
#pragma unroll
    for (int t = 0; t < NB; ++t) s -= row[t] * y[t];
  }
  return s;
}

// One right-hand-side column per thread (columns in batches of kThreads), blocked by 32 rows; L tiles are
// staged in shared memory in T, the diagonal blocks are applied through X_r. LT is the factor's type.
template <typename T, typename LT>
__device__ void solve_A(const LT* __restrict__ S, const double* __restrict__ H, int n, T* __restrict__ X,
                        T* __restrict__ Lp, T* __restrict__ Xf) {
  constexpr int LDA = Ld<T>::v;
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
          Lp[i * LDA + t] = i < rb ? (T)S[(size_t)(r0 + i) * n + q0 + t] : T(0);
        }
        __syncthreads();
        if (act) {
          T y[NB];
#pragma unroll
          for (int t = 0; t < NB; ++t) y[t] = X[(size_t)(q0 + t) * n + c];
#pragma unroll
          for (int i = 0; i < NB; ++i) acc[i] = row_dot_sub(Lp + i * LDA, y, acc[i]);
        }
        __syncthreads();
      }
      // X_r for y = X_r acc (lower triangular)
      for (int e = tid; e < NB * NB; e += kThreads) {
        const int a = e >> 5, t = e & 31;
        Xf[a * LDA + t] = (a < rb && t < rb) ? (T)xinv(S, n, r0, a, t) : T(0);
      }
      __syncthreads();
      if (act) {
        if constexpr (sizeof(T) == 4) {
          T o[NB];
#pragma unroll
          for (int a = 0; a < NB; ++a) {   // row a of X_r is zero beyond a: whole 4-groups up to a
            float s = 0.0f;
#pragma unroll
            for (int t = 0; t <= (a | 3); t += 4) {
              const float4 x4 = *reinterpret_cast<const float4*>(Xf + a * LDA + t);
              s = fmaf(x4.x, acc[t], s);
              s = fmaf(x4.y, acc[t + 1], s);
              s = fmaf(x4.z, acc[t + 2], s);
              s = fmaf(x4.w, acc[t + 3], s);
            }
            o[a] = s;
          }
#pragma unroll
          for (int a = 0; a < NB; ++a)
            if (a < rb) X[(size_t)(r0 + a) * n + c] = o[a];
        } else {
#pragma unroll
          for (int a = NB - 1; a >= 0; --a) {   // y = X_r acc (lower triangular: row a uses acc[0..a])
            T s = T(0);
#pragma unroll
            for (int t = 0; t <= a; ++t) s += Xf[a * LDA + t] * acc[t];
            if (a < rb) X[(size_t)(r0 + a) * n + c] = s;
            acc[a] = s;
          }
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
          Lp[i * LDA + t] = (t < qb && i < rb) ? (T)S[(size_t)(q0 + t) * n + r0 + i] : T(0);
        }
        __syncthreads();
        if (act) {
          T x[NB];
#pragma unroll
          for (int t = 0; t < NB; ++t) x[t] = t < qb ? X[(size_t)(q0 + t) * n + c] : T(0);
#pragma unroll
          for (int i = 0; i < NB; ++i) acc[i] = row_dot_sub(Lp + i * LDA, x, acc[i]);
        }
        __syncthreads();
      }
      if constexpr (sizeof(T) == 4) {
        // X_r^T staged by rows: Xf[a][t] = X_r[t][a], zero for t < a
        for (int e = tid; e < NB * NB; e += kThreads) {
          const int a = e >> 5, t = e & 31;
          Xf[a * LDA + t] = (a < rb && t < rb) ? (T)xinv(S, n, r0, t, a) : T(0);
        }
      } else {
        for (int e = tid; e < NB * NB; e += kThreads) {
          const int a = e >> 5, t = e & 31;
          Xf[a * LDA + t] = (a < rb && t < rb) ? (T)xinv(S, n, r0, a, t) : T(0);
        }
      }
      __syncthreads();
      if (act) {
        if constexpr (sizeof(T) == 4) {
          T o[NB];
#pragma unroll
          for (int a = 0; a < NB; ++a) {   // x = X_r^T acc (row a of X_r^T is zero before a)
            float s = 0.0f;
#pragma unroll
            for (int t = a & ~3; t < NB; t += 4) {
              const float4 x4 = *reinterpret_cast<const float4*>(Xf + a * LDA + t);
              s = fmaf(x4.x, acc[t], s);
              s = fmaf(x4.y, acc[t + 1], s);
              s = fmaf(x4.z, acc[t + 2], s);
              s = fmaf(x4.w, acc[t + 3], s);
            }
            o[a] = s;
          }
#pragma unroll
          for (int a = 0; a < NB; ++a)
            if (a < rb) X[(size_t)(r0 + a) * n + c] = o[a];
        } else {
#pragma unroll
          for (int a = 0; a < NB; ++a) {   // x = X_r^T acc (upper triangular: row a uses acc[a..])
            T s = T(0);
#pragma unroll
            for (int t = a; t < NB; ++t) s += Xf[t * LDA + a] * acc[t];
            if (a < rb) X[(size_t)(r0 + a) * n + c] = s;
            acc[a] = s;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Register-tiled form of the same solves for the mixed preparation. Right-hand sides: columns c < n of
// T_J(H0) (result into X, n x n) and, when bq > 0, the centre columns of the identity (result into W,
// n x bq). Columns go in batches of 64; thread (tr, tc) (tr < 8, tc < 16) owns rows 4tr..4tr+3 of the
// current 32-row block and columns 4tc..4tc+3 of the batch, so every step of the inner loop is two
// 16-byte shared loads and 16 FMAs. Chunks of 32 columns of L and 32 rows of the solution are staged
// through registers, the next chunk's global loads in flight while the current one is used.
// Shared memory: sm holds kRtSmem floats.
constexpr int kRtLd = NB + 4;                  // LT, XT rows (16-byte aligned)
constexpr int kRtCb = 64;                      // columns per batch
constexpr int kRtYd = kRtCb + 4;               // YC / AC rows
constexpr int kRtSmem = 2 * NB * kRtLd + NB * kRtYd;

__device__ __forceinline__ float rt_rhs(const double* __restrict__ H, int n, int c0, int row, int col) {
  return col < n ? (float)H[(size_t)row * n + col] : (row == c0 + col - n ? 1.0f : 0.0f);
}

// kMode 0: X = L^-T L^-1 T_J(H0) (and W = L^-T L^-1 E_c); kMode 1: forward only, X = L^-1 T_J(H0) (and
// W = L^-1 E_c); kMode 2: forward only with the transposed right-hand side Yt^T, X = L^-1 Yt^T (Yt n x n).
template <int kMode>
__device__ void solve_A_rt(const float* __restrict__ L, const double* __restrict__ H, int n, int c0, int bq,
                           float* __restrict__ X, float* __restrict__ W, float* __restrict__ sm,
                           const float* __restrict__ Yt = nullptr) {
  const int tid = threadIdx.x;
  // a warp covers 4 values of tr and 8 of tc, so each step of the inner loop reads 64 B of LT and 128 B
  // of YC per warp (one shared-memory wavefront each)
  const int lane = tid & 31, wrp = tid >> 5;
  const int tr = 4 * (wrp & 1) + (lane >> 3), tc = 8 * (wrp >> 1) + (lane & 7);
  const int nblk = (n + NB - 1) / NB;
  const int ncol = n + bq;
  float* LT = sm;                       // [32][kRtLd]
  float* XT = sm + NB * kRtLd;          // [32][kRtLd]
  float* YC = sm + 2 * NB * kRtLd;      // [32][kRtYd], also the accumulator exchange
  // element (row, col) of the result / right-hand-side array of global column col
  auto addr = [&](int row, int col) -> float* {
    return col < n ? X + (size_t)row * n + col : W + (size_t)row * bq + (col - n);
  };
  for (int cb = 0; cb < ncol; cb += kRtCb) {
    for (int pass = 0; pass < (kMode == 0 ? 2 : 1); ++pass) {   // 0: forward Y = L^-1 B; 1: backward L^-T Y
      for (int s = 0; s < nblk; ++s) {
        const int rbk = pass == 0 ? s : nblk - 1 - s;
        const int r0 = rbk * NB, rb = min(NB, n - r0);
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int row = r0 + 4 * tr + a;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int col = cb + 4 * tc + c;
            float v = 0.0f;
            if (row < n && col < ncol) {
              if (pass == 1) v = *addr(row, col);
              else if (kMode == 2) v = Yt[(size_t)col * n + row];
              else v = rt_rhs(H, n, c0, row, col);
            }
            acc[a][c] = v;
          }
        }
        // chunks of the coupling: forward q0 in [0, r0), backward q0 in [r0 + rb, n)
        const int q_begin = pass == 0 ? 0 : r0 + rb;
        const int q_end = pass == 0 ? r0 : n;
        float lreg[8], yreg[16];
        auto load_chunk = [&](int q0) {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = tid + 128 * u;
            if (pass == 0) {   // LT[t][i] = L[r0+i][q0+t]
              const int i = e >> 5, t = e & 31;
              lreg[u] = (i < rb && q0 + t < q_end) ? L[(size_t)(r0 + i) * n + q0 + t] : 0.0f;
            } else {           // LT[t][i] = L[q0+t][r0+i]
              const int t = e >> 5, i = e & 31;
              lreg[u] = (i < rb && q0 + t < q_end) ? L[(size_t)(q0 + t) * n + r0 + i] : 0.0f;
            }
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {   // YC[k][j] = result[q0+k][cb+j]
            const int e = tid + 128 * u;
            const int k = e >> 6, j = e & 63;
            const int row = q0 + k, col = cb + j;
            yreg[u] = (row < q_end && col < ncol) ? *addr(row, col) : 0.0f;
          }
        };
        auto store_chunk = [&]() {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = tid + 128 * u;
            if (pass == 0) LT[(e & 31) * kRtLd + (e >> 5)] = lreg[u];
            else LT[(e >> 5) * kRtLd + (e & 31)] = lreg[u];
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int e = tid + 128 * u;
            YC[(e >> 6) * kRtYd + (e & 63)] = yreg[u];
          }
        };
        if (q_begin < q_end) load_chunk(q_begin);
        for (int q0 = q_begin; q0 < q_end; q0 += NB) {
          store_chunk();
          __syncthreads();
          if (q0 + NB < q_end) load_chunk(q0 + NB);   // in flight during the FMAs below
#pragma unroll 8
          for (int k = 0; k < NB; ++k) {
            const float4 l4 = *reinterpret_cast<const float4*>(LT + k * kRtLd + 4 * tr);
            const float4 y4 = *reinterpret_cast<const float4*>(YC + k * kRtYd + 4 * tc);
            const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
            const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(-lv[a], yv[c], acc[a][c]);
          }
          __syncthreads();
        }
        // the diagonal block: forward y = X_r acc (XT[t][a] = X_r[a][t]); backward x = X_r^T acc
        // (XT[t][a] = X_r[t][a]); the accumulators of the block go through YC
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = tid + 128 * u;
          const int p = e >> 5, q = e & 31;   // coalesced along q
          if (pass == 0) XT[q * kRtLd + p] = (p < rb && q < rb) ? xinv32(L, n, r0, p, q) : 0.0f;
          else XT[p * kRtLd + q] = (p < rb && q < rb) ? xinv32(L, n, r0, p, q) : 0.0f;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
          *reinterpret_cast<float4*>(YC + (4 * tr + a) * kRtYd + 4 * tc) =
              make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        __syncthreads();
        float o[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) o[a][c] = 0.0f;
#pragma unroll 8
        for (int t = 0; t < NB; ++t) {
          const float4 x4 = *reinterpret_cast<const float4*>(XT + t * kRtLd + 4 * tr);
          const float4 y4 = *reinterpret_cast<const float4*>(YC + t * kRtYd + 4 * tc);
          const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
          const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) o[a][c] = fmaf(xv[a], yv[c], o[a][c]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int row = r0 + 4 * tr + a;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int col = cb + 4 * tc + c;
            if (4 * tr + a < rb && col < ncol) *addr(row, col) = o[a][c];
          }
        }
        __syncthreads();
      }
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

// ------------------------------------------------------------------------------------ mixed-precision Q
// W <- L^-1 W for the b columns of W (n x b row-major, FP32), with the FP32 factor.
__device__ void forward_cols32(const float* __restrict__ L, int n, int b, float* __restrict__ W,
                             float (*Acc)[kMaxB + 1], float (*Xd)[NB + 4]) {
  const int tid = threadIdx.x;
  const int nblk = (n + NB - 1) / NB;
  for (int rbk = 0; rbk < nblk; ++rbk) {   // forward
    const int r0 = rbk * NB, rb = min(NB, n - r0);
    for (int e = tid; e < rb * b; e += kThreads) {
      const int i = e / b, c = e - i * b;
      const float* Li = L + (size_t)(r0 + i) * n;
      // four independent partial sums (the FMA chain is the latency bound here)
      float s0 = W[(size_t)(r0 + i) * b + c], s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
      int q = 0;
      for (; q + 4 <= r0; q += 4) {
        s0 = fmaf(-Li[q], W[(size_t)q * b + c], s0);
        s1 = fmaf(-Li[q + 1], W[(size_t)(q + 1) * b + c], s1);
        s2 = fmaf(-Li[q + 2], W[(size_t)(q + 2) * b + c], s2);
        s3 = fmaf(-Li[q + 3], W[(size_t)(q + 3) * b + c], s3);
      }
      for (; q < r0; ++q) s0 = fmaf(-Li[q], W[(size_t)q * b + c], s0);
      Acc[i][c] = (s0 + s1) + (s2 + s3);
    }
    for (int e = tid; e < NB * NB; e += kThreads) {
      const int a = e >> 5, t = e & 31;
      Xd[a][t] = (a < rb && t < rb) ? xinv32(L, n, r0, a, t) : 0.0f;
    }
    __syncthreads();
    for (int e = tid; e < rb * b; e += kThreads) {
      const int a = e / b, c = e - a * b;
      float s = 0.0f;
      for (int t = 0; t <= a; ++t) s = fmaf(Xd[a][t], Acc[t][c], s);
      W[(size_t)(r0 + a) * b + c] = s;
    }
    __syncthreads();
  }
}

// W <- L^-T W.
__device__ void backward_cols32(const float* __restrict__ L, int n, int b, float* __restrict__ W,
                             float (*Acc)[kMaxB + 1], float (*Xd)[NB + 4]) {
  const int tid = threadIdx.x;
  const int nblk = (n + NB - 1) / NB;
  for (int rbk = nblk - 1; rbk >= 0; --rbk) {   // backward
    const int r0 = rbk * NB, rb = min(NB, n - r0);
    for (int e = tid; e < rb * b; e += kThreads) {
      const int i = e / b, c = e - i * b;
      // four independent partial sums (the FMA chain is the latency bound here)
      float s0 = W[(size_t)(r0 + i) * b + c], s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
      int q = r0 + rb;
      for (; q + 4 <= n; q += 4) {
        s0 = fmaf(-L[(size_t)q * n + r0 + i], W[(size_t)q * b + c], s0);
        s1 = fmaf(-L[(size_t)(q + 1) * n + r0 + i], W[(size_t)(q + 1) * b + c], s1);
        s2 = fmaf(-L[(size_t)(q + 2) * n + r0 + i], W[(size_t)(q + 2) * b + c], s2);
        s3 = fmaf(-L[(size_t)(q + 3) * n + r0 + i], W[(size_t)(q + 3) * b + c], s3);
      }
      for (; q < n; ++q) s0 = fmaf(-L[(size_t)q * n + r0 + i], W[(size_t)q * b + c], s0);
      Acc[i][c] = (s0 + s1) + (s2 + s3);
    }
    for (int e = tid; e < NB * NB; e += kThreads) {
      const int a = e >> 5, t = e & 31;
      Xd[a][t] = (a < rb && t < rb) ? xinv32(L, n, r0, a, t) : 0.0f;
    }
    __syncthreads();
    for (int e = tid; e < rb * b; e += kThreads) {
      const int a = e / b, c = e - a * b;
      float s = 0.0f;
      for (int t = a; t < rb; ++t) s = fmaf(Xd[t][a], Acc[t][c], s);
      W[(size_t)(r0 + a) * b + c] = s;
    }
    __syncthreads();
  }
}

// W <- L^-T L^-1 W for the b columns of W (n x b row-major, FP32), with the FP32 factor.
__device__ void solve_cols32(const float* __restrict__ L, int n, int b, float* __restrict__ W,
                             float (*Acc)[kMaxB + 1], float (*Xd)[NB + 4]) {
  forward_cols32(L, n, b, W, Acc, Xd);
  backward_cols32(L, n, b, W, Acc, Xd);
}

// s = hi + lo: hi the leading 24 significant bits of s (truncated), lo the next 24 (rounded), so 48 of
// the 53 bits, by integer operations and conversions only (no FP64 arithmetic: the FP64 pipe is ~1/60
// of the FP32 one here). For |s| < 2^-74 only hi is kept.
__device__ __forceinline__ float2 split_f64(double s) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(s);
  const float hi = __double2float_rz(__longlong_as_double((long long)(u & ~0x1FFFFFFFull)));
  const int e = (int)((u >> 52) & 0x7FF);
  float lo = 0.0f;
  if (e >= 949 && e <= 1150) {
    // the low 29 significand bits are an integer in units of 2^(e - 1075)
    lo = __uint2float_rn((unsigned)(u & 0x1FFFFFFFull)) * __int_as_float((e - 948) << 23);
    if (u >> 63) lo = -lo;
  }
  return make_float2(hi, lo);
}

// s + c <- s + c + p with s = fl(s + p) and the rounding error of that sum added to c (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float& s, float& c, float p) {
  const float t = s + p;
  const float z = t - s;
  c += (s - (t - z)) + (p - z);
  s = t;
}

// R = E_c - S q (S the full symmetric T_J(S) in FP64, q given as hi + lo FP32 pairs), written to R in
// FP32, in double-FP32 arithmetic (the compensated dot product of Ogita, Rump and Oishi): the hi*hi
// products are split exactly (fmaf) and summed with TwoSum, the hi*lo and lo*hi products summed plainly.
// The sums are accurate to about n 2^-48 of |S||q|, which is what the refinement of q needs from its
// residual. One thread per row (no cross-lane sums), the row read four elements at a time, q broadcast;
// up to 8 columns of q per sweep.
__device__ void residual_df(const double* __restrict__ S, int n, int c0, int b, const float2* __restrict__ qp,
                            float* __restrict__ R) {
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const double* Si = S + (size_t)i * n;
    for (int cg = 0; cg < b; cg += 8) {
      const int cn = min(8, b - cg);
      float sh[8], sl[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) sh[c] = sl[c] = 0.0f;
      int k = 0;
      for (; k + 4 <= n; k += 4) {
        double sv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) sv[u] = Si[k + u];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 a = split_f64(sv[u]);
          const float2* qk = qp + (size_t)(k + u) * b + cg;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (c < cn) {
              const float2 v = qk[c];
              const float p = a.x * v.x;
              sl[c] += fmaf(a.x, v.x, -p);
              two_sum(sh[c], sl[c], p);
              sl[c] = fmaf(a.x, v.y, fmaf(a.y, v.x, sl[c]));
            }
          }
        }
      }
      for (; k < n; ++k) {
        const float2 a = split_f64(Si[k]);
        const float2* qk = qp + (size_t)k * b + cg;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c < cn) {
            const float2 v = qk[c];
            const float p = a.x * v.x;
            sl[c] += fmaf(a.x, v.x, -p);
            two_sum(sh[c], sl[c], p);
            sl[c] = fmaf(a.x, v.y, fmaf(a.y, v.x, sl[c]));
          }
        }
      }
      // 1 - sh is exact when sh is within a factor 2 of 1 (Sterbenz), as it is near the solution
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < cn) R[(size_t)i * b + cg + c] = ((i == c0 + cg + c ? 1.0f : 0.0f) - sh[c]) - sl[c];
    }
  }
}

// Gershgorin interval of A (n x n, FP32 or FP64) widened by its rounding, into lam[2J], lam[2J+1].
template <typename TA>
__device__ void gershgorin(const TA* __restrict__ A, int n, double* lam, float* rlo, float* rhi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float lo = INFINITY, hi = -INFINITY;
  for (int i0 = 4 * warp; i0 < n; i0 += 4 * (kThreads / 32)) {   // four rows per warp pass, lanes along them
    float r[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int j = lane; j < n; j += 32) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        if (i < n && j != i) r[u] += fabsf((float)A[(size_t)i * n + j]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      for (int o = 16; o > 0; o >>= 1) r[u] += __shfl_xor_sync(0xffffffffu, r[u], o);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u;
      if (i < n) {
        const float d = (float)A[(size_t)i * n + i];
        lo = fminf(lo, d - r[u]);
        hi = fmaxf(hi, d + r[u]);
      }
    }
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
    lam[0] = (double)rlo[0] - w;
    lam[1] = (double)rhi[0] + w;
  }
}


// ------------------------------------------------------------------------------------ kernels
template <typename TA>
__global__ void __launch_bounds__(kThreads, 2) k_prepare(PrepArgs g, TA* __restrict__ Acache) {
  extern __shared__ __align__(16) double Ps[];   // factorisation panel: n x (NB+1) doubles
  __shared__ double Xs[NB][NB + 1];
  __shared__ __align__(16) unsigned char raw[sizeof(double) * NB * (kMaxB + 1)];
  __shared__ double s_rinv[2];
  __shared__ int s_bad;
  __shared__ float rlo[kThreads], rhi[kThreads];
  const int J = g.j0 + blockIdx.x;
  if (g.only_flagged && g.prep_status[J] != kSubRefine) return;
  const int n = g.sub_n[J];
  const int bJ = g.nbf[J];
  const int c0 = g.sub_c0[J];
  double* S = g.ws + (g.a_off[J] - g.a_base);
  const double* H = S + g.chunk_n2;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const bool ok = cholesky<double>(S, n, Ps, Xs, s_rinv, &s_bad);
  if (threadIdx.x == 0) g.prep_status[J] = ok ? kSubOk : kSubNotSpd;
  if (!ok) return;   // uniform: every thread read the flag after the same barrier
  // A_J in TA (shared memory reused: two T tiles)
  TA* A = Acache + g.a_off[J];
  TA* Lp = reinterpret_cast<TA*>(Ps);
  solve_A<TA, double>(S, H, n, A, Lp, Lp + NB * Ld<TA>::v);
  __syncthreads();
  // Q_J in FP64
  solve_Q(S, n, c0, bJ, g.Q + g.c_off[J], reinterpret_cast<double (*)[kMaxB + 1]>(raw), Xs);
  __syncthreads();
  gershgorin(A, n, g.lam + 2 * J, rlo, rhi);
}

__global__ void __launch_bounds__(kThreads, 4) k_prepare_mixed(PrepArgs g, float* __restrict__ Acache) {
  extern __shared__ __align__(16) float Pf[];   // panel (n x (NB+4)), then solve tiles ((n+36) x (NB+4))
  __shared__ __align__(16) float Xs[NB][NB + 4];
  __shared__ int s_bad;
  __shared__ float rlo[kThreads], rhi[kThreads];
  __shared__ float red_d[kThreads / 32];
  __shared__ double red_q[kThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int J = g.order ? g.order[blockIdx.x] : g.j0 + (int)blockIdx.x;   // largest submatrices first
  const int n = g.sub_n[J];
  const int bJ = g.nbf[J];
  const int c0 = g.sub_c0[J];
  const double* S = g.ws + (g.a_off[J] - g.a_base);
  const double* H = S + g.chunk_n2;
  float* L = g.L32 + (g.a_off[J] - g.a_base);
  float (*Acc)[kMaxB + 1] = reinterpret_cast<float (*)[kMaxB + 1]>(Pf);   // solve_cols32 (after the solves)
  if (tid == 0) s_bad = 0;
  __syncthreads();
  bool ok = cholesky32(L, S, n, Pf, Xs, &s_bad);
  if (ok && g.cond) {
    // cond(T_J(S)) >= (max_i L_ii / min_i L_ii)^2; the factor keeps 1 / L_ii on its diagonal, whose ratio is
    // the same
    float mn = INFINITY, mx = 0.0f;
    for (int i = tid; i < n; i += kThreads) {
      const float d = L[(size_t)i * n + i];
      mn = fminf(mn, d);
      mx = fmaxf(mx, d);
    }
    rlo[tid] = mn;
    rhi[tid] = mx;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
      if (tid < s) {
        rlo[tid] = fminf(rlo[tid], rlo[tid + s]);
        rhi[tid] = fmaxf(rhi[tid], rhi[tid + s]);
      }
      __syncthreads();
    }
    if (tid == 0) g.cond[J] = (rhi[0] / rlo[0]) * (rhi[0] / rlo[0]);
    __syncthreads();
  }
  if (ok) {
    // A_J = L^-T L^-1 T_J(H0) in FP32, and the FP32 first solve of Q when its b columns fit in the
    // last column batch
    float* A = Acache + g.a_off[J];
    const int nbc = n * bJ;
    float* w = g.W32 + (g.c_off[J] - g.c_base);
    float2* qp = g.Qp + (g.c_off[J] - g.c_base);
    double* q = g.Q + g.c_off[J];
    const bool merge_q = !g.sym && (n + bJ + kRtCb - 1) / kRtCb == (n + kRtCb - 1) / kRtCb;
    if (g.sym) {
      // the symmetric form M = L^-1 T_J(H0) L^-T = L^-1 (L^-1 T_J(H0))^T and W_c = L^-1 E_c
      float* Y = g.Ysym + (g.a_off[J] - g.a_base);
      solve_A_rt<1>(L, H, n, c0, bJ, Y, w, Pf);
      for (int e = tid; e < nbc; e += kThreads) g.Wc[g.c_off[J] + e] = (double)w[e];
      __syncthreads();
      solve_A_rt<2>(L, H, n, c0, 0, A, nullptr, Pf, Y);
    } else {
      solve_A_rt<0>(L, H, n, c0, merge_q ? bJ : 0, A, w, Pf);
    }
    if (!merge_q) {
      for (int e = tid; e < nbc; e += kThreads) {
        const int i = e / bJ, c = e - i * bJ;
        w[e] = (i == c0 + c) ? 1.0f : 0.0f;
      }
      __syncthreads();
      solve_cols32(L, n, bJ, w, Acc, Xs);
    }
    // Q_J: refinement with the double-FP32 residual
    for (int e = tid; e < nbc; e += kThreads) q[e] = (double)w[e];
    __syncthreads();
    bool conv = false;
    for (int it = 0; it < kRefineMax && !conv; ++it) {
      for (int e = tid; e < nbc; e += kThreads) qp[e] = split_f64(q[e]);
      __syncthreads();
      residual_df(S, n, c0, bJ, qp, w);
      __syncthreads();
      solve_cols32(L, n, bJ, w, Acc, Xs);
      float dmax = 0.0f;
      double qmax = 0.0;
      bool finite = true;
      for (int e = tid; e < nbc; e += kThreads) {
        const float d = w[e];
        const double qe = q[e] + (double)d;
        q[e] = qe;
        finite = finite && isfinite(d) && isfinite(qe);
        dmax = fmaxf(dmax, fabsf(d));
        qmax = fmax(qmax, fabs(qe));
      }
      if (!finite) dmax = INFINITY;
      for (int o = 16; o > 0; o >>= 1) {
        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        qmax = fmax(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
      }
      if (lane == 0) {
        red_d[warp] = dmax;
        red_q[warp] = qmax;
      }
      __syncthreads();
      float dm = 0.0f;
      double qm = 0.0;
      for (int w2 = 0; w2 < kThreads / 32; ++w2) {
        dm = fmaxf(dm, red_d[w2]);
        qm = fmax(qm, red_q[w2]);
      }
      conv = (double)dm <= kRefineTol * qm;   // the same shared values in every thread
      __syncthreads();
    }
    ok = conv;
    if (ok) gershgorin(A, n, g.lam + 2 * J, rlo, rhi);
  }
  // a failed FP32 factor or a refinement that did not contract: the FP64 preparation takes the
  // submatrix again when its panel fits in shared memory; otherwise T_J(S) counts as not positive
  // definite in working precision
  if (tid == 0) g.prep_status[J] = ok ? kSubOk : (n <= g.fallback_max_n ? kSubRefine : kSubNotSpd);
}

// One row i of R = E_c - T_J(S) q for CN centre columns: S_i[k] at Si[k] (kCol false: Si is row i, each lane
// streams its own row through L1) or at Si[k n] (kCol: Si is column i of the symmetric T_J(S), the lanes of a
// warp read consecutive entries; better for long rows, whose lines leave L1 before their reuse); against q
// (float2 hi/lo pairs, rows of stride bJ), products and sums in double-FP32 arithmetic (each product's
// rounding error by FMA, each sum's by TwoSum); column c is on the diagonal of E_c when c == ce. Writes w[c]
// (FP32) when rv.
template <int CN, bool kCol>
__device__ __forceinline__ void residual_row(const double* __restrict__ Si, const float2* __restrict__ q, int n,
                                             int bJ, bool rv, int ce, float* __restrict__ w) {
  float sh[CN], sl[CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) sh[c] = sl[c] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < n; ++k) {
    const float2 a = split_f64(Si[kCol ? (size_t)k * n : (size_t)k]);
    const float2* qk = q + (size_t)k * bJ;
#pragma unroll
    for (int c = 0; c < CN; ++c) {
      const float2 v = qk[c];
      const float pr = a.x * v.x;
      sl[c] += fmaf(a.x, v.x, -pr);
      two_sum(sh[c], sl[c], pr);
      sl[c] = fmaf(a.x, v.y, fmaf(a.y, v.x, sl[c]));
    }
  }
  if (rv) {
#pragma unroll
    for (int c = 0; c < CN; ++c) w[c] = ((c == ce ? 1.0f : 0.0f) - sh[c]) - sl[c];
  }
}

// One row i of the correction X R (kCol false: xi is row i of X) or X^T R (kCol: xi is column i; X =
// T_J(S)^-1 is symmetric up to its rounding, so its transpose serves as the approximate inverse as well) for
// CN columns of R (FP32, rows of stride bJ): four interleaved FP32 partial sums along k per column, added at
// the end; d[c] for c < CN.
template <int CN, bool kCol>
__device__ __forceinline__ void update_row(const float* __restrict__ xi, const float* __restrict__ R, int n, int bJ,
                                           float (&d)[8]) {
  float acc[4][CN];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int c = 0; c < CN; ++c) acc[u][c] = 0.0f;
  int k = 0;
  for (; k + 4 <= n; k += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float x = xi[kCol ? (size_t)(k + u) * n : (size_t)(k + u)];
      const float* rk = R + (size_t)(k + u) * bJ;
#pragma unroll
      for (int c = 0; c < CN; ++c) acc[u][c] = fmaf(x, rk[c], acc[u][c]);
    }
  }
  for (; k < n; ++k) {
    const float x = xi[kCol ? (size_t)k * n : (size_t)k];
    const float* rk = R + (size_t)k * bJ;
#pragma unroll
    for (int c = 0; c < CN; ++c) acc[0][c] = fmaf(x, rk[c], acc[0][c]);
  }
#pragma unroll
  for (int c = 0; c < CN; ++c) d[c] = (acc[0][c] + acc[1][c]) + (acc[2][c] + acc[3][c]);
}

// After the tensor-core inverse square root (Eqs. inv1-inv3), which leaves X = T_J(S)^-1 in FP32 (in g.L32,
// accurate to about 1e-6 of its norm) and A_J in Acache: the centre columns of T_J(S)^-1 by iterative
// refinement with X as the approximate inverse (for n above 256 its transpose, read coalesced: X is symmetric up
// to its rounding), q <- q + X (E_c - T_J(S) q) from q = X[:, centre], the
// residual in double-FP32 arithmetic (as in k_prepare_mixed), until the correction is below 1e-6 of q; then
// the Gershgorin interval of A_J. A submatrix the inverse kernel flagged, or whose refinement does not
// contract, is left flagged for the FP64 preparation.
__global__ void __launch_bounds__(kThreads) k_ns_qrefine(PrepArgs g, const float* __restrict__ Acache) {
  extern __shared__ __align__(16) float Wsh[];   // the residual, n x b
  __shared__ float rlo[kThreads], rhi[kThreads];
  __shared__ float red_d[kThreads / 32];
  __shared__ double red_q[kThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int J = g.order ? g.order[blockIdx.x] : g.j0 + (int)blockIdx.x;
  if (g.prep_status[J] != kSubOk) return;
  const int n = g.sub_n[J], bJ = g.nbf[J], c0 = g.sub_c0[J], nbc = n * bJ;
  const double* S = g.ws + (g.a_off[J] - g.a_base);
  const float* X = g.L32 + (g.a_off[J] - g.a_base);
  float2* qp = g.Qp + (g.c_off[J] - g.c_base);
  double* q = g.Q + g.c_off[J];
  for (int e = tid; e < nbc; e += kThreads) {
    const int i = e / bJ, c = e - i * bJ;
    q[e] = (double)X[(size_t)i * n + c0 + c];
  }
  if (g.cond) {   // cond(T_J(S)) >= max_i S_ii (T_J(S)^-1)_ii
    float mx = 0.0f;
    for (int i = tid; i < n; i += kThreads) mx = fmaxf(mx, (float)S[(size_t)i * n + i] * X[(size_t)i * n + i]);
    rhi[tid] = mx;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
      if (tid < s) rhi[tid] = fmaxf(rhi[tid], rhi[tid + s]);
      __syncthreads();
    }
    if (tid == 0) g.cond[J] = rhi[0];
  }
  __syncthreads();
  bool conv = false;
  constexpr int kWarps = kThreads / 32;
  // rows of T_J(S) and X read along the row by each lane up to 256 columns, as columns (coalesced) beyond
  const bool col = n > 256;
  for (int it = 0; it < kRefineMax && !conv; ++it) {
    for (int e = tid; e < nbc; e += kThreads) qp[e] = split_f64(q[e]);
    __syncthreads();
    // R = E_c - T_J(S) q: one row per lane (for n above 256 read as the column of the symmetric T_J(S):
    // coalesced), the row's products along k in double-FP32 arithmetic (as residual_df), up to 8 centre columns
    // per sweep; every lane reads the same entries of q
    for (int i0 = 32 * warp; i0 < n; i0 += 32 * kWarps) {
      const int i = i0 + lane;
      const bool rv = i < n;
      const double* Si = col ? S + (rv ? i : 0) : S + (size_t)(rv ? i : 0) * n;   // row i (or column i)
      for (int cg = 0; cg < bJ; cg += 8) {
        float* w = Wsh + (size_t)(rv ? i : 0) * bJ + cg;
        const float2* qc = qp + cg;
        const int ce = i - c0 - cg;   // row i holds the 1 of E_c's column cg + c when c == ce
        switch (min(8, bJ - cg)) {
          case 1: col ? residual_row<1, true>(Si, qc, n, bJ, rv, ce, w) : residual_row<1, false>(Si, qc, n, bJ, rv, ce, w); break;
          case 2: col ? residual_row<2, true>(Si, qc, n, bJ, rv, ce, w) : residual_row<2, false>(Si, qc, n, bJ, rv, ce, w); break;
          case 3: col ? residual_row<3, true>(Si, qc, n, bJ, rv, ce, w) : residual_row<3, false>(Si, qc, n, bJ, rv, ce, w); break;
          case 4: col ? residual_row<4, true>(Si, qc, n, bJ, rv, ce, w) : residual_row<4, false>(Si, qc, n, bJ, rv, ce, w); break;
          case 5: col ? residual_row<5, true>(Si, qc, n, bJ, rv, ce, w) : residual_row<5, false>(Si, qc, n, bJ, rv, ce, w); break;
          case 6: col ? residual_row<6, true>(Si, qc, n, bJ, rv, ce, w) : residual_row<6, false>(Si, qc, n, bJ, rv, ce, w); break;
          case 7: col ? residual_row<7, true>(Si, qc, n, bJ, rv, ce, w) : residual_row<7, false>(Si, qc, n, bJ, rv, ce, w); break;
          default: col ? residual_row<8, true>(Si, qc, n, bJ, rv, ce, w) : residual_row<8, false>(Si, qc, n, bJ, rv, ce, w); break;
        }
      }
    }
    __syncthreads();
    // q <- q + X R (for n above 256 X^T R, one column of X per lane: coalesced), R from shared memory (the
    // same entries for every lane)
    float dmax = 0.0f;
    double qmax = 0.0;
    bool finite = true;
    for (int i0 = 32 * warp; i0 < n; i0 += 32 * kWarps) {
      const int i = i0 + lane;
      const bool rv = i < n;
      const float* xi = col ? X + (rv ? i : 0) : X + (size_t)(rv ? i : 0) * n;
      for (int cg = 0; cg < bJ; cg += 8) {
        const int cn = min(8, bJ - cg);
        float d[8];
        switch (cn) {
          case 1: col ? update_row<1, true>(xi, Wsh + cg, n, bJ, d) : update_row<1, false>(xi, Wsh + cg, n, bJ, d); break;
          case 2: col ? update_row<2, true>(xi, Wsh + cg, n, bJ, d) : update_row<2, false>(xi, Wsh + cg, n, bJ, d); break;
          case 3: col ? update_row<3, true>(xi, Wsh + cg, n, bJ, d) : update_row<3, false>(xi, Wsh + cg, n, bJ, d); break;
          case 4: col ? update_row<4, true>(xi, Wsh + cg, n, bJ, d) : update_row<4, false>(xi, Wsh + cg, n, bJ, d); break;
          case 5: col ? update_row<5, true>(xi, Wsh + cg, n, bJ, d) : update_row<5, false>(xi, Wsh + cg, n, bJ, d); break;
          case 6: col ? update_row<6, true>(xi, Wsh + cg, n, bJ, d) : update_row<6, false>(xi, Wsh + cg, n, bJ, d); break;
          case 7: col ? update_row<7, true>(xi, Wsh + cg, n, bJ, d) : update_row<7, false>(xi, Wsh + cg, n, bJ, d); break;
          default: col ? update_row<8, true>(xi, Wsh + cg, n, bJ, d) : update_row<8, false>(xi, Wsh + cg, n, bJ, d); break;
        }
        if (rv) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (c < cn) {
              const size_t e = (size_t)i * bJ + cg + c;
              const double qe = q[e] + (double)d[c];
              q[e] = qe;
              finite = finite && isfinite(d[c]) && isfinite(qe);
              dmax = fmaxf(dmax, fabsf(d[c]));
              qmax = fmax(qmax, fabs(qe));
            }
          }
        }
      }
    }
    if (!finite) dmax = INFINITY;
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      qmax = fmax(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
    }
    if (lane == 0) {
      red_d[warp] = dmax;
      red_q[warp] = qmax;
    }
    __syncthreads();
    float dm = 0.0f;
    double qm = 0.0;
    for (int w2 = 0; w2 < kWarps; ++w2) {
      dm = fmaxf(dm, red_d[w2]);
      qm = fmax(qm, red_q[w2]);
    }
    // converged when the correction is below 1e-6 of q, or after the first step when that correction (the
    // error of X's columns, about the contraction factor ||I - X T_J(S)|| too) is below 1e-5 of q: the error
    // left is then about its square, below 1e-10 of q
    conv = (double)dm <= kRefineTol * qm || (it == 0 && (double)dm <= kNsOneStep * qm);
    __syncthreads();
  }
  if (conv) gershgorin(Acache + g.a_off[J], n, g.lam + 2 * J, rlo, rhi);
  if (tid == 0) g.prep_status[J] = conv ? kSubOk : (n <= g.fallback_max_n ? kSubRefine : kSubNotSpd);
}

// The symmetric form's last step, after the sign kernel: its centre-column phase leaves
// U = 1/2 (I - X~) W_c in Dc (W_c = L^-1 E_c, X~ = sign of M - mu I); here D_c = L^-T U with the FP32 factor
// (Eq. purification_submatrix: T_J(D) = L^-T 1/2 (I - X~) L^-1), and the partial traces in FP64.
__global__ void __launch_bounds__(kThreads) k_sym_finish(SymArgs g) {
  extern __shared__ __align__(16) float Wsh[];   // n x b
  __shared__ float Acc[NB][kMaxB + 1];
  __shared__ __align__(16) float Xd[NB][NB + 4];
  __shared__ double red[2][kThreads / 32];
  const int tid = threadIdx.x;
  const int J = g.list ? g.list[blockIdx.x] : g.j0 + (int)blockIdx.x;
  if (J < 0 || g.prep_status[J] != kSubOk) return;
  const int n = g.sub_n[J], b = g.nbf[J], nb = n * b;
  const float* L = g.L + g.a_off[J];
  double* Dc = g.Dc + g.c_off[J];
  for (int e = tid; e < nb; e += kThreads) Wsh[e] = (float)Dc[e];
  __syncthreads();
  backward_cols32(L, n, b, Wsh, Acc, Xd);
  double ps = 0.0, ph = 0.0;
  const double* Sc = g.Sc + g.c_off[J];
  const double* Hc = g.Hc + g.c_off[J];
  for (int e = tid; e < nb; e += kThreads) {
    const double d = (double)Wsh[e];
    Dc[e] = d;
    ps += d * Sc[e];
    ph += d * Hc[e];
  }
  for (int o = 16; o > 0; o >>= 1) {
    ps += __shfl_xor_sync(0xffffffffu, ps, o);
    ph += __shfl_xor_sync(0xffffffffu, ph, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = ps;
    red[1][tid >> 5] = ph;
  }
  __syncthreads();
  if (tid == 0) {
    double ts = 0.0, th = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      ts += red[0][w];
      th += red[1][w];
    }
    g.tS[J] = ts;
    g.tH[J] = th;
    if (g.status[J] == kSubOk && !(isfinite(ts) && isfinite(th))) g.status[J] = kSubNonFinite;
  }
}

size_t smem_fp64(int max_n) { return sizeof(double) * (size_t)std::max(max_n, 2 * NB) * (NB + 1); }
size_t smem_mixed(int max_n) {
  return sizeof(float) * std::max((size_t)(std::max(max_n, 2 * NB) + 36) * Ld<float>::v, (size_t)kRtSmem);
}
constexpr size_t kSmemLimit = 200 * 1024;

}  // namespace

int prepare_fp64_max_n() { return (int)(kSmemLimit / (sizeof(double) * (NB + 1))); }

nolsm_status launch_prepare(const PrepArgs& g, int count, int max_n, bool fp64_A, void* Acache, cudaStream_t st) {
  const size_t smem = smem_fp64(max_n);
  if (smem > kSmemLimit) {
    set_error("submatrix dimension %d exceeds the FP64 factorisation panel's shared memory (n <= %d)", max_n,
              prepare_fp64_max_n());
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

nolsm_status launch_sym_finish(const SymArgs& g, int count, int max_n, int max_b, cudaStream_t st) {
  if (count <= 0) return NOLSM_OK;
  const size_t smem = sizeof(float) * (size_t)max_n * max_b;
  NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_sym_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sym_finish<<<count, kThreads, smem, st>>>(g);
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}

nolsm_status launch_ns_qrefine(const PrepArgs& g, int count, int max_n, int max_b, float* Acache, cudaStream_t st) {
  const size_t smem = sizeof(float) * (size_t)max_n * max_b;
  if (smem > kSmemLimit) {
    set_error("submatrix dimension %d x %d centre columns exceed the refinement's shared memory", max_n, max_b);
    return NOLSM_ERR_UNSUPPORTED;
  }
  NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_ns_qrefine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_ns_qrefine<<<count, kThreads, smem, st>>>(g, Acache);
  NOLSM_LAUNCH_CHECK();
  PrepArgs f = g;
  f.only_flagged = 1;
  NOLSM_TRY(launch_prepare(f, count, std::min(max_n, prepare_fp64_max_n()), false, Acache, st));
  return NOLSM_OK;
}

nolsm_status launch_prepare_mixed(const PrepArgs& g, int count, int max_n, float* Acache, cudaStream_t st) {
  const size_t smem = smem_mixed(max_n);
  if (smem > kSmemLimit) {
    set_error("submatrix dimension %d exceeds the FP32 factorisation panel's shared memory (n <= %d)", max_n,
              (int)(kSmemLimit / (sizeof(float) * Ld<float>::v)));
    return NOLSM_ERR_UNSUPPORTED;
  }
  NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_prepare_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_prepare_mixed<<<count, kThreads, smem, st>>>(g, Acache);
  NOLSM_LAUNCH_CHECK();
  // the FP64 preparation again for the flagged submatrices (every other CTA returns at once); the
  // symmetric form flags none (it has no FP64 fallback)
  if (g.sym) return NOLSM_OK;
  PrepArgs f = g;
  f.only_flagged = 1;
  NOLSM_TRY(launch_prepare(f, count, std::min(max_n, prepare_fp64_max_n()), false, Acache, st));
  return NOLSM_OK;
}

}  // namespace nolsm
