// a4 bound sources other than the Gershgorin interval, and a10, the learned bound predictor.
//
// Power iteration (a4): the extreme eigenvalues of A_J = T_J(S)^-1 T_J(H0) (real: A_J is similar to the
// symmetric L^-1 T_J(H0) L^-T) from two shifted power iterations run side by side on the prepared A_J:
//   u <- (A - lo I) u / ||.||   ->  ||(A - lo I) u|| -> hi_true - lo
//   v <- (hi I - A) v / ||.||   ->  ||(hi I - A) v|| -> hi - lo_true
// where [lo, hi] is the Gershgorin interval (every eigenvalue of both shifted matrices is >= 0). After
// k steps the estimates are widened by 5 % of the estimated spectral width on each side and clipped to
// the Gershgorin interval. The Newton-Schulz iteration tolerates a scale down to rho / sqrt(3), and a
// submatrix that still fails the convergence test is solved again with the Gershgorin interval.
//
// Learned predictor (a10): features of each submatrix (dimension, Gershgorin interval, neighbourhood
// size, statistics of the on-site energies, mu) -> three dense layers of width 128 (tanh, tanh, linear)
// -> (lowest eigenvalue, highest eigenvalue, Newton-Schulz steps / 16), trained on the power-iteration
// interval (already widened) and step counts. The predicted interval, widened by 1 % of its width for the
// network's own error and clipped to the Gershgorin interval, sets the scale; the predicted step count sets
// a per-submatrix step budget. Any submatrix that fails the convergence test under the learned bounds
// is solved again with power-iteration bounds, so none is accepted unconverged.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bounds.cuh"
#include "nolsm_internal.cuh"

namespace nolsm {

namespace {

constexpr int kPowThreads = 256;

__device__ __forceinline__ float block_sum_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = 0.0f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// One CTA per submatrix of the list (or of [j0, j0 + count) when list is null).
template <typename TA>
__global__ void __launch_bounds__(kPowThreads) k_power_bounds(PowArgs g, const TA* __restrict__ Acache) {
  extern __shared__ float sv[];   // u[n], v[n], u'[n], v'[n]
  __shared__ float red[kPowThreads / 32];
  const int J = g.list ? g.list[blockIdx.x] : g.j0 + (int)blockIdx.x;
  if (J < 0) return;
  const int n = g.sub_n[J];
  if (g.prep_status[J] != kSubOk) {
    if (threadIdx.x == 0) {
      g.lam_p[2 * J] = g.lam[2 * J];
      g.lam_p[2 * J + 1] = g.lam[2 * J + 1];
    }
    return;
  }
  const TA* A = Acache + g.a_off[J];
  const float lo = (float)g.lam[2 * J], hi = (float)g.lam[2 * J + 1];
  float* u = sv;
  float* v = sv + n;
  float* u2 = sv + 2 * n;
  float* v2 = sv + 3 * n;
  // start vector 1 + (i mod 7) / 7 (positive, no random numbers), normalised
  float ss = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float x = 1.0f + (float)(i % 7) / 7.0f;
    u[i] = x;
    v[i] = x;
    ss += x * x;
  }
  ss = block_sum_f(ss, red);
  const float inv0 = rsqrtf(ss);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    u[i] *= inv0;
    v[i] *= inv0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float eu = 0.0f, ev = 0.0f;
  for (int it = 0; it < g.iters; ++it) {
    // u2 = A u - lo u, v2 = hi v - A v: one warp per row, lanes along the row
    for (int i = warp; i < n; i += nw) {
      const TA* Ai = A + (size_t)i * n;
      float au = 0.0f, av = 0.0f;
      for (int k = lane; k < n; k += 32) {
        const float a = (float)Ai[k];
        au = fmaf(a, u[k], au);
        av = fmaf(a, v[k], av);
      }
      for (int o = 16; o > 0; o >>= 1) {
        au += __shfl_xor_sync(0xffffffffu, au, o);
        av += __shfl_xor_sync(0xffffffffu, av, o);
      }
      if (lane == 0) {
        u2[i] = au - lo * u[i];
        v2[i] = hi * v[i] - av;
      }
    }
    __syncthreads();
    float su = 0.0f, sw = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      su += u2[i] * u2[i];
      sw += v2[i] * v2[i];
    }
    su = block_sum_f(su, red);
    sw = block_sum_f(sw, red);
    eu = sqrtf(su);
    ev = sqrtf(sw);
    const float iu = eu > 0.0f ? 1.0f / eu : 0.0f, iv = ev > 0.0f ? 1.0f / ev : 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      u[i] = u2[i] * iu;
      v[i] = v2[i] * iv;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double ehi = (double)lo + (double)eu, elo = (double)hi - (double)ev;
    const double w = fmax(ehi - elo, 1e-12);
    double plo = elo - 0.05 * w, phi = ehi + 0.05 * w;
    plo = fmax(plo, g.lam[2 * J]);
    phi = fmin(phi, g.lam[2 * J + 1]);
    if (!(plo < phi) || !isfinite(plo) || !isfinite(phi)) {
      plo = g.lam[2 * J];
      phi = g.lam[2 * J + 1];
    }
    g.lam_p[2 * J] = plo;
    g.lam_p[2 * J + 1] = phi;
  }
}

// On-site statistics per molecule I: sum and sum of squares of diag(H0_II), and b_I.
// The same sums from the element model's on-site energies (generated elements: H0_II = diag(onsite of I)).
__global__ void k_onsite_model(int32_t n_mol, const int64_t* __restrict__ off, const double* __restrict__ e,
                               double* __restrict__ out /* [n_mol][2] */) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_mol) return;
  double s = 0.0, q = 0.0;
  for (int64_t k = off[I]; k < off[I + 1]; ++k) {
    s += e[k];
    q += e[k] * e[k];
  }
  out[2 * I] = s;
  out[2 * I + 1] = q;
}

__global__ void k_onsite(int32_t n_mol, const int32_t* __restrict__ nbf, const int32_t* __restrict__ rp,
                         const int32_t* __restrict__ ci, const int64_t* __restrict__ boff,
                         const double* __restrict__ vals, double* __restrict__ out /* [n_mol][2] */) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_mol) return;
  int lo = rp[I], hi = rp[I + 1] - 1, k = -1;
  while (lo <= hi) {   // the block row is sorted; find column I
    const int m = (lo + hi) >> 1;
    const int c = ci[m];
    if (c == I) { k = m; break; }
    if (c < I) lo = m + 1; else hi = m - 1;
  }
  double s = 0.0, q = 0.0;
  const int b = nbf[I];
  if (k >= 0) {
    const double* blk = vals + boff[k];
    for (int a = 0; a < b; ++a) {
      const double d = blk[(size_t)a * b + a];
      s += d;
      q += d * d;
    }
  }
  out[2 * I] = s;
  out[2 * I + 1] = q;
}

// Feature vector of submatrix J (order of the oracle's features()).
__global__ void k_features(FeatArgs g) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = g.j0 + k;
  if (J >= g.j1) return;
  float* f = g.feat + (size_t)J * kFeatures;
  const int p0 = g.nb_ptr[J], p1 = g.nb_ptr[J + 1];
  double s = 0.0, q = 0.0, cnt = 0.0;
  for (int p = p0; p < p1; ++p) {
    const int I = g.nb_idx[p];
    s += g.onsite[2 * I];
    q += g.onsite[2 * I + 1];
    cnt += g.nbf[I];
  }
  const double mean = s / cnt;
  const double var = fmax(q / cnt - mean * mean, 0.0);
  f[0] = (float)(g.sub_n[J] / 100.0);
  f[1] = (float)g.lam[2 * J];
  f[2] = (float)g.lam[2 * J + 1];
  f[3] = (float)((p1 - p0) / 32.0);
  f[4] = (float)mean;
  f[5] = (float)sqrt(var);
  f[6] = (float)g.mu;
}

// Predicted interval (widened, clipped to the Gershgorin interval) and step budget from the MLP outputs.
__global__ void k_mlp_bounds(int32_t j0, int32_t j1, const float* __restrict__ y, const double* __restrict__ lam,
                             int32_t max_iter, double* __restrict__ lam_m, int32_t* __restrict__ budget) {
  const int J = j0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= j1) return;
  const float* yj = y + (size_t)J * kOutputs;
  double a = yj[0], b = yj[1];
  if (a > b) { const double t = a; a = b; b = t; }
  const double w = fmax(b - a, 1e-6);
  double lo = fmax(a - 0.01 * w, lam[2 * J]);
  double hi = fmin(b + 0.01 * w, lam[2 * J + 1]);
  if (!(lo < hi) || !isfinite(lo) || !isfinite(hi)) {
    lo = lam[2 * J];
    hi = lam[2 * J + 1];
  }
  lam_m[2 * J] = lo;
  lam_m[2 * J + 1] = hi;
  const float k = yj[2] * 16.0f;
  int bud = isfinite(k) ? (int)ceilf(1.5f * fmaxf(k, 1.0f)) + 3 : max_iter;
  budget[J] = min(max(bud, 4), max_iter);
}

// Training targets of submatrix J: power-iteration interval and Newton-Schulz steps / 16.
__global__ void k_targets(int32_t j0, int32_t j1, const double* __restrict__ lam_p, const int32_t* __restrict__ iters,
                          float* __restrict__ t) {
  const int J = j0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= j1) return;
  t[(size_t)J * kOutputs] = (float)lam_p[2 * J];
  t[(size_t)J * kOutputs + 1] = (float)lam_p[2 * J + 1];
  t[(size_t)J * kOutputs + 2] = (float)iters[J] / 16.0f;
}

// Submatrices of [j0, j1) whose sign iteration failed (not converged or non-finite), into list[0, count).
__global__ void k_failed(int32_t j0, int32_t j1, const int32_t* __restrict__ status, int32_t* __restrict__ list,
                         int32_t* __restrict__ count) {
  const int J = j0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= j1) return;
  const int s = status[J];
  if (s == kSubNotConv || s == kSubNonFinite) list[atomicAdd(count, 1)] = J;
}

}  // namespace

// ==================================================================================== the MLP
// Parameters (FP32, one flat array): W1 [7][128], b1 [128], W2 [128][128], b2 [128], W3 [128][3], b3 [3],
// weights [fan_in][fan_out] row-major. Activations saved by the forward pass: act[b] = (h1, h2).

namespace {

constexpr int kW2Ld = kWidth + 1;                                  // W2 rows in shared memory (bank spread)
constexpr int kMlpThreads = 256;                                   // 8 warps, one sample per warp
constexpr size_t kMlpSmemFloats = (size_t)kFeatures * kWidth + kWidth + (size_t)kWidth * kW2Ld + kWidth +
                                  (size_t)kWidth * kOutputs + kOutputs + 8 * 2 * kWidth;
constexpr int kChunk = 32;                                         // samples per weight-gradient block

struct MlpSmem {
  float* W1; float* b1; float* W2; float* b2; float* W3; float* b3; float* wbuf;
};

__device__ MlpSmem load_params(const float* __restrict__ p, float* sm) {
  MlpSmem s;
  s.W1 = sm;
  s.b1 = s.W1 + kFeatures * kWidth;
  s.W2 = s.b1 + kWidth;
  s.b2 = s.W2 + kWidth * kW2Ld;
  s.W3 = s.b2 + kWidth;
  s.b3 = s.W3 + kWidth * kOutputs;
  s.wbuf = s.b3 + kOutputs + 1;   // per-warp vectors (2 x 128 floats)
  s.wbuf = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(s.wbuf) + 15) & ~uintptr_t(15));
  for (int e = threadIdx.x; e < kFeatures * kWidth; e += blockDim.x) s.W1[e] = p[kOffW1 + e];
  for (int e = threadIdx.x; e < kWidth; e += blockDim.x) {
    s.b1[e] = p[kOffB1 + e];
    s.b2[e] = p[kOffB2 + e];
  }
  for (int e = threadIdx.x; e < kWidth * kWidth; e += blockDim.x) s.W2[(e >> 7) * kW2Ld + (e & 127)] = p[kOffW2 + e];
  for (int e = threadIdx.x; e < kWidth * kOutputs; e += blockDim.x) s.W3[e] = p[kOffW3 + e];
  if (threadIdx.x < kOutputs) s.b3[threadIdx.x] = p[kOffB3 + threadIdx.x];
  __syncthreads();
  return s;
}

// y = W3^T tanh(W2^T tanh(W1^T x + b1) + b2) + b3 per sample; act (nullable) receives h1, h2.
__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(const float* __restrict__ params, int32_t B,
                                                             const float* __restrict__ x, float* __restrict__ y,
                                                             float* __restrict__ act) {
  extern __shared__ __align__(16) float msm[];
  const MlpSmem s = load_params(params, msm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* h1w = s.wbuf + warp * 2 * kWidth;
  for (int b = blockIdx.x * 8 + warp; b < B; b += gridDim.x * 8) {
    float xv[kFeatures];
#pragma unroll
    for (int k = 0; k < kFeatures; ++k) xv[k] = x[(size_t)b * kFeatures + k];
    float h1[4], h2[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int u = lane + 32 * m;
      float z = s.b1[u];
#pragma unroll
      for (int k = 0; k < kFeatures; ++k) z = fmaf(xv[k], s.W1[k * kWidth + u], z);
      h1[m] = tanhf(z);
      h1w[u] = h1[m];
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int u = lane + 32 * m;
      float z = s.b2[u];
      for (int k = 0; k < kWidth; ++k) z = fmaf(h1w[k], s.W2[k * kW2Ld + u], z);
      h2[m] = tanhf(z);
    }
    float yo[kOutputs];
#pragma unroll
    for (int o = 0; o < kOutputs; ++o) {
      float p = 0.0f;
#pragma unroll
      for (int m = 0; m < 4; ++m) p = fmaf(h2[m], s.W3[(lane + 32 * m) * kOutputs + o], p);
      for (int off = 16; off > 0; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
      yo[o] = p + s.b3[o];
    }
    if (lane == 0)
#pragma unroll
      for (int o = 0; o < kOutputs; ++o) y[(size_t)b * kOutputs + o] = yo[o];
    if (act) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        act[(size_t)b * 2 * kWidth + lane + 32 * m] = h1[m];
        act[(size_t)b * 2 * kWidth + kWidth + lane + 32 * m] = h2[m];
      }
    }
    __syncwarp();
  }
}

// Per sample: dy = (y - t) / B, dz2 = (dy W3^T) * (1 - h2^2), dz1 = (dz2 W2^T) * (1 - h1^2); the loss
// 1/(2B) sum (y - t)^2 is accumulated into loss (FP64).
__global__ void __launch_bounds__(kMlpThreads) k_mlp_backward(const float* __restrict__ params, int32_t B,
                                                              const float* __restrict__ act,
                                                              const float* __restrict__ y, const float* __restrict__ t,
                                                              float* __restrict__ dz, float* __restrict__ dy,
                                                              double* __restrict__ loss) {
  extern __shared__ __align__(16) float msm[];
  const MlpSmem s = load_params(params, msm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* dz2w = s.wbuf + warp * 2 * kWidth;
  double lsum = 0.0;
  for (int b = blockIdx.x * 8 + warp; b < B; b += gridDim.x * 8) {
    float d[kOutputs];
#pragma unroll
    for (int o = 0; o < kOutputs; ++o) {
      const float r = y[(size_t)b * kOutputs + o] - t[(size_t)b * kOutputs + o];
      d[o] = r / (float)B;
      if (lane == 0) lsum += 0.5 * (double)r * (double)r / (double)B;
    }
    const float* a = act + (size_t)b * 2 * kWidth;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int u = lane + 32 * m;
      float g = 0.0f;
#pragma unroll
      for (int o = 0; o < kOutputs; ++o) g = fmaf(d[o], s.W3[u * kOutputs + o], g);
      const float h2 = a[kWidth + u];
      const float z2 = g * (1.0f - h2 * h2);
      dz2w[u] = z2;
      dz[(size_t)b * 2 * kWidth + kWidth + u] = z2;
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int k = lane + 32 * m;
      float g = 0.0f;
      for (int u = 0; u < kWidth; ++u) g = fmaf(s.W2[k * kW2Ld + u], dz2w[u], g);
      const float h1 = a[k];
      dz[(size_t)b * 2 * kWidth + k] = g * (1.0f - h1 * h1);
    }
    if (lane < kOutputs) dy[(size_t)b * kOutputs + lane] = d[lane];
    __syncwarp();
  }
  if (lane == 0 && lsum != 0.0) atomicAdd(loss, lsum);
}

// Partial weight gradients of one chunk of kChunk samples into part[chunk][kParams].
__global__ void __launch_bounds__(256) k_mlp_wgrad(int32_t B, const float* __restrict__ x,
                                                   const float* __restrict__ act, const float* __restrict__ dz,
                                                   const float* __restrict__ dy, float* __restrict__ part) {
  __shared__ __align__(16) float ha[kChunk][kWidth];   // h1, later h2
  __shared__ __align__(16) float zb[kChunk][kWidth];   // dz2, later dz1
  __shared__ float xs[kChunk][kFeatures];
  __shared__ float ds[kChunk][kOutputs];
  const int c0 = blockIdx.x * kChunk;
  const int tid = threadIdx.x;
  float* out = part + (size_t)blockIdx.x * kParams;
  for (int e = tid; e < kChunk * kWidth; e += 256) {
    const int b = e >> 7, u = e & 127;
    const bool ok = c0 + b < B;
    ha[b][u] = ok ? act[(size_t)(c0 + b) * 2 * kWidth + u] : 0.0f;
    zb[b][u] = ok ? dz[(size_t)(c0 + b) * 2 * kWidth + kWidth + u] : 0.0f;
  }
  for (int e = tid; e < kChunk * kFeatures; e += 256) {
    const int b = e / kFeatures, k = e - b * kFeatures;
    xs[b][k] = c0 + b < B ? x[(size_t)(c0 + b) * kFeatures + k] : 0.0f;
  }
  for (int e = tid; e < kChunk * kOutputs; e += 256) {
    const int b = e / kOutputs, o = e - b * kOutputs;
    ds[b][o] = c0 + b < B ? dy[(size_t)(c0 + b) * kOutputs + o] : 0.0f;
  }
  __syncthreads();
  // gW2[i][j] = sum_b h1[b][i] dz2[b][j]: 8 x 8 outputs per thread
  {
    const int ti = tid >> 4, tj = tid & 15;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = 0.0f;
    for (int b = 0; b < kChunk; ++b) {
      float hv[8], zv[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) hv[a] = ha[b][ti + 16 * a];
#pragma unroll
      for (int c = 0; c < 8; ++c) zv[c] = zb[b][tj + 16 * c];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(hv[a], zv[c], acc[a][c]);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) out[kOffW2 + (ti + 16 * a) * kWidth + tj + 16 * c] = acc[a][c];
  }
  // gb2[j] = sum_b dz2[b][j]
  if (tid < kWidth) {
    float s = 0.0f;
    for (int b = 0; b < kChunk; ++b) s += zb[b][tid];
    out[kOffB2 + tid] = s;
  }
  __syncthreads();
  // second pass: h2 and dz1
  for (int e = tid; e < kChunk * kWidth; e += 256) {
    const int b = e >> 7, u = e & 127;
    const bool ok = c0 + b < B;
    ha[b][u] = ok ? act[(size_t)(c0 + b) * 2 * kWidth + kWidth + u] : 0.0f;
    zb[b][u] = ok ? dz[(size_t)(c0 + b) * 2 * kWidth + u] : 0.0f;
  }
  __syncthreads();
  // gW1[k][u] = sum_b x[b][k] dz1[b][u]
  for (int e = tid; e < kFeatures * kWidth; e += 256) {
    const int k = e >> 7, u = e & 127;
    float s = 0.0f;
    for (int b = 0; b < kChunk; ++b) s = fmaf(xs[b][k], zb[b][u], s);
    out[kOffW1 + e] = s;
  }
  // gb1[u] = sum_b dz1[b][u]
  if (tid < kWidth) {
    float s = 0.0f;
    for (int b = 0; b < kChunk; ++b) s += zb[b][tid];
    out[kOffB1 + tid] = s;
  }
  // gW3[u][o] = sum_b h2[b][u] dy[b][o]
  for (int e = tid; e < kWidth * kOutputs; e += 256) {
    const int u = e / kOutputs, o = e - u * kOutputs;
    float s = 0.0f;
    for (int b = 0; b < kChunk; ++b) s = fmaf(ha[b][u], ds[b][o], s);
    out[kOffW3 + e] = s;
  }
  // gb3[o] = sum_b dy[b][o]
  if (tid < kOutputs) {
    float s = 0.0f;
    for (int b = 0; b < kChunk; ++b) s += ds[b][tid];
    out[kOffB3 + tid] = s;
  }
}

// grad[p] = sum over chunks (fixed order) of part[chunk][p]
__global__ void k_mlp_reduce(int32_t chunks, const float* __restrict__ part, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float s = 0.0f;
  for (int c = 0; c < chunks; ++c) s += part[(size_t)c * kParams + p];
  grad[p] = s;
}

// Adam with bias correction (step t >= 1).
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int32_t t, float lr, float b1, float b2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.0f - powf(b1, (float)t));
  const float vh = vi / (1.0f - powf(b2, (float)t));
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

// SplitMix64 (Steele, Lea and Flood; constants from its published definition) as a counter-based
// generator: the value for counter c is the mixed state seed + (c + 1) * golden gamma.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Glorot-uniform weights U(-sqrt(6/(fan_in+fan_out)), +...), zero biases.
__global__ void k_mlp_init(float* __restrict__ p, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  float lim = 0.0f;
  if (i < kOffB1) lim = sqrtf(6.0f / (kFeatures + kWidth));
  else if (i >= kOffW2 && i < kOffB2) lim = sqrtf(6.0f / (kWidth + kWidth));
  else if (i >= kOffW3 && i < kOffB3) lim = sqrtf(6.0f / (kWidth + kOutputs));
  const float u = (float)(splitmix64(seed, (uint64_t)i) >> 40) * (1.0f / 16777216.0f);   // [0, 1)
  p[i] = lim * (2.0f * u - 1.0f);
}

// Minibatch gather: sample r of the batch is idx = (start + r) * 7919 + epoch * 104729 (mod N).
__global__ void k_mlp_batch(int32_t N, int32_t start, int32_t count, int32_t epoch, const float* __restrict__ x,
                            const float* __restrict__ t, float* __restrict__ xb, float* __restrict__ tb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= count) return;
  const int64_t i = (((int64_t)(start + r) * 7919 + (int64_t)epoch * 104729) % N + N) % N;
  for (int k = 0; k < kFeatures; ++k) xb[(size_t)r * kFeatures + k] = x[(size_t)i * kFeatures + k];
  for (int o = 0; o < kOutputs; ++o) tb[(size_t)r * kOutputs + o] = t[(size_t)i * kOutputs + o];
}

}  // namespace

}  // namespace nolsm

// ==================================================================================== host side

struct nolsm_mlp {
  float* params = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  double* loss = nullptr;
  // per-sample workspaces for up to cap samples
  float* act = nullptr; float* dz = nullptr; float* dy = nullptr; float* y = nullptr; float* part = nullptr;
  float* xb = nullptr; float* tb = nullptr;
  int32_t cap = 0;
  int32_t step = 0;   // Adam steps taken
  ~nolsm_mlp() {
    for (void* p : {(void*)params, (void*)grad, (void*)m, (void*)v, (void*)loss, (void*)act, (void*)dz, (void*)dy,
                    (void*)y, (void*)part, (void*)xb, (void*)tb})
      if (p) cudaFree(p);
  }
};

namespace nolsm {

namespace {

size_t mlp_smem_bytes() { return sizeof(float) * kMlpSmemFloats + 64; }

nolsm_status mlp_reserve(nolsm_mlp* m, int32_t B) {
  if (B <= m->cap) return NOLSM_OK;
  for (float** p : {&m->act, &m->dz, &m->dy, &m->y, &m->part, &m->xb, &m->tb}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  m->cap = 0;
  const size_t b = (size_t)B, chunks = (b + kChunk - 1) / kChunk;
  NOLSM_CUDA_TRY(cudaMalloc(&m->act, sizeof(float) * b * 2 * kWidth));
  NOLSM_CUDA_TRY(cudaMalloc(&m->dz, sizeof(float) * b * 2 * kWidth));
  NOLSM_CUDA_TRY(cudaMalloc(&m->dy, sizeof(float) * b * kOutputs));
  NOLSM_CUDA_TRY(cudaMalloc(&m->y, sizeof(float) * b * kOutputs));
  NOLSM_CUDA_TRY(cudaMalloc(&m->part, sizeof(float) * chunks * kParams));
  NOLSM_CUDA_TRY(cudaMalloc(&m->xb, sizeof(float) * b * kFeatures));
  NOLSM_CUDA_TRY(cudaMalloc(&m->tb, sizeof(float) * b * kOutputs));
  m->cap = B;
  return NOLSM_OK;
}

int mlp_grid(int32_t B) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return std::max(1, std::min((B + 7) / 8, 3 * sms));
}

nolsm_status mlp_set_smem() {
  static bool done = false;
  if (!done) {
    NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes()));
    NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes()));
    done = true;
  }
  return NOLSM_OK;
}

// forward (activations kept) + backward + weight gradients into m->grad; loss accumulated into m->loss
nolsm_status mlp_grad(nolsm_mlp* m, int32_t B, const float* x, const float* t, cudaStream_t st) {
  NOLSM_TRY(mlp_set_smem());
  k_mlp_forward<<<mlp_grid(B), kMlpThreads, mlp_smem_bytes(), st>>>(m->params, B, x, m->y, m->act);
  NOLSM_LAUNCH_CHECK();
  k_mlp_backward<<<mlp_grid(B), kMlpThreads, mlp_smem_bytes(), st>>>(m->params, B, m->act, m->y, t, m->dz, m->dy,
                                                                       m->loss);
  NOLSM_LAUNCH_CHECK();
  const int chunks = (B + kChunk - 1) / kChunk;
  k_mlp_wgrad<<<chunks, 256, 0, st>>>(B, x, m->act, m->dz, m->dy, m->part);
  NOLSM_LAUNCH_CHECK();
  k_mlp_reduce<<<(kParams + 255) / 256, 256, 0, st>>>(chunks, m->part, m->grad);
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}

nolsm_status mlp_adam(nolsm_mlp* m, float lr, cudaStream_t st) {
  m->step += 1;
  k_mlp_adam<<<(kParams + 255) / 256, 256, 0, st>>>(m->params, m->grad, m->m, m->v, m->step, lr, 0.9f, 0.999f, 1e-8f);
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}

nolsm_status ensure_buf(nolsm_plan* plan, DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return NOLSM_OK;
  dev_free(plan, b);
  return dev_alloc(plan, b, bytes);
}

}  // namespace

nolsm_status power_bounds(nolsm_plan* plan, int cls, int64_t j0, int64_t j1, const int32_t* list, int32_t count,
                          cudaStream_t st) {
  const size_t n = (size_t)plan->n_mol;
  NOLSM_TRY(ensure_buf(plan, plan->lam_p, sizeof(double) * 2 * n));
  if (plan->pow_done.size() != n || plan->pow_cls != cls) {
    plan->pow_done.assign(n, 0);
    plan->pow_cls = cls;
  }
  int64_t a = j0, b = j1;
  if (!list) {   // skip what is cached
    while (a < b && plan->pow_done[a]) ++a;
    while (b > a && plan->pow_done[b - 1]) --b;
    if (a >= b) return NOLSM_OK;
  }
  PowArgs g;
  g.j0 = (int32_t)a;
  g.list = list;
  g.sub_n = plan->sub_n.as<int32_t>(); g.a_off = plan->a_off.as<int64_t>();
  g.prep_status = plan->prep_status.as<int32_t>();
  g.lam = plan->lam.as<double>(); g.lam_p = plan->lam_p.as<double>();
  g.iters = 30;
  const int blocks = list ? count : (int)(b - a);
  if (blocks <= 0) return NOLSM_OK;
  const size_t smem = sizeof(float) * 4 * (size_t)std::max(plan->max_n, 1);
  if (cls == kPrepFP64) {
    NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_power_bounds<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_power_bounds<double><<<blocks, kPowThreads, smem, st>>>(g, plan->prep64.A.as<double>());
  } else {
    NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_power_bounds<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_power_bounds<float><<<blocks, kPowThreads, smem, st>>>(g, prepared(plan, cls).A.as<float>());
  }
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 1;
  if (!list)
    for (int64_t J = a; J < b; ++J) plan->pow_done[J] = 1;
  return NOLSM_OK;
}

nolsm_status features(nolsm_plan* plan, double mu, int64_t j0, int64_t j1, cudaStream_t st) {
  const size_t n = (size_t)plan->n_mol;
  NOLSM_TRY(ensure_buf(plan, plan->feat, sizeof(float) * kFeatures * n));
  if (!plan->onsite_done) {   // per molecule of the input system (a grouped plan has fewer submatrices)
    const int32_t nm = plan->sys.n_mol;
    NOLSM_TRY(ensure_buf(plan, plan->onsite, sizeof(double) * 2 * (size_t)nm));
    if (plan->gen)
      k_onsite_model<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(nm, plan->onsite_off.as<int64_t>(),
                                                                   plan->model.onsite, plan->onsite.as<double>());
    else
      k_onsite<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(nm, plan->sys.nbf, plan->sys.h_row_ptr,
                                                             plan->sys.h_col_idx, plan->h_blk_off.as<int64_t>(),
                                                             plan->sys.h_vals, plan->onsite.as<double>());
    NOLSM_LAUNCH_CHECK();
    plan->stats.launches += 1;
    plan->onsite_done = true;
  }
  FeatArgs g;
  g.j0 = (int32_t)j0; g.j1 = (int32_t)j1;
  g.sub_n = plan->sub_n.as<int32_t>(); g.nbf = plan->sys.nbf;
  g.nb_ptr = plan->nb_ptr.as<int32_t>(); g.nb_idx = plan->nb_idx.as<int32_t>();
  g.lam = plan->lam.as<double>(); g.onsite = plan->onsite.as<double>();
  g.mu = mu;
  g.feat = plan->feat.as<float>();
  k_features<<<(unsigned)((j1 - j0 + 255) / 256), 256, 0, st>>>(g);
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 1;
  return NOLSM_OK;
}

nolsm_status mlp_bounds(nolsm_plan* plan, int64_t j0, int64_t j1, int32_t max_iter, cudaStream_t st) {
  if (!plan->mlp) {
    set_error("bound source NOLSM_BOUND_MLP needs a network (nolsm_plan_set_mlp)");
    return NOLSM_ERR_ARG;
  }
  const size_t n = (size_t)plan->n_mol;
  NOLSM_TRY(ensure_buf(plan, plan->mlp_y, sizeof(float) * kOutputs * n));
  NOLSM_TRY(ensure_buf(plan, plan->lam_m, sizeof(double) * 2 * n));
  NOLSM_TRY(ensure_buf(plan, plan->budget, sizeof(int32_t) * n));
  NOLSM_TRY(mlp_set_smem());
  const int32_t B = (int32_t)(j1 - j0);
  k_mlp_forward<<<mlp_grid(B), kMlpThreads, mlp_smem_bytes(), st>>>(
      plan->mlp->params, B, plan->feat.as<float>() + (size_t)j0 * kFeatures, plan->mlp_y.as<float>() + (size_t)j0 * kOutputs,
      nullptr);
  NOLSM_LAUNCH_CHECK();
  k_mlp_bounds<<<(unsigned)((B + 255) / 256), 256, 0, st>>>((int32_t)j0, (int32_t)j1, plan->mlp_y.as<float>(),
                                                             plan->lam.as<double>(), max_iter, plan->lam_m.as<double>(),
                                                             plan->budget.as<int32_t>());
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 2;
  return NOLSM_OK;
}

nolsm_status training_targets(nolsm_plan* plan, int64_t j0, int64_t j1, float* t, cudaStream_t st) {
  k_targets<<<(unsigned)((j1 - j0 + 255) / 256), 256, 0, st>>>((int32_t)j0, (int32_t)j1, plan->lam_p.as<double>(),
                                                                plan->iters.as<int32_t>(), t);
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 1;
  return NOLSM_OK;
}

nolsm_status failed_list(nolsm_plan* plan, int64_t j0, int64_t j1, cudaStream_t st, int32_t* count) {
  const size_t n = (size_t)plan->n_mol;
  NOLSM_TRY(ensure_buf(plan, plan->rerun, sizeof(int32_t) * (n + 1)));
  int32_t* list = plan->rerun.as<int32_t>();
  NOLSM_CUDA_TRY(cudaMemsetAsync(list + n, 0, sizeof(int32_t), st));
  k_failed<<<(unsigned)((j1 - j0 + 255) / 256), 256, 0, st>>>((int32_t)j0, (int32_t)j1, plan->status.as<int32_t>(),
                                                               list, list + n);
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 1;
  NOLSM_CUDA_TRY(cudaMemcpyAsync(count, list + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  return NOLSM_OK;
}

}  // namespace nolsm

using namespace nolsm;

extern "C" {

int32_t nolsm_mlp_param_count(void) { return kParams; }

nolsm_status nolsm_mlp_create(uint64_t seed, nolsm_stream_t stream, nolsm_mlp** out) {
  if (!out) { set_error("nolsm_mlp_create: NULL out"); return NOLSM_ERR_ARG; }
  *out = nullptr;
  nolsm_mlp* m = new nolsm_mlp();
  cudaStream_t st = (cudaStream_t)stream;
  auto fail = [&](nolsm_status s) { delete m; return s; };
  if (cudaMalloc(&m->params, sizeof(float) * kParams) != cudaSuccess ||
      cudaMalloc(&m->grad, sizeof(float) * kParams) != cudaSuccess ||
      cudaMalloc(&m->m, sizeof(float) * kParams) != cudaSuccess ||
      cudaMalloc(&m->v, sizeof(float) * kParams) != cudaSuccess || cudaMalloc(&m->loss, sizeof(double)) != cudaSuccess) {
    set_error("nolsm_mlp_create: device allocation failed");
    return fail(NOLSM_ERR_OOM);
  }
  k_mlp_init<<<(kParams + 255) / 256, 256, 0, st>>>(m->params, seed);
  if (cudaGetLastError() != cudaSuccess || cudaMemsetAsync(m->m, 0, sizeof(float) * kParams, st) != cudaSuccess ||
      cudaMemsetAsync(m->v, 0, sizeof(float) * kParams, st) != cudaSuccess ||
      cudaMemsetAsync(m->grad, 0, sizeof(float) * kParams, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("nolsm_mlp_create: initialisation failed");
    return fail(NOLSM_ERR_CUDA);
  }
  *out = m;
  return NOLSM_OK;
}

void nolsm_mlp_destroy(nolsm_mlp* mlp) { delete mlp; }

nolsm_status nolsm_mlp_get_params(const nolsm_mlp* mlp, float* host_params) {
  if (!mlp || !host_params) { set_error("nolsm_mlp_get_params: NULL argument"); return NOLSM_ERR_ARG; }
  NOLSM_CUDA_TRY(cudaMemcpy(host_params, mlp->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
  return NOLSM_OK;
}

nolsm_status nolsm_mlp_set_params(nolsm_mlp* mlp, const float* host_params) {
  if (!mlp || !host_params) { set_error("nolsm_mlp_set_params: NULL argument"); return NOLSM_ERR_ARG; }
  NOLSM_CUDA_TRY(cudaMemcpy(mlp->params, host_params, sizeof(float) * kParams, cudaMemcpyHostToDevice));
  NOLSM_CUDA_TRY(cudaMemset(mlp->m, 0, sizeof(float) * kParams));
  NOLSM_CUDA_TRY(cudaMemset(mlp->v, 0, sizeof(float) * kParams));
  mlp->step = 0;
  return NOLSM_OK;
}

nolsm_status nolsm_mlp_forward(nolsm_mlp* mlp, int32_t B, const float* x, float* y, nolsm_stream_t stream) {
  if (!mlp || !x || !y || B < 1) { set_error("nolsm_mlp_forward: invalid argument"); return NOLSM_ERR_ARG; }
  NOLSM_TRY(mlp_set_smem());
  k_mlp_forward<<<mlp_grid(B), kMlpThreads, mlp_smem_bytes(), (cudaStream_t)stream>>>(mlp->params, B, x, y, nullptr);
  NOLSM_LAUNCH_CHECK();
  NOLSM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return NOLSM_OK;
}

nolsm_status nolsm_mlp_gradient(nolsm_mlp* mlp, int32_t B, const float* x, const float* t, nolsm_stream_t stream,
                                float* grad_host, double* loss) {
  if (!mlp || !x || !t || B < 1) { set_error("nolsm_mlp_gradient: invalid argument"); return NOLSM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  NOLSM_TRY(mlp_reserve(mlp, B));
  NOLSM_CUDA_TRY(cudaMemsetAsync(mlp->loss, 0, sizeof(double), st));
  NOLSM_TRY(mlp_grad(mlp, B, x, t, st));
  if (grad_host)
    NOLSM_CUDA_TRY(cudaMemcpyAsync(grad_host, mlp->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, st));
  double l = 0.0;
  NOLSM_CUDA_TRY(cudaMemcpyAsync(&l, mlp->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return NOLSM_OK;
}

nolsm_status nolsm_mlp_adam_step(nolsm_mlp* mlp, float lr, nolsm_stream_t stream) {
  if (!mlp || !(lr > 0.0f)) { set_error("nolsm_mlp_adam_step: invalid argument"); return NOLSM_ERR_ARG; }
  NOLSM_TRY(mlp_adam(mlp, lr, (cudaStream_t)stream));
  NOLSM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return NOLSM_OK;
}

nolsm_status nolsm_mlp_train(nolsm_mlp* mlp, int32_t N, const float* x, const float* t, int32_t epochs,
                             int32_t batch, float lr, nolsm_stream_t stream, double* epoch_loss) {
  if (!mlp || !x || !t || N < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f)) {
    set_error("nolsm_mlp_train: invalid argument");
    return NOLSM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t bs = std::min(batch, N);
  NOLSM_TRY(mlp_reserve(mlp, bs));
  const int32_t steps = (N + bs - 1) / bs;
  for (int32_t e = 0; e < epochs; ++e) {
    NOLSM_CUDA_TRY(cudaMemsetAsync(mlp->loss, 0, sizeof(double), st));
    for (int32_t s = 0; s < steps; ++s) {
      const int32_t start = s * bs, cnt = std::min(bs, N - start);
      k_mlp_batch<<<(cnt + 255) / 256, 256, 0, st>>>(N, start, cnt, e, x, t, mlp->xb, mlp->tb);
      NOLSM_LAUNCH_CHECK();
      NOLSM_TRY(mlp_grad(mlp, cnt, mlp->xb, mlp->tb, st));
      NOLSM_TRY(mlp_adam(mlp, lr, st));
    }
    if (epoch_loss) {
      double l = 0.0;
      NOLSM_CUDA_TRY(cudaMemcpyAsync(&l, mlp->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
      NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
      epoch_loss[e] = l / steps;
    }
  }
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  return NOLSM_OK;
}

}  // extern "C"
