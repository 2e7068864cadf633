// Geometry preparation (a1 gather, a2 FP64 Cholesky, a3 A = T_J(S)^-1 T_J(H0) and the centre
// columns of T_J(S)^-1), the plain FP64 sign iteration (a4-a7), the trace reductions and the
// write-back (a8). The FP64 sign iteration is the reference GPU path; the tensor-core paths reuse
// everything here except the sign iteration itself.
#include <algorithm>
#include <cmath>

#include "nolsm_internal.cuh"
#include "prep.cuh"
#include "tc_path.cuh"

namespace nolsm {

namespace {

__device__ __forceinline__ int owner_of(const int32_t* __restrict__ nb_ptr, int n_mol, int64_t p) {
  // largest J with nb_ptr[J] <= p
  int lo = 0, hi = n_mol;  // invariant: nb_ptr[lo] <= p < nb_ptr[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)nb_ptr[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int find_sorted(const int32_t* __restrict__ a, int lo, int hi, int32_t key) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid;
  }
  return -1;
}

// ------------------------------------------------------------------------------------ a1: gather
// One warp per row band (J, a): rows of molecule I_a inside T_J, eight bands per block. For every
// molecule I_c of N(J) the block (I_a, I_c) of S and of H0 is looked up by binary search in block row
// I_a; the band is written in full (zeros where no block is stored), so the workspace needs no clearing.
// Also writes the centre columns of T_J(S) and T_J(H0) into the geometry caches.
struct GatherArgs {
  int32_t n_mol;
  const int32_t* nbf;   // per molecule
  const int32_t* sub_b; // centre columns per submatrix
  const int32_t* srp; const int32_t* sci; const int64_t* soff; const double* sval;
  const int32_t* hrp; const int32_t* hci; const int64_t* hoff; const double* hval;
  const int32_t* nb_ptr; const int32_t* nb_idx; const int32_t* nb_off;
  const int32_t* sub_n; const int32_t* sub_c0;
  const int64_t* a_off; const int64_t* c_off;
  int64_t a_base;       // a_off of the chunk's first submatrix
  int64_t chunk_n2;     // sum of n^2 over the chunk (offset of the T(H0) half)
  int64_t p0, p1;       // row bands [p0, p1) of the chunk
  int32_t max_nq;       // largest |N(J)|: each warp's lookup tables hold 3 max_nq ints
  double* ws;           // [2*chunk_n2]
  double* Sc; double* Hc;
  // elements generated from the geometry (gen != 0) instead of read from sval / hval
  int gen;
  const double* pos; double cell[3]; const double* onsite; const int64_t* onsite_off;
  double s_exp, hop, hop_len, aniso; const double* dirs;
};

// The synthetic element model of nolsm_plan_set_elements for the block (Ia, Ic), Ia != Ic: the isotropic
// values of S and H0 and the unit vector from Ia to Ic. Every product and sum is rounded on its own (no
// contraction into FMAs), in the order the model states them.
struct BlockModel { double s, h, ux, uy, uz; };
__device__ __forceinline__ BlockModel block_model(const GatherArgs& g, int Ia, int Ic, int ba, int bc) {
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double v = __dsub_rn(g.pos[3 * Ic + k], g.pos[3 * Ia + k]);
    d[k] = __dsub_rn(v, __dmul_rn(g.cell[k], rint(__ddiv_rn(v, g.cell[k]))));   // minimum image
  }
  const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2])));
  const double inv = __ddiv_rn(1.0, sqrt((double)(ba * bc)));
  BlockModel m;
  m.s = __dmul_rn(inv, exp(__dmul_rn(__dmul_rn(-g.s_exp, r), r)));
  m.h = __dmul_rn(inv, __dmul_rn(g.hop, exp(__ddiv_rn(-r, g.hop_len))));
  m.ux = __ddiv_rn(d[0], r);
  m.uy = __ddiv_rn(d[1], r);
  m.uz = __ddiv_rn(d[2], r);
  return m;
}

// the direction modulation 1 + aniso (u . dirs[k][a] - u . dirs[k][c])
__device__ __forceinline__ double aniso_factor(const GatherArgs& g, int k, const BlockModel& m, int a, int c) {
  const double* da = g.dirs + (k * 64 + a) * 3;
  const double* dc = g.dirs + (k * 64 + c) * 3;
  const double ua = __dadd_rn(__dadd_rn(__dmul_rn(m.ux, da[0]), __dmul_rn(m.uy, da[1])), __dmul_rn(m.uz, da[2]));
  const double uc = __dadd_rn(__dadd_rn(__dmul_rn(m.ux, dc[0]), __dmul_rn(m.uy, dc[1])), __dmul_rn(m.uz, dc[2]));
  return __dadd_rn(1.0, __dmul_rn(g.aniso, __dsub_rn(ua, uc)));
}

constexpr int kGatherWarps = 8;
constexpr int kGatherTableBytes = 32;   // per block column of a band: two int64 offsets, three int32, padding

__global__ void __launch_bounds__(32 * kGatherWarps) k_gather(GatherArgs g) {
  extern __shared__ __align__(8) unsigned char gsm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t p = g.p0 + (int64_t)blockIdx.x * kGatherWarps + w;
  if (p >= g.p1) return;   // whole warps only; no block-wide barrier follows
  // this warp's tables, one entry per block column c of the band (32 bytes each): the offsets of block
  // (Ia, Ic) in the stored S and H0 values (-1: no block), its first column, its width and Ic; the block
  // models of generated elements follow every warp's tables
  int64_t* sbase = reinterpret_cast<int64_t*>(gsm + (size_t)w * kGatherTableBytes * g.max_nq);
  int64_t* hbase = sbase + g.max_nq;
  int32_t* coff = reinterpret_cast<int32_t*>(hbase + g.max_nq);
  int32_t* bcs = coff + g.max_nq;
  int32_t* mol = bcs + g.max_nq;
  BlockModel* bm = reinterpret_cast<BlockModel*>(gsm + (size_t)kGatherWarps * kGatherTableBytes * g.max_nq) +
                   w * g.max_nq;
  const int J = owner_of(g.nb_ptr, g.n_mol, p);
  const int q0 = g.nb_ptr[J], nq = g.nb_ptr[J + 1] - q0;
  const int Ia = g.nb_idx[p];
  const int ba = g.nbf[Ia];
  const int offa = g.nb_off[p];
  const int n = g.sub_n[J];
  for (int c = lane; c < nq; c += 32) {
    const int32_t Ic = g.nb_idx[q0 + c];
    const int ss = find_sorted(g.sci, g.srp[Ia], g.srp[Ia + 1], Ic);
    const int hs = find_sorted(g.hci, g.hrp[Ia], g.hrp[Ia + 1], Ic);
    sbase[c] = ss < 0 ? -1 : (g.gen ? 0 : g.soff[ss]);
    hbase[c] = hs < 0 ? -1 : (g.gen ? 0 : g.hoff[hs]);
    coff[c] = g.nb_off[q0 + c];
    bcs[c] = g.nbf[Ic];
    mol[c] = Ic;
    if (g.gen && Ic != Ia) bm[c] = block_model(g, Ia, Ic, ba, g.nbf[Ic]);
  }
  __syncwarp();
  const int c0 = g.sub_c0[J];
  const int bJ = g.sub_b[J];
  double* TS = g.ws + (g.a_off[J] - g.a_base);
  double* TH = TS + g.chunk_n2;
  double* Sc = g.Sc + g.c_off[J];
  double* Hc = g.Hc + g.c_off[J];
  int c = 0;   // block column of col; columns advance by 32, blocks by at least one function
  for (int col = lane; col < n; col += 32) {
    while (c + 1 < nq && coff[c + 1] <= col) ++c;
    const int bc = bcs[c], cc = col - coff[c];
    const int64_t sb = sbase[c], hb = hbase[c];
    const bool intra = mol[c] == Ia;
    const bool centre = col >= c0 && col < c0 + bJ;
    // the column's ba rows, four at a time: their loads issued together, then their stores
    for (int r0 = 0; r0 < ba; r0 += 4) {
      double vs[4], vh[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + u;
        vs[u] = vh[u] = 0.0;
        if (r >= ba) continue;
        if (!g.gen) {
          if (sb >= 0) vs[u] = __ldg(g.sval + sb + r * bc + cc);
          if (hb >= 0) vh[u] = __ldg(g.hval + hb + r * bc + cc);
        } else if (intra) {   // intra-molecular: identity and the on-site energies
          vs[u] = (sb >= 0 && r == cc) ? 1.0 : 0.0;
          vh[u] = (hb >= 0 && r == cc) ? g.onsite[g.onsite_off[Ia] + r] : 0.0;
        } else {
          const BlockModel& m = bm[c];
          vs[u] = sb >= 0 ? (g.aniso != 0.0 ? __dmul_rn(m.s, aniso_factor(g, 0, m, r, cc)) : m.s) : 0.0;
          vh[u] = hb >= 0 ? (g.aniso != 0.0 ? __dmul_rn(m.h, aniso_factor(g, 1, m, r, cc)) : m.h) : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + u;
        if (r >= ba) break;
        const int64_t at = (int64_t)(offa + r) * n + col;
        TS[at] = vs[u];
        TH[at] = vh[u];
        if (centre) {
          Sc[(int64_t)(offa + r) * bJ + (col - c0)] = vs[u];
          Hc[(int64_t)(offa + r) * bJ + (col - c0)] = vh[u];
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------ FP64 GEMM in one CTA
// C = A B for n x n row-major matrices (leading dimension n), 256 threads, 64 x 64 output tiles, each
// thread 4 x 4 outputs at rows ty + 16 i and columns tx + 16 j; epi(i, j, acc) consumes each output.
constexpr int kTile = 64, kKc = 16;

template <class Epi>
__device__ __forceinline__ void cta_dgemm(const double* __restrict__ A, const double* __restrict__ B, int n,
                                          double (*As)[kTile + 1], double (*Bs)[kTile + 1], Epi&& epi) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int tm = 0; tm < n; tm += kTile) {
    for (int tn = 0; tn < n; tn += kTile) {
      double acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
      for (int k0 = 0; k0 < n; k0 += kKc) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int idx = tid + 256 * q;
          const int m = idx >> 4, k = idx & 15;  // A tile: 64 rows x 16 k
          const int gm = tm + m, gk = k0 + k;
          As[k][m] = (gm < n && gk < n) ? A[(int64_t)gm * n + gk] : 0.0;
          const int kb = idx >> 6, nn = idx & 63;  // B tile: 16 k x 64 cols
          const int gk2 = k0 + kb, gn = tn + nn;
          Bs[kb][nn] = (gk2 < n && gn < n) ? B[(int64_t)gk2 * n + gn] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKc; ++k) {
          double a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gi = tm + ty + 16 * i, gj = tn + tx + 16 * j;
          if (gi < n && gj < n) epi(gi, gj, acc[i][j]);
        }
    }
  }
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// ------------------------------------------------------------------------------------ a4-a7 (FP64)
struct NsArgs {
  int32_t j0, j1;
  const int32_t* sub_n; const int32_t* nbf;
  const int64_t* a_off; const int64_t* c_off;
  const double* A; const double* Q; const double* Sc; const double* Hc; const double* lam;
  const double* lam_g;         // Gershgorin interval (the scale never drops below its alpha / 1.7)
  const int32_t* prep_status;
  double mu, tol;
  int32_t max_iter;
  const int32_t* budget;       // per-submatrix step cap (nullable)
  const int32_t* list;         // work list (nullable: [j0, j1))
  int32_t count;
  double* ws; int64_t slot_elems;
  int32_t* next;               // work counter
  double* Dc; double* tS; double* tH; int32_t* iters; int32_t* status; int32_t* rsteps;
  int32_t* nbelow;             // eigenvalues below mu: (n - Tr X) / 2
};

__global__ void __launch_bounds__(256) k_ns_fp64(NsArgs g) {
  __shared__ double As[kKc][kTile + 1];
  __shared__ double Bs[kKc][kTile + 1];
  __shared__ double red[33];
  __shared__ int job;
  double* X = g.ws + (int64_t)blockIdx.x * 3 * g.slot_elems;
  double* T = X + g.slot_elems;
  double* Xn = T + g.slot_elems;
  for (;;) {
    if (threadIdx.x == 0) {
      const int k = atomicAdd(g.next, 1);
      job = g.list ? (k < g.count ? g.list[k] : -1) : (g.j0 + k < g.j1 ? g.j0 + k : -1);
    }
    __syncthreads();
    const int J = job;
    __syncthreads();
    if (J < 0) break;
    if (g.prep_status[J] != kSubOk) {
      if (threadIdx.x == 0) {
        g.status[J] = g.prep_status[J];
        g.iters[J] = 0;
        g.rsteps[J] = 0;
        g.tS[J] = 0.0;
        g.tH[J] = 0.0;
      }
      continue;
    }
    const int n = g.sub_n[J];
    const int64_t nn = (int64_t)n * n;
    const double* A = g.A + g.a_off[J];
    // a4: X_0 = (A - mu I) / alpha, alpha = max(hi - mu, mu - lo) from the interval of the bound source
    const double alpha = scale_alpha(g.lam, g.lam_g, J, g.mu);
    const double inv_alpha = 1.0 / alpha;
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
      X[e] = (A[e] - (i == j ? g.mu : 0.0)) * inv_alpha;
    }
    __syncthreads();
    // a5: X <- 1/2 X (3I - X^2) until the defect test passes
    int it = 0, st = kSubNotConv;
    double* x = X;
    double* xn = Xn;
    const int cap = g.budget ? min(g.max_iter, g.budget[J]) : g.max_iter;
    while (it < cap) {
      double part = 0.0;
      cta_dgemm(x, x, n, As, Bs, [&](int i, int j, double acc) {
        const double v = (i == j ? 1.0 : 0.0) - acc;   // (I - X^2)_ij
        part += v * v;
        T[(int64_t)i * n + j] = v + (i == j ? 2.0 : 0.0);  // 3I - X^2
      });
      const double defect = sqrt(block_sum(part, red) / n);
      cta_dgemm(x, T, n, As, Bs, [&](int i, int j, double acc) { xn[(int64_t)i * n + j] = 0.5 * acc; });
      __syncthreads();
      double* t = x; x = xn; xn = t;
      ++it;
      if (!isfinite(defect)) { st = kSubNonFinite; break; }
      if (defect <= g.tol) { st = kSubOk; break; }
    }
    // a7: centre columns of T_J(D) = 1/2 (I - X) T_J(S)^-1 and the partial traces
    const int b = g.nbf[J];
    const double* Q = g.Q + g.c_off[J];
    const double* Sc = g.Sc + g.c_off[J];
    const double* Hc = g.Hc + g.c_off[J];
    double* Dc = g.Dc + g.c_off[J];
    double ps = 0.0, ph = 0.0;
    for (int e = threadIdx.x; e < n * b; e += blockDim.x) {
      const int i = e / b, c = e - i * b;
      const double* xi = x + (int64_t)i * n;
      double s = 0.0;
      for (int k = 0; k < n; ++k) s = fma(xi[k], Q[(int64_t)k * b + c], s);
      const double d = 0.5 * (Q[e] - s);
      Dc[e] = d;
      ps += d * Sc[e];
      ph += d * Hc[e];
    }
    double px = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) px += x[(int64_t)i * n + i];
    const double ts = block_sum(ps, red);
    const double th = block_sum(ph, red);
    const double tx = block_sum(px, red);
    if (threadIdx.x == 0) {
      if (st == kSubOk && !(isfinite(ts) && isfinite(th))) st = kSubNonFinite;
      g.tS[J] = ts;
      g.tH[J] = th;
      g.iters[J] = it;
      g.rsteps[J] = 0;
      g.status[J] = st;
      g.nbelow[J] = (int32_t)lrint(0.5 * (n - tx));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------ reductions
// Sums of t_S and t_H over [j0, j1) in a fixed order (one block), the first failing submatrix, and
// the work counters: sum of steps n^3 (paper convention), of the tensor products' n^3 (x3 for split
// steps) on unpadded and padded shapes, and of steps.
__global__ void __launch_bounds__(256) k_reduce(int32_t j0, int32_t j1, const double* __restrict__ tS,
                                                const double* __restrict__ tH, const int32_t* __restrict__ status,
                                                const int32_t* __restrict__ iters, const int32_t* __restrict__ rsteps,
                                                const int32_t* __restrict__ sub_n, int terms_main,
                                                const int32_t* __restrict__ list, int32_t count, double* out) {
  __shared__ double red[33];
  __shared__ int first[256];
  double a = 0.0, b = 0.0, w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
  int f = INT32_MAX;
  for (int J = j0 + threadIdx.x; J < j1; J += blockDim.x) {
    a += tS[J];
    b += tH[J];
    if (status[J] != 0 && J < f) f = J;
  }
  // work counters over the submatrices this call solved (the list, else the whole range): submatrices
  // kept from an earlier solve are not counted again
  const int32_t m = list ? count : j1 - j0;
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    const int J = list ? list[e] : j0 + e;
    const double n = sub_n[J];
    const double n64 = (double)((sub_n[J] + 63) & ~63), R = (double)((sub_n[J] + 127) & ~127);
    const double prod = (double)terms_main * (iters[J] - rsteps[J]) + 3.0 * rsteps[J];
    w0 += iters[J] * n * n * n;
    w1 += prod * n * n * n;
    w2 += prod * R * n64 * n64;
    w3 += iters[J];
  }
  const double sa = block_sum(a, red);
  const double sb = block_sum(b, red);
  const double s0 = block_sum(w0, red);
  const double s1 = block_sum(w1, red);
  const double s2 = block_sum(w2, red);
  const double s3 = block_sum(w3, red);
  first[threadIdx.x] = f;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) first[threadIdx.x] = min(first[threadIdx.x], first[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sa;
    out[1] = sb;
    out[2] = first[0] == INT32_MAX ? -1.0 : (double)first[0];
    out[3] = first[0] == INT32_MAX ? 0.0 : (double)status[first[0]];
    out[4] = 4.0 * s0;
    out[5] = 4.0 * s1;
    out[6] = 4.0 * s2;
    out[7] = s3;
  }
}

// ------------------------------------------------------------------------------------ a8: write-back
// One warp per (J, I in N(J)): block (I, J) of D <- rows of I in the centre columns of T_J(D).
__global__ void __launch_bounds__(256) k_scatter(int32_t n_mol, int64_t p0, int64_t p1, const int32_t* __restrict__ nbf,
                                                 const int32_t* __restrict__ nb_ptr, const int32_t* __restrict__ nb_idx,
                                                 const int32_t* __restrict__ nb_off, const int32_t* __restrict__ d_slot,
                                                 const int64_t* __restrict__ d_blk_off,
                                                 const int64_t* __restrict__ c_off, const double* __restrict__ Dc,
                                                 double* __restrict__ D) {
  const int64_t p = p0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (p >= p1) return;
  const int J = owner_of(nb_ptr, n_mol, p);
  const int I = nb_idx[p];
  const int bI = nbf[I], bJ = nbf[J];
  const double* src = Dc + c_off[J] + (int64_t)nb_off[p] * bJ;
  double* dst = D + d_blk_off[d_slot[p]];
  for (int e = lane; e < bI * bJ; e += 32) dst[e] = src[e];  // both b_I x b_J row-major
}

}  // namespace

// ==================================================================================== host side

static nolsm_status ensure(nolsm_plan* plan, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return NOLSM_OK;
  dev_free(plan, b);
  return dev_alloc(plan, b, bytes);
}

// Stopping rule of the tensor-core inverse square root: the step whose ||I - Z_k Y_k||_F / sqrt(n) is below
// kNsInvTol is the last (the iteration converges quadratically, so its Z is about kNsInvTol^2 from the
// limit, below the three-term products' own rounding); a submatrix still above it after kNsInvMaxSteps
// steps is prepared with the FP64 factorisation.
constexpr float kNsInvTol = 1e-3f;
constexpr int kNsInvMaxSteps = 40;

nolsm_status prepare(nolsm_plan* plan, int64_t j0, int64_t j1, int cls, cudaStream_t st) {
  const bool keep_fp64_A = cls == kPrepFP64;
  const bool sym = cls == kPrepSym;
  Prepared& P = prepared(plan, cls);
  const int32_t n_mol = plan->n_mol;
  const size_t esz = keep_fp64_A ? sizeof(double) : sizeof(float);
  if (!P.A.p) {
    NOLSM_TRY(dev_alloc(plan, P.A, esz * (size_t)std::max<int64_t>(plan->h_a_off[n_mol], 1)));
    P.done.assign(n_mol, 0);
    P.fp64 = keep_fp64_A;
  }
  const int64_t nc = std::max<int64_t>(plan->h_c_off[n_mol], 1);
  if (!plan->Q.p) {
    NOLSM_TRY(dev_alloc(plan, plan->Q, sizeof(double) * nc));
    NOLSM_TRY(dev_alloc(plan, plan->Sc, sizeof(double) * nc));
    NOLSM_TRY(dev_alloc(plan, plan->Hc, sizeof(double) * nc));
    NOLSM_TRY(dev_alloc(plan, plan->lam, sizeof(double) * 2 * n_mol));
    NOLSM_TRY(dev_alloc(plan, plan->prep_status, sizeof(int32_t) * n_mol));
    NOLSM_CUDA_TRY(cudaMemsetAsync(plan->prep_status.p, 0, sizeof(int32_t) * n_mol, st));
  }
  const bool ratio = !keep_fp64_A && !sym;   // the tensor-core classes record their cond(T_J(S)) estimate
  if (ratio && !P.cond.p) {
    NOLSM_TRY(dev_alloc(plan, P.cond, sizeof(float) * (size_t)std::max(n_mol, 1)));
    P.h_cond.assign((size_t)n_mol, 0.0f);
  }
  bool any_chunk = false;
  if (sym && !plan->Lsym.p) {
    NOLSM_TRY(dev_alloc(plan, plan->Lsym, sizeof(float) * (size_t)std::max<int64_t>(plan->h_a_off[n_mol], 1)));
    NOLSM_TRY(dev_alloc(plan, plan->Wc, sizeof(double) * nc));
  }
  int max_nq = 1;
  for (int64_t J = j0; J < j1; ++J) max_nq = std::max(max_nq, plan->h_nb_ptr[J + 1] - plan->h_nb_ptr[J]);
  const int64_t budget = (int64_t)1 << 34;  // bytes of gathered T_J(S), T_J(H0) per chunk (16 GB of the 288)
  int64_t J = j0;
  while (J < j1) {
    while (J < j1 && P.done[J]) ++J;
    if (J >= j1) break;
    int64_t e = J;
    while (e < j1 && !P.done[e] &&
           (e == J || 2 * 8 * (plan->h_a_off[e + 1] - plan->h_a_off[J]) <= budget))
      ++e;
    const int64_t n2 = plan->h_a_off[e] - plan->h_a_off[J];
    NOLSM_TRY(ensure(plan, plan->ws_dense, sizeof(double) * 2 * (size_t)n2));
    GatherArgs g{};
    g.n_mol = n_mol;
    g.nbf = plan->sys.nbf;
    g.sub_b = plan->sub_b.as<int32_t>();
    g.srp = plan->sys.s_row_ptr; g.sci = plan->sys.s_col_idx; g.soff = plan->s_blk_off.as<int64_t>();
    g.sval = plan->sys.s_vals;
    g.hrp = plan->sys.h_row_ptr; g.hci = plan->sys.h_col_idx; g.hoff = plan->h_blk_off.as<int64_t>();
    g.hval = plan->sys.h_vals;
    g.nb_ptr = plan->nb_ptr.as<int32_t>(); g.nb_idx = plan->nb_idx.as<int32_t>(); g.nb_off = plan->nb_off.as<int32_t>();
    g.sub_n = plan->sub_n.as<int32_t>(); g.sub_c0 = plan->sub_c0.as<int32_t>();
    g.a_off = plan->a_off.as<int64_t>(); g.c_off = plan->c_off.as<int64_t>();
    g.a_base = plan->h_a_off[J];
    g.chunk_n2 = n2;
    g.p0 = plan->h_nb_ptr[J];
    g.ws = plan->ws_dense.as<double>();
    g.Sc = plan->Sc.as<double>(); g.Hc = plan->Hc.as<double>();
    const int64_t bands = plan->h_nb_ptr[e] - plan->h_nb_ptr[J];
    g.p1 = plan->h_nb_ptr[e];
    g.max_nq = max_nq;
    g.gen = plan->gen ? 1 : 0;
    if (plan->gen) {
      const nolsm_element_model& m = plan->model;
      g.pos = m.pos; g.cell[0] = m.cell[0]; g.cell[1] = m.cell[1]; g.cell[2] = m.cell[2];
      g.onsite = m.onsite; g.onsite_off = plan->onsite_off.as<int64_t>();
      g.s_exp = m.s_exp; g.hop = m.hop; g.hop_len = m.hop_len; g.aniso = m.aniso; g.dirs = m.dirs;
    } else if (!plan->sys.s_vals || !plan->sys.h_vals) {
      set_error("the plan has neither element values nor an element model (nolsm_plan_set_elements)");
      return NOLSM_ERR_ARG;
    }
    pmark(plan, st);
    const size_t gsm = (size_t)kGatherTableBytes * kGatherWarps * max_nq +
                       (plan->gen ? sizeof(BlockModel) * kGatherWarps * (size_t)max_nq : 0);
    if (gsm > 48 * 1024) NOLSM_CUDA_TRY(cudaFuncSetAttribute(k_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    k_gather<<<(unsigned)((bands + kGatherWarps - 1) / kGatherWarps), 32 * kGatherWarps, gsm, st>>>(g);
    NOLSM_LAUNCH_CHECK();
    pmark(plan, st);
    PrepArgs pa;
    any_chunk = true;
    if (ratio) {   // a submatrix whose FP32 preparation fails keeps this huge estimate (bytes 0x7F: about 3.4e38)
      pa.cond = P.cond.as<float>();
      NOLSM_CUDA_TRY(cudaMemsetAsync(pa.cond + J, 0x7F, sizeof(float) * (size_t)(e - J), st));
    }
    pa.j0 = (int32_t)J;
    pa.sub_n = plan->sub_n.as<int32_t>(); pa.sub_c0 = plan->sub_c0.as<int32_t>(); pa.nbf = plan->sub_b.as<int32_t>();
    pa.a_off = plan->a_off.as<int64_t>(); pa.c_off = plan->c_off.as<int64_t>();
    pa.a_base = g.a_base; pa.chunk_n2 = n2; pa.ws = g.ws;
    pa.Q = plan->Q.as<double>(); pa.lam = plan->lam.as<double>(); pa.prep_status = plan->prep_status.as<int32_t>();
    int chunk_max_n = 1;
    for (int64_t k = J; k < e; ++k) chunk_max_n = std::max(chunk_max_n, plan->h_sub_n[k]);
    if (keep_fp64_A) {
      NOLSM_TRY(launch_prepare(pa, (int)(e - J), chunk_max_n, true, P.A.p, st));
      plan->stats.launches += 2;
    } else if (cls == kPrepNS) {
      // the coupled Newton-Schulz inverse square root on the tensor cores (A_J and X = T_J(S)^-1 in FP32),
      // then the refinement of the centre columns of T_J(S)^-1 with X, then the FP64 preparation of what
      // either of them flagged
      const int64_t nbc = plan->h_c_off[e] - plan->h_c_off[J];
      NOLSM_TRY(ensure(plan, plan->ws_refine, (sizeof(double) + sizeof(float)) * (size_t)std::max<int64_t>(nbc, 1)));
      NOLSM_TRY(ensure(plan, plan->ws_l32, sizeof(float) * (size_t)n2));
      std::vector<int32_t> ord((size_t)(e - J));
      for (int64_t k = J; k < e; ++k) ord[(size_t)(k - J)] = (int32_t)k;
      std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return plan->h_sub_n[a] > plan->h_sub_n[b]; });
      NOLSM_TRY(ensure(plan, plan->prep_order, sizeof(int32_t) * ord.size()));
      NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->prep_order.p, ord.data(), sizeof(int32_t) * ord.size(),
                                     cudaMemcpyHostToDevice, st));
      NOLSM_CUDA_TRY(cudaStreamSynchronize(st));   // ord is a host temporary
      NsInvArgs ia;
      ia.order = plan->prep_order.as<int32_t>();
      ia.count = (int32_t)(e - J);
      ia.n_large = 0;
      while (ia.n_large < ia.count && plan->h_sub_n[ord[(size_t)ia.n_large]] > 192) ++ia.n_large;
      ia.max_n = chunk_max_n;
      ia.ws = g.ws;
      ia.a_base = g.a_base;
      ia.chunk_n2 = n2;
      ia.Aout = P.A.as<float>();
      ia.Xout = plan->ws_l32.as<float>();
      ia.prep_out = plan->prep_status.as<int32_t>();
      ia.tol_inv = kNsInvTol;
      ia.max_inv = kNsInvMaxSteps;
      tmark(plan, st);
      NOLSM_TRY(launch_ns_inverse(plan, ia, st));
      tmark(plan, st);
      pa.order = ia.order;
      pa.L32 = plan->ws_l32.as<float>();
      pa.c_base = plan->h_c_off[J];
      pa.Qp = plan->ws_refine.as<float2>();
      pa.W32 = reinterpret_cast<float*>(pa.Qp + std::max<int64_t>(nbc, 1));
      pa.fallback_max_n = prepare_fp64_max_n();
      NOLSM_TRY(launch_ns_qrefine(pa, (int)(e - J), chunk_max_n, plan->max_b, P.A.as<float>(), st));
      plan->stats.launches += 2;
    } else {
      // FP32 factor, A in FP32, Q refined to FP64 accuracy; the FP64 factorisation only where flagged
      const int64_t nbc = plan->h_c_off[e] - plan->h_c_off[J];
      NOLSM_TRY(ensure(plan, plan->ws_refine, (sizeof(double) + sizeof(float)) * (size_t)std::max<int64_t>(nbc, 1)));
      if (sym) {   // the factors stay for the finishing step D_c = L^-T U
        NOLSM_TRY(ensure(plan, plan->ws_ysym, sizeof(float) * (size_t)n2));
        pa.L32 = plan->Lsym.as<float>() + plan->h_a_off[J];
        pa.sym = 1;
        pa.Ysym = plan->ws_ysym.as<float>();
        pa.Wc = plan->Wc.as<double>();
      } else {
        NOLSM_TRY(ensure(plan, plan->ws_l32, sizeof(float) * (size_t)n2));
        pa.L32 = plan->ws_l32.as<float>();
      }
      pa.c_base = plan->h_c_off[J];
      pa.Qp = plan->ws_refine.as<float2>();
      pa.W32 = reinterpret_cast<float*>(pa.Qp + std::max<int64_t>(nbc, 1));
      pa.fallback_max_n = sym ? 0 : prepare_fp64_max_n();   // no FP64 fallback for the symmetric form
      {   // CTAs take the chunk's submatrices largest first, so that the last wave is made of small ones
        std::vector<int32_t> ord((size_t)(e - J));
        for (int64_t k = J; k < e; ++k) ord[(size_t)(k - J)] = (int32_t)k;
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int32_t a, int32_t b) { return plan->h_sub_n[a] > plan->h_sub_n[b]; });
        NOLSM_TRY(ensure(plan, plan->prep_order, sizeof(int32_t) * ord.size()));
        NOLSM_CUDA_TRY(cudaMemcpyAsync(plan->prep_order.p, ord.data(), sizeof(int32_t) * ord.size(),
                                       cudaMemcpyHostToDevice, st));
        NOLSM_CUDA_TRY(cudaStreamSynchronize(st));   // ord is a host temporary
        pa.order = plan->prep_order.as<int32_t>();
      }
      NOLSM_TRY(launch_prepare_mixed(pa, (int)(e - J), chunk_max_n, P.A.as<float>(), st));
      plan->stats.launches += 3;
    }
    pmark(plan, st);
    plan->stats.factor_launches += 1;
    for (int64_t k = J; k < e; ++k) {
      const double m = plan->h_sub_n[k], b = plan->h_sub_b[k];
      // algorithmic flops (2 per FMA): Cholesky m^3/3 FMAs; two triangular solves with m right-hand sides
      // m^3 FMAs (A = L^-T L^-1 H, or M = L^-1 (L^-1 H)^T); the Q solves m^2 b FMAs each (FP64 path: one;
      // mixed: the first solve and one correction, plus m^2 b / 2 for W_c in the symmetric form); the
      // residual of the refinement m^2 b FMAs (counted once, not its double-FP32 emulation)
      const double fma_fact = m * m * m / 3.0 + m * m * m;
      if (keep_fp64_A) {
        plan->stats.flops_fp64 += 2.0 * (fma_fact + m * m * b);
      } else if (cls == kPrepNS) {
        // the tensor products are counted by launch_ns_inverse; here the refinement's FP32 X r products
        plan->stats.flops_fp32 += 2.0 * 2.0 * m * m * b;
      } else {
        plan->stats.flops_fp32 += 2.0 * (fma_fact + (sym ? 3.5 : 3.0) * m * m * b);
      }
      P.done[k] = 1;
    }
    J = e;
  }
  if (ratio && any_chunk) {
    NOLSM_CUDA_TRY(cudaMemcpyAsync(P.h_cond.data() + j0, P.cond.as<float>() + j0, sizeof(float) * (size_t)(j1 - j0),
                                   cudaMemcpyDeviceToHost, st));
    NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return NOLSM_OK;
}

nolsm_status ensure_results(nolsm_plan* plan) {
  const int32_t n_mol = plan->n_mol;
  if (!plan->Dc.p) {
    NOLSM_TRY(dev_alloc(plan, plan->Dc, sizeof(double) * (size_t)std::max<int64_t>(plan->h_c_off[n_mol], 1)));
    NOLSM_TRY(dev_alloc(plan, plan->t_S, sizeof(double) * n_mol));
    NOLSM_TRY(dev_alloc(plan, plan->t_H, sizeof(double) * n_mol));
    NOLSM_TRY(dev_alloc(plan, plan->iters, sizeof(int32_t) * n_mol));
    NOLSM_TRY(dev_alloc(plan, plan->status, sizeof(int32_t) * n_mol));
    NOLSM_TRY(dev_alloc(plan, plan->sums, sizeof(double) * 8));
    NOLSM_TRY(dev_alloc(plan, plan->rsteps, sizeof(int32_t) * n_mol));
    NOLSM_TRY(dev_alloc(plan, plan->nbelow, sizeof(int32_t) * n_mol));
    NOLSM_TRY(dev_alloc(plan, plan->counter, sizeof(int32_t) * 4));
  }
  return NOLSM_OK;
}

nolsm_status solve_fp64(nolsm_plan* plan, double mu, const nolsm_options& o, int64_t j0, int64_t j1,
                        const SolveSpec& spec, cudaStream_t st) {
  NOLSM_TRY(ensure_results(plan));
  int dev = 0, sms = 0;
  NOLSM_CUDA_TRY(cudaGetDevice(&dev));
  NOLSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int slots = (int)std::min<int64_t>(2 * sms, spec.list ? spec.count : j1 - j0);
  if (slots <= 0) return NOLSM_OK;
  int32_t maxn = 0;
  for (int64_t J = j0; J < j1; ++J) maxn = std::max(maxn, plan->h_sub_n[J]);
  const int64_t slot_elems = (int64_t)maxn * maxn;
  NOLSM_TRY(ensure(plan, plan->ws_ns, sizeof(double) * 3 * (size_t)slot_elems * slots));
  NOLSM_CUDA_TRY(cudaMemsetAsync(plan->counter.p, 0, sizeof(int32_t), st));
  NsArgs g;
  g.j0 = (int32_t)j0; g.j1 = (int32_t)j1;
  g.sub_n = plan->sub_n.as<int32_t>(); g.nbf = plan->sub_b.as<int32_t>();
  g.a_off = plan->a_off.as<int64_t>(); g.c_off = plan->c_off.as<int64_t>();
  g.A = plan->prep64.A.as<double>(); g.Q = plan->Q.as<double>(); g.Sc = plan->Sc.as<double>();
  g.Hc = plan->Hc.as<double>(); g.lam = spec.lam ? spec.lam : plan->lam.as<double>();
  g.lam_g = plan->lam.as<double>();
  g.prep_status = plan->prep_status.as<int32_t>();
  g.mu = mu; g.tol = o.tol_ns;
  g.max_iter = o.max_iter;
  g.budget = spec.budget; g.list = spec.list; g.count = spec.count;
  g.ws = plan->ws_ns.as<double>(); g.slot_elems = slot_elems;
  g.next = plan->counter.as<int32_t>();
  g.Dc = plan->Dc.as<double>(); g.tS = plan->t_S.as<double>(); g.tH = plan->t_H.as<double>();
  g.iters = plan->iters.as<int32_t>(); g.status = plan->status.as<int32_t>();
  g.rsteps = plan->rsteps.as<int32_t>();
  g.nbelow = plan->nbelow.as<int32_t>();
  k_ns_fp64<<<slots, 256, 0, st>>>(g);
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 1;
  return NOLSM_OK;
}

nolsm_status reduce_traces(nolsm_plan* plan, int64_t j0, int64_t j1, int terms_main, cudaStream_t st, double* tS,
                           double* tH, int32_t* first_bad_status, const int32_t* list, int32_t count) {
  k_reduce<<<1, 256, 0, st>>>((int32_t)j0, (int32_t)j1, plan->t_S.as<double>(), plan->t_H.as<double>(),
                              plan->status.as<int32_t>(), plan->iters.as<int32_t>(), plan->rsteps.as<int32_t>(),
                              plan->sub_n.as<int32_t>(), terms_main, list, count, plan->sums.as<double>());
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 1;
  double h[8];
  NOLSM_CUDA_TRY(cudaMemcpyAsync(h, plan->sums.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  *tS = h[0];
  *tH = h[1];
  *first_bad_status = h[2] < 0 ? 0 : (int32_t)h[3];
  plan->stats.flops_paper += h[4];
  plan->stats.flops_tensor += h[5];
  plan->stats.flops_tensor_padded += h[6];
  plan->stats.ns_steps += (int64_t)h[7];
  return NOLSM_OK;
}

nolsm_status scatter(nolsm_plan* plan, double* D, int64_t j0, int64_t j1, cudaStream_t st, const double* src) {
  if (plan->grouped) return scatter_grouped(plan, D, j0, j1, st, src);
  const int64_t p0 = plan->h_nb_ptr[j0], p1 = plan->h_nb_ptr[j1];
  if (p1 <= p0) return NOLSM_OK;
  const int64_t threads = (p1 - p0) * 32;
  k_scatter<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      plan->n_mol, p0, p1, plan->sys.nbf, plan->nb_ptr.as<int32_t>(), plan->nb_idx.as<int32_t>(),
      plan->nb_off.as<int32_t>(), plan->d_slot.as<int32_t>(), plan->d_blk_off.as<int64_t>(), plan->c_off.as<int64_t>(),
      src ? src : plan->Dc.as<double>(), D);
  NOLSM_LAUNCH_CHECK();
  plan->stats.launches += 1;
  return NOLSM_OK;
}

}  // namespace nolsm
