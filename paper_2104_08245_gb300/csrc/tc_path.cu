// a4-a7 on the 5th-generation tensor cores (tcgen05) for the low-precision modes.
//
// Newton-Schulz sign iteration (Eq. NS1): X_{k+1} = 1/2 X_k (3I - X_k^2), two products per step:
//   GEMM0: Y = X X      -> epilogue writes T = 3I - Y and sums the defect ||I - X^2||_F^2
//   GEMM1: Z = X T      -> epilogue writes X_{k+1} = Z / 2 (the last one feeds the centre columns)
// Each product is either one tensor-core product of the rounded operands (BF16 or FP16) or the
// three-term split hi*hi + hi*lo + lo*hi with x = hi + lo (hi = round(x), lo = round(x - hi)),
// accumulated in FP32 in tensor memory.
//
// One persistent CTA per SM keeps two submatrices in flight ("slots", taken largest first from a
// work counter) and interleaves their products: while the tensor cores run a product of one slot,
// the epilogue drains, rounds and stores the previous product of the other, so neither the operand
// fill nor the epilogue of a product serialises the CTA. Operands live in per-slot scratch in global
// memory (L2-resident) as 2-byte planes [X0 hi, X0 lo, X1 hi, X1 lo, T hi, T lo], each R x LD
// (R = n rounded up to 128 rows, LD = n rounded up to 64 columns, zero padded). Output tiles are
// 128 rows x up to 256 columns; the K dimension streams in slices of 64 through a two-stage TMA
// pipeline with 128-byte swizzle; the epilogue writes the rounded planes back with TMA stores.
// Warp roles: warp 0 (one thread) schedules the products of both slots and issues their TMA loads,
// publishing one descriptor per product in a small ring; warp 1 (one thread) issues tcgen05.mma in
// that order; warps 4-11 (two groups of four, even and odd 32-column chunks) drain the
// double-buffered TMEM accumulators (2 x 256 columns), decide convergence and start and finish the
// slots' submatrices. All waits are bounded by the global timer; a wait that runs out marks the
// submatrices in flight as timed out.
//
// The same kernel, instantiated in its second mode, prepares A_J = T_J(S)^-1 T_J(H0) on the tensor cores
// by the coupled Newton-Schulz iteration for the inverse square root (Eqs. inv1-inv3): with Y_0 = T_J(S)/c
// and Z_0 = I, V_k = Z_k Y_k, Y_{k+1} = 1/2 Y_k (3I - V_k), Z_{k+1} = 1/2 (3I - V_k) Z_k, Z_k tends to
// (T_J(S)/c)^-1/2, so T_J(S)^-1 = Z^2 / c (Eq. inv3) and A_J = (Z^2 / c) T_J(H0). Every product is a
// three-term FP16 split. The step whose V_k has ||I - V_k||_F / sqrt(n) <= tol_inv is the last (its Y
// update is skipped, Z alone is needed); c = Tr T_J(S) / n, the mean eigenvalue, so that the eigenvalues
// of Y_0 average 1 and lie in (0, 2), where the iteration converges, unless the largest eigenvalue of
// T_J(S) exceeds twice the mean (then the defect grows, and the submatrix, like any whose iteration does
// not reach tol_inv within max_inv steps, is flagged for the FP64 preparation). X = T_J(S)^-1 is also
// written in FP32 for the refinement of the centre columns of T_J(S)^-1.
// This mode runs 512 threads: three epilogue groups (warps 4-15, every third chunk each), since the start
// of a submatrix (three operand pairs from T_J(S)) and T_J(H0) weigh more against its few products; its
// tiles are 128 x up to 192 columns, and the TMA / MMA warpgroup hands registers to the epilogue (setmaxnreg).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <cmath>

#include "nolsm_internal.cuh"
#include "prep.cuh"
#include "tc_path.cuh"
#include "tcgen05.cuh"
#include "tmap.cuh"

namespace nolsm {

namespace {

constexpr int kStages = 2;
constexpr uint32_t kABytes = 128 * 64 * 2;        // one A plane slice: 128 rows x 64 K
constexpr int kMaxEpiWarps = 12;

// The two launch shapes. Warp 0 issues the TMA loads, warp 1 the MMAs; the epilogue warps from warp 4 on
// come in groups of four (each group covers the 128 TMEM lanes) and deal a tile's 32-column chunks round
// robin. Shape 0: 384 threads, two groups, tiles of 128 x up to 256 columns. Shape 1: 512 threads, three
// groups, tiles of 128 x up to 192 columns (so that the twelve 4 KB staging buffers fit beside the two
// operand stages), with a register split (below). Which one runs a bucket of submatrices is measured
// (tc_shape): shape 0 wins for the sign iteration, shape 1 for the inverse square root, whose per-submatrix
// start (operand pairs from T_J(S)) and T_J(H0) weigh more against its few products.
template <int kShape>
struct Shape {
  static constexpr int kThreads = kShape == 0 ? 384 : 512;
  static constexpr int kEpiWarps = kThreads / 32 - 4;
  static constexpr int kEpiThreads = 32 * kEpiWarps;
  static constexpr int kGroups = kEpiWarps / 4;
  static constexpr int kTileN = kShape == 0 ? 256 : 192;       // N of one MMA
  static constexpr uint32_t kBBytes = 64 * kTileN * 2;        // one B plane slice: 64 K x up to kTileN columns
  static constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;
  static constexpr uint32_t kStgTotal = 4096 * kEpiWarps;    // a 4 KB hi/lo staging buffer per epilogue warp
  static constexpr int kSmemBytes = kStages * kStageBytes + kStgTotal + 1024;
};
static_assert(Shape<1>::kEpiWarps <= kMaxEpiWarps && Shape<0>::kEpiWarps <= kMaxEpiWarps, "epilogue warps");
static_assert(Shape<0>::kSmemBytes <= 227 * 1024 && Shape<1>::kSmemBytes <= 227 * 1024, "shared memory");
// Register split of the 512-thread shape: the launch gives every thread kRegsLaunch registers (512 x 128 = the
// SM's 65,536); the first warpgroup (TMA and MMA threads) releases down to kRegsLow and the three epilogue
// warpgroups take kRegsEpi: 128 x 56 + 384 x 152 = 65,536, so the increase never waits on registers that do
// not exist.
constexpr int kRegsLaunch = 128, kRegsLow = 56, kRegsEpi = 152;
static_assert(128 * kRegsLow + Shape<1>::kEpiThreads * kRegsEpi <= Shape<1>::kThreads * kRegsLaunch,
              "register split above the launch");
constexpr int kPlanes = 6;
constexpr uint64_t kWaitNs = 2000000000ull;        // default limit per wait (2 s); one product takes < 1 ms

enum : int { FMT_F16 = 0, FMT_BF16 = 1, FMT_E4M3 = 2 };

struct Fmt {
  int fmt;    // FMT_F16 / FMT_BF16 / FMT_E4M3
  int terms;  // 1 or 3 (E4M3: 1)
};

// E4M3 operands carry a fixed power-of-two scale: the symmetric iterates have |x_ij| <= rho <= 1.7 (the
// scale guard), so x * 2^7 stays below 218 of E4M3's 448 and values down to 2^-16 keep a subnormal; a
// product of two scaled operands is scaled back by 2^-14.
constexpr float kF8Up = 128.0f;
constexpr float kF8Down = 1.0f / 16384.0f;
constexpr float kF8Switch = 0.1f;   // defect at which the E4M3 phase hands over to the refinement format
// K extent of an E4M3 operand row: whole 128-byte slices
__host__ __device__ inline int k8_extent(int n64) { return (n64 + 127) & ~127; }

struct TcArgs {
  int32_t j0, j1;
  const int32_t* order;       // submatrices of [j0, j1), largest first
  const int32_t* sub_n; const int32_t* nbf;
  const int64_t* a_off; const int64_t* c_off;
  const float* A;             // FP32 A_J
  const double* Q; const double* Sc; const double* Hc; const double* lam;
  const double* lam_g;        // Gershgorin interval (the scale never drops below its alpha / 1.7)
  const int32_t* prep_status;
  double mu;
  float tol_ns, tol_accept;
  int32_t max_iter, refine_steps;
  const int32_t* budget;      // per-submatrix step cap (nullable)
  Fmt main_fmt, refine_fmt;
  uint16_t* planes;           // [slots*6][R][LD]
  int32_t R, LD;
  int32_t* next;              // work counter
  int32_t* err;               // global error flag (timeouts)
  double* Dc; double* tS; double* tH; int32_t* iters; int32_t* status; int32_t* rsteps;
  int32_t* nbelow;            // eigenvalues below mu, (n - Tr X) / 2 (nullable)
  uint64_t wait_ns;           // limit of every wait on another role (the teardown's own waits: 50 ms)
  const float* cond;          // preparation's cond(T_J(S)) estimate (nullable): above cond_max the submatrix
  float cond_max;             // is left to the FP64 path (its status stays as it is) when it has at most
  int32_t ill_max_n;          // ill_max_n rows (what the FP64 preparation takes)
  // inverse-square-root mode: the chunk's gathered T_J(S), T_J(H0) (FP64, at a_off[J] - a_base and
  // chunk_n2 further), the outputs and the iteration's stopping rule
  const double* ws;
  int64_t a_base, chunk_n2;
  float* Aout;                // FP32 A_J at a_off[J]
  float* Xout;                // FP32 T_J(S)^-1 at a_off[J] - a_base
  int32_t* prep_out;          // kSubOk, or kSubRefine when the iteration failed (FP64 preparation next)
  float tol_inv;
  int32_t max_inv;
  double* flops;              // [2]: 2 n^3 per product (method count) and the split's issued flops, summed
};

// Epilogue of a product: what is done with the accumulator P
enum : int {
  kEpiT = 0,      // T = 3I - P to the planes, and the defect ||I - P||_F^2
  kEpiScale = 1,  // scale * P to the planes
  kEpiX = 2,      // scale * P to the planes and in FP32 to Xout
  kEpiA = 3       // P in FP32 to Aout (no planes)
};
constexpr int kPlanesInv = 10;   // inverse mode: plane pairs Y (then T_J(H0)), Z, T (then X), Y', Z'

constexpr int kSlots = 2;   // submatrices in flight per CTA (their products interleave)
constexpr int kRing = 4;    // product descriptors between the scheduler and the MMA / epilogue warps

// Iteration state of one in-flight submatrix. Written by the epilogue (thread 128) before it arrives
// on the slot's epi_done barrier; read by the scheduler after waiting on that barrier.
struct SlotState {
  int job;                       // submatrix index, -1 when the slot has retired
  int n, n64, R, nrb, ncb, nks;  // dimension and tiling
  int kind;                      // next product: 0 (X X) or 1 (X T)
  int cur;                       // which X plane pair holds the current iterate
  int phase, refine_left, steps, rsteps, status, last;
  float dprev;                   // defect of the previous step (E4M3 stagnation test)
  Fmt fcur, fnxt;
  int yc, zc;                    // inverse mode: plane pairs of the current Y and Z
  int zdone;                     // inverse mode: this step's Z update was made at the start (step 0)
  float cinv;                    // inverse mode: 1 / c
  float zs;                      // inverse mode: Z = zs x (Z's planes); 1/2 until the first Z update, whose
                                 // planes hold T_0 = 2 Z_1
};

// One product as scheduled by the producer: read in order by the MMA issuer and the epilogue.
struct Desc {
  int term;                      // 1: no more products, exit
  int slot, kind, last;
  Fmt f, fo;                     // format of the operands; of the operand the epilogue writes
  int n, n64, nrb, ncb, nks;
  int za, zb, zo;                // plane indices (hi planes) of A, B and the output
  int epi;                       // kEpi*
  float scale;                   // kEpiScale, kEpiX
  float pscale;                  // kEpiT: the product is pscale P
};

struct Shared {
  uint64_t full[kStages], empty[kStages], accf[2], acce[2], idle;
  uint64_t epi_done[kSlots], desc_full[kRing];
  uint32_t tmem;
  int err;
  int fetch;
  SlotState slot[kSlots];
  Desc ring[kRing];
  float red[2][kMaxEpiWarps];    // defect partial sums, by product parity
  double dred[3][kMaxEpiWarps];
};

__device__ __forceinline__ float from_bits(uint16_t b, int fmt) {
  if (fmt == FMT_BF16) return __bfloat162float(__ushort_as_bfloat16(b));
  return __half2float(__ushort_as_half(b));
}

// Two values rounded to the 2-byte format (packed) and their low parts x - round(x) rounded likewise.
__device__ __forceinline__ void split2(float a, float b, int fmt, uint32_t& hi, uint32_t& lo) {
  if (fmt == FMT_BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// s + c <- s + c + p with s = fl(s + p) and the rounding error of that sum added to c (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float& s, float& c, float p) {
  const float t = s + p;
  const float z = t - s;
  c += (s - (t - z)) + (p - z);
  s = t;
}

// 32 consecutive values of one row as packed hi (and lo) pairs; the format a template parameter (one
// branch per chunk, none per pair), the lo parts only when the format has them.
template <int kFmt, bool kLo>
__device__ __forceinline__ void split_pack_t(const float (&v)[32], uint32_t (&h)[16], uint32_t (&l)[16]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (kLo) {
      split2(v[2 * j], v[2 * j + 1], kFmt, h[j], l[j]);
    } else if (kFmt == FMT_BF16) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      h[j] = *reinterpret_cast<const uint32_t*>(&b);
    } else {
      const __half2 b = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
      h[j] = *reinterpret_cast<const uint32_t*>(&b);
    }
  }
}
__device__ __forceinline__ void split_pack(const float (&v)[32], Fmt f, uint32_t (&h)[16], uint32_t (&l)[16]) {
  if (f.fmt == FMT_BF16) {
    if (f.terms > 1) split_pack_t<FMT_BF16, true>(v, h, l);
    else split_pack_t<FMT_BF16, false>(v, h, l);
  } else {
    if (f.terms > 1) split_pack_t<FMT_F16, true>(v, h, l);
    else split_pack_t<FMT_F16, false>(v, h, l);
  }
}

// One row of X (2-byte hi and, with kLo, lo planes; n64 columns, zero padded) times 8 columns of Q in
// FP32 (rows of stride bp, zero padded to n64 rows): FP32 partial sums of 16 products, each added to
// sh + sl with TwoSum. The row is read in 32-column pieces, eight 16-byte loads in flight.
template <int kFmt, bool kLo>
__device__ __forceinline__ void xq_row(const uint16_t* __restrict__ xh, const uint16_t* __restrict__ xl, int n64,
                                       const float* __restrict__ Qs, int bp, float (&sh)[8], float (&sl)[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) sh[c] = sl[c] = 0.0f;
  for (int k0 = 0; k0 < n64; k0 += 32) {
    uint4 hv[4], lv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      hv[t] = *reinterpret_cast<const uint4*>(xh + k0 + 8 * t);
      lv[t] = kLo ? *reinterpret_cast<const uint4*>(xl + k0 + 8 * t) : make_uint4(0, 0, 0, 0);
    }
    float p[8];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      if ((u & 15) == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) p[c] = 0.0f;
      }
      const uint4 h4 = hv[u >> 3], l4 = lv[u >> 3];
      const int w = (u & 7) >> 1, sft = 16 * (u & 1);
      const uint32_t hw = w == 0 ? h4.x : w == 1 ? h4.y : w == 2 ? h4.z : h4.w;
      const uint32_t lw = w == 0 ? l4.x : w == 1 ? l4.y : w == 2 ? l4.z : l4.w;
      float x = from_bits((uint16_t)(hw >> sft), kFmt);
      if (kLo) x += from_bits((uint16_t)(lw >> sft), kFmt);
      const float4 qa = *reinterpret_cast<const float4*>(Qs + (size_t)(k0 + u) * bp);
      const float4 qb = *reinterpret_cast<const float4*>(Qs + (size_t)(k0 + u) * bp + 4);
      const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
#pragma unroll
      for (int c = 0; c < 8; ++c) p[c] = fmaf(x, qv[c], p[c]);
      if ((u & 15) == 15) {
#pragma unroll
        for (int c = 0; c < 8; ++c) two_sum(sh[c], sl[c], p[c]);
      }
    }
  }
}

// named barrier 3 for the N epilogue threads
template <int N>
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 3, %0;" ::"n"(N) : "memory"); }
// barrier 3 with an OR over the N epilogue threads' predicates
template <int N>
__device__ __forceinline__ bool epi_bar_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred P, Q;\n\tsetp.ne.u32 P, %1, 0;\n\tbar.red.or.pred Q, 3, %2, P;\n\tselp.u32 %0, 1, 0, Q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p), "n"(N)
      : "memory");
  return r != 0;
}

// Whether row tile mb of a product is an M = 64 tile: the last one of a kind::f16 product whose n64 is an odd
// multiple of 64 (n = 129..192 runs as 128 + 64 rows instead of 2 x 128). Its accumulator rows r sit in TMEM
// lanes 32 (r / 16) + r % 16, the first 16 lanes of each warp's quarter.
__device__ __forceinline__ bool tail64(const Desc& d, int mb) {
  return d.f.fmt != FMT_E4M3 && d.fo.fmt != FMT_E4M3 && mb == d.nrb - 1 && (d.n64 & 127) == 64;
}

// kMode 0: the sign iteration (a4-a7); kMode 1: the inverse square root of T_J(S) and A_J (a2-a3); kShape:
// the launch shape (Shape)
template <int kMode, int kShape>
__global__ void __launch_bounds__(Shape<kShape>::kThreads, 1)
    k_ns_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
            const __grid_constant__ CUtensorMap mapS, const __grid_constant__ CUtensorMap mapA8,
            const __grid_constant__ CUtensorMap mapB8, const __grid_constant__ CUtensorMap mapS16,
            const __grid_constant__ CUtensorMap mapS2, const __grid_constant__ CUtensorMap mapS16x2, TcArgs g) {
  constexpr int kPps = kMode == 0 ? kPlanes : kPlanesInv;   // planes per slot
  constexpr int kEpiWarps = Shape<kShape>::kEpiWarps, kEpiThreads = Shape<kShape>::kEpiThreads;
  constexpr int kGroups = Shape<kShape>::kGroups, kTileN = Shape<kShape>::kTileN;
  constexpr uint32_t kBBytes = Shape<kShape>::kBBytes, kStageBytes = Shape<kShape>::kStageBytes;
  constexpr uint32_t kStgTotal = Shape<kShape>::kStgTotal;
  extern __shared__ uint8_t smraw[];
  uint8_t* stage_mem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ Shared sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&sh.full[s], 1);
      tc::mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&sh.accf[b], 1);
      tc::mbar_init(&sh.acce[b], kEpiThreads);
    }
    for (int s = 0; s < kSlots; ++s) tc::mbar_init(&sh.epi_done[s], kEpiThreads);
    for (int r = 0; r < kRing; ++r) tc::mbar_init(&sh.desc_full[r], 1);
    tc::mbar_init(&sh.idle, 1);
    tc::fence_mbar_init();
    sh.err = 0;
    tc::prefetch_tmap(&mapA);
    tc::prefetch_tmap(&mapB);
    tc::prefetch_tmap(&mapS);
    tc::prefetch_tmap(&mapA8);
    tc::prefetch_tmap(&mapB8);
    tc::prefetch_tmap(&mapS16);
    tc::prefetch_tmap(&mapS2);
    tc::prefetch_tmap(&mapS16x2);
  }
  if (warp == 0) {
    tc::tmem_alloc(&sh.tmem, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sh.tmem;
  const size_t plane_elems = (size_t)g.R * g.LD;
  uint8_t* const stg = stage_mem + kStages * kStageBytes;   // epilogue staging: 4 KB per epilogue warp
  const int sub0 = blockIdx.x * kSlots;                      // scratch sub-slot of this CTA's slot 0
  uint32_t arm_phase[kStages] = {0, 0};                      // producer: parity of the last load armed per stage
  bool armed[kStages] = {false, false};

  if (warp < 4) {
  if constexpr (kShape == 1) tc::setmaxnreg_dec<kRegsLow>();   // the TMA / MMA warpgroup gives registers up
  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ producer: schedules the products of the slots
    // a slot's next product is issued once the epilogue of its previous product (or its initialisation) has
    // arrived on the slot's epi_done barrier; the live slots are polled round robin from the one after the
    // last pick, and the first that is ready goes (no slot waits behind another's epilogue)
    bool alive[kSlots];
    uint32_t epar[kSlots];
    for (int c = 0; c < kSlots; ++c) {
      alive[c] = true;
      epar[c] = 0;
    }
    uint32_t kcount = 0;
    int s = 0;
    for (uint32_t i = 0;; ++i) {
      int pick = -1;
      const uint64_t deadline = tc::globaltimer() + 4 * g.wait_ns;
      for (;;) {
        bool any = false;
        for (int t = 0; t < kSlots && pick < 0; ++t) {
          const int c = (s + t) % kSlots;
          if (!alive[c]) continue;
          any = true;
          if (!tc::mbar_test_wait(&sh.epi_done[c], epar[c])) continue;
          epar[c] ^= 1;
          tc::fence_proxy_async_global();   // the epilogue's plane writes, before TMA reads them
          if (sh.slot[c].job >= 0) pick = c;
          else alive[c] = false;
        }
        if (pick >= 0 || !any || sh.err) break;
        if (tc::globaltimer() > deadline) {
          sh.err = 1;
          break;
        }
      }
      Desc d;
      d.term = pick < 0 ? 1 : 0;
      if (pick >= 0) {
        const SlotState& st = sh.slot[pick];
        d.slot = pick;
        d.kind = st.kind;
        d.f = st.fcur;
        d.n = st.n; d.n64 = st.n64; d.nrb = st.nrb; d.ncb = st.ncb; d.nks = st.nks;
        const int zb = (sub0 + pick) * kPps;
        d.pscale = 1.0f;
        if constexpr (kMode == 0) {   // the epilogue derives epi and scale from the kind
          d.last = st.kind == 1 && st.last;
          d.fo = st.kind == 0 ? st.fcur : st.fnxt;
          d.za = zb + 2 * st.cur;
          d.zb = st.kind == 0 ? d.za : zb + 4;
          // X_{k+1} overwrites X_k when one column tile covers the matrix: row block mb of X_k is read
          // (as the A operand) only by tile (mb, 0), whose loads have completed before its epilogue writes
          d.zo = st.kind == 0 ? zb + 4 : (st.ncb == 1 ? d.za : zb + 2 * (st.cur ^ 1));
        } else {
          // pairs: Y in 0 (updated in place when one column tile covers the matrix, else ping-pong with 3),
          // Z in 1 or 4 (ping-pong: every row tile of T Z reads all of Z; until the first Z update the pair
          // holds T_0 = 2 Z_1, hence the factor zs), T and then X in 2; T_J(H0) goes into Y's pair once Y is
          // no longer needed
          d.last = st.kind == 4;
          d.scale = 0.5f;
          d.fo = st.fcur;
          switch (st.kind) {
            case 0:  // V = Z Y -> T = 3I - V
              d.za = zb + 2 * st.zc; d.zb = zb + 2 * st.yc; d.zo = zb + 4; d.epi = kEpiT; d.pscale = st.zs; break;
            case 1:  // Y' = 1/2 Y T (row block mb of Y is read only by tile (mb, 0), as for X X T); at step 0
                     // T_0 is in Z's pair
              d.za = zb + 2 * st.yc; d.zb = st.zdone ? zb + 2 * st.zc : zb + 4;
              d.zo = st.ncb == 1 ? d.za : zb + 2 * (st.yc == 0 ? 3 : 0);
              d.epi = kEpiScale; break;
            case 2:  // Z' = 1/2 T Z
              d.za = zb + 4; d.zb = zb + 2 * st.zc; d.zo = zb + 2 * (st.zc == 1 ? 4 : 1); d.epi = kEpiScale;
              d.scale = 0.5f * st.zs; break;
            case 3:  // X = Z Z / c = T_J(S)^-1
              d.za = zb + 2 * st.zc; d.zb = d.za; d.zo = zb + 4; d.epi = kEpiX; d.scale = st.cinv * st.zs * st.zs;
              break;
            default:  // A_J = X T_J(H0)
              d.za = zb + 4; d.zb = zb + 2 * st.yc; d.zo = zb + 4; d.epi = kEpiA; break;
          }
        }
      }
      sh.ring[i % kRing] = d;
      tc::mbar_arrive(&sh.desc_full[i % kRing]);
      if (d.term) break;
      const int two = d.f.terms > 1 ? 2 : 1;
      const bool f8 = d.f.fmt == FMT_E4M3;
      const int nks = f8 ? k8_extent(d.n64) / 128 : d.nks;   // E4M3: 128-byte K slices
      for (int mb = 0; mb < d.nrb && !sh.err; ++mb)
        for (int cb = 0; cb < d.ncb && !sh.err; ++cb) {
          const int nt = min(kTileN, d.n64 - kTileN * cb);
          // an M = 64 tile loads 64 rows of A (the B map's 64 x 64 box)
          const bool m64 = tail64(d, mb);
          const uint32_t abytes = m64 ? kABytes / 2 : kABytes;
          // E4M3: both operands K-major (the symmetric iterate is its own transpose); the B box is always
          // kTileN rows (rows past R are zero-filled by the copy)
          const uint32_t bytes = f8 ? kABytes + (uint32_t)kTileN * 128u : (uint32_t)two * (abytes + (uint32_t)nt * 128u);
          for (int ks = 0; ks < nks; ++ks) {
            const int st = kcount % kStages;
            const uint32_t ph = (kcount / kStages) & 1;
            if (!tc::mbar_wait(&sh.empty[st], ph ^ 1, tc::globaltimer() + g.wait_ns)) { sh.err = 1; break; }
            uint8_t* sm = stage_mem + st * kStageBytes;
            tc::mbar_arrive_expect_tx(&sh.full[st], bytes);
            armed[st] = true;
            arm_phase[st] = ph;
            if (f8) {
              tc::tma_load_3d(sm, &mapA8, &sh.full[st], 128 * ks, 128 * mb, d.za);
              tc::tma_load_3d(sm + 2 * kABytes, &mapB8, &sh.full[st], 128 * ks, kTileN * cb, d.zb);
            } else {
              for (int z = 0; z < two; ++z) {
                tc::tma_load_3d(sm + z * kABytes, m64 ? &mapB : &mapA, &sh.full[st], 64 * ks, 128 * mb, d.za + z);
                uint8_t* bdst = sm + 2 * kABytes + z * kBBytes;
                for (int c = 0; c < nt / 64; ++c)
                  tc::tma_load_3d(bdst + c * 8192, &mapB, &sh.full[st], kTileN * cb + 64 * c, 64 * ks, d.zb + z);
              }
            }
            ++kcount;
          }
        }
      s = (pick + 1) % kSlots;
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer: the products in the scheduler's order
    uint32_t kcount = 0, tcount = 0;
    for (uint32_t i = 0; !sh.err; ++i) {
      if (!tc::mbar_wait(&sh.desc_full[i % kRing], (i / kRing) & 1, tc::globaltimer() + 8 * g.wait_ns)) {
        sh.err = 1;
        break;
      }
      const Desc d = sh.ring[i % kRing];
      if (d.term) break;
      const bool f8 = d.f.fmt == FMT_E4M3;
      const int nks = f8 ? k8_extent(d.n64) / 128 : d.nks;
      // kind::f16 products run over n16 = n rounded up to 16 in N and K (the loads stay whole 64-wide slices):
      // the operands' rows and columns past n are zero, so the entries the trimmed product leaves out are 0
      const int n16 = (d.n + 15) & ~15;
      for (int mb = 0; mb < d.nrb && !sh.err; ++mb)
        for (int cb = 0; cb < d.ncb && !sh.err; ++cb) {
          const int nt = min(kTileN, d.n64 - kTileN * cb);
          const int ntu = min(nt, n16 - kTileN * cb);
          // kind::f16: A K-major, B MN-major; kind::f8f6f4 (E4M3 = 0): both K-major
          const uint32_t id = f8 ? tc::idesc(0, 0, 0, 0, 128, nt)
                                 : tc::idesc(d.f.fmt, d.f.fmt, 0, 1, tail64(d, mb) ? 64 : 128, ntu);
          const int buf = tcount & 1;
          if (!tc::mbar_wait(&sh.acce[buf], ((tcount >> 1) & 1) ^ 1, tc::globaltimer() + g.wait_ns)) {
            sh.err = 1;
            break;
          }
          tc::tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)buf * 256;
          for (int ks = 0; ks < nks; ++ks) {
            const int st = kcount % kStages;
            const uint32_t ph = (kcount / kStages) & 1;
            if (!tc::mbar_wait(&sh.full[st], ph, tc::globaltimer() + g.wait_ns)) { sh.err = 1; break; }
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_u32(stage_mem + st * kStageBytes);
            const uint32_t b0 = a0 + 2 * kABytes;
            if (f8) {   // four K = 32 steps of 32 bytes through the 128-byte slice
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                tc::mma_f8(dt, tc::sdesc_sw128(a0 + kk * 32, 16, 1024), tc::sdesc_sw128(b0 + kk * 32, 16, 1024), id,
                           (ks > 0 || kk > 0) ? 1u : 0u);
              tc::mma_commit(&sh.empty[st]);
              ++kcount;
              continue;
            }
            const int kku = min(4, (n16 - 64 * ks) / 16);   // K = 16 steps below n16 (at least one)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              if (kk >= kku) break;
              const uint64_t ah = tc::sdesc_sw128(a0 + kk * 32, 16, 1024);
              const uint64_t bh = tc::sdesc_sw128(b0 + kk * 2048, 8192, 1024);
              tc::mma_f16(dt, ah, bh, id, (ks > 0 || kk > 0) ? 1u : 0u);
              if (d.f.terms > 1) {
                const uint64_t al = tc::sdesc_sw128(a0 + kABytes + kk * 32, 16, 1024);
                const uint64_t bl = tc::sdesc_sw128(b0 + kBBytes + kk * 2048, 8192, 1024);
                tc::mma_f16(dt, ah, bl, id, 1u);
                tc::mma_f16(dt, al, bh, id, 1u);
              }
            }
            tc::mma_commit(&sh.empty[st]);
            ++kcount;
          }
          tc::mma_commit(&sh.accf[buf]);
          ++tcount;
        }
    }
  }
  } else {
  if constexpr (kShape == 1) tc::setmaxnreg_inc<kRegsEpi>();   // to the epilogue groups
  {
    // ------------------------------------------------ epilogue: drains products, decides, finishes and starts slots
    const int etid = tid - 128;              // 0..255
    const int q = warp & 3;                  // TMEM lane quarter of this warp
    const int grp = (warp - 4) >> 2;         // epilogue group: chunks grp, grp + 3, ... of a tile
    uint32_t tcount = 0;

    // One FP64 n x n matrix M (row-major) as an n64 x n64 operand (zero padded) into the 3-term FP16 planes
    // hi, lo (hi + plane_elems): four rows per warp pass, 8 consecutive columns per lane, the pass's 32 loads
    // all issued before its first store, then 16-byte stores.
    auto fill_pair = [&](uint16_t* hi, int n, int n64, const double* __restrict__ M) {
      uint16_t* lo = hi + plane_elems;
      for (int i0 = 4 * (warp - 4); i0 < n64; i0 += 4 * kEpiWarps) {
        for (int j0 = 8 * lane; j0 < n64; j0 += 256) {
          float vv[4][8];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int i = i0 + r;
#pragma unroll
            for (int u = 0; u < 8; ++u) vv[r][u] = (i < n && j0 + u < n) ? (float)__ldg(M + (size_t)i * n + j0 + u) : 0.0f;
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int i = i0 + r;
            if (i >= n64) break;
            const float (&v)[8] = vv[r];
            uint32_t h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) split2(v[2 * u], v[2 * u + 1], FMT_F16, h[u], l[u]);
            *reinterpret_cast<uint4*>(hi + (size_t)i * g.LD + j0) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(lo + (size_t)i * g.LD + j0) = make_uint4(l[0], l[1], l[2], l[3]);
          }
        }
      }
    };

    // inverse mode, a new submatrix J in slot s: c = Tr T_J(S) / n and step 0 without products, since Z_0 = I:
    // V_0 = Y_0 = T_J(S) / c and T_0 = 3I - Y_0 are written directly (pairs 0 and 1, Z's pair: Z_1 = T_0 / 2,
    // the factor 1/2 applied by the products that read Z until its first update), with the defect
    // ||I - Y_0||_F / sqrt(n); only Y_1 = Y_0 T_0 / 2 needs the tensor cores.
    auto start_inverse = [&](int s, int J) {
      SlotState& st = sh.slot[s];
      const int n = g.sub_n[J], n64 = (n + 63) & ~63, R = (n + 127) & ~127;
      const double* S = g.ws + (g.a_off[J] - g.a_base);
      const double* H = S + g.chunk_n2;
      // the trace of T_J(S) (every warp sums it alike, lanes along the diagonal)
      double tr = 0.0;
      for (int i = lane; i < n; i += 32) tr += S[(size_t)i * n + i];
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
      const double c = tr / n;
      const float inv = (float)(1.0 / c);
      uint16_t* base = g.planes + (size_t)(sub0 + s) * kPps * plane_elems;
      float dpart = 0.0f;   // this thread's share of ||I - Y_0||_F^2
      // Y_0 and T_0 from one read of T_J(S): the same pass pattern as fill_pair, two pairs out
      for (int i0 = 4 * (warp - 4); i0 < n64; i0 += 4 * kEpiWarps) {
        for (int j0 = 8 * lane; j0 < n64; j0 += 256) {
          float sv[4][8];   // the pass's 32 loads, all issued before its first store
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int i = i0 + r;
#pragma unroll
            for (int u = 0; u < 8; ++u) sv[r][u] = (i < n && j0 + u < n) ? (float)__ldg(S + (size_t)i * n + j0 + u) : 0.0f;
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int i = i0 + r;
            if (i >= n64) break;
            float y[8], t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int j = j0 + u;
              const bool in = i < n && j < n;
              y[u] = sv[r][u] * inv;
              const float e = (i == j && in ? 1.0f : 0.0f) - y[u];
              dpart += e * e;
              t[u] = in ? (i == j ? 3.0f : 0.0f) - y[u] : 0.0f;
            }
            uint32_t h[4], l[4];
            const size_t off = (size_t)i * g.LD + j0;
#pragma unroll
            for (int u = 0; u < 4; ++u) split2(y[2 * u], y[2 * u + 1], FMT_F16, h[u], l[u]);
            *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(base + plane_elems + off) = make_uint4(l[0], l[1], l[2], l[3]);
#pragma unroll
            for (int u = 0; u < 4; ++u) split2(t[2 * u], t[2 * u + 1], FMT_F16, h[u], l[u]);
            *reinterpret_cast<uint4*>(base + 2 * plane_elems + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(base + 3 * plane_elems + off) = make_uint4(l[0], l[1], l[2], l[3]);
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) dpart += __shfl_xor_sync(0xffffffffu, dpart, o);
      if (lane == 0) sh.dred[0][warp - 4] = dpart;
      epi_bar<kEpiThreads>();
      if (tid == 128) {
        float dsum = 0.0f;
        for (int w = 0; w < kEpiWarps; ++w) dsum += (float)sh.dred[0][w];
        const float d0 = sqrtf(dsum / (float)n);
        st.job = J;
        st.n = n; st.n64 = n64; st.R = R;
        st.nrb = R / 128; st.ncb = (n64 + kTileN - 1) / kTileN; st.nks = n64 / 64;
        st.yc = 0; st.zc = 1; st.cinv = inv; st.zs = 0.5f;
        st.steps = 1; st.rsteps = 0; st.status = kSubOk;
        st.fcur = Fmt{FMT_F16, 3}; st.fnxt = st.fcur;
        st.dprev = INFINITY;
        if (!(c > 0.0) || !isfinite(c) || !isfinite(d0)) st.status = kSubRefine;   // the FP64 preparation takes it
        st.last = d0 <= g.tol_inv ? 1 : 0;
        st.kind = st.last ? 3 : 1;     // step 0 the last: X = Z_1 Z_1 / c next; else Y_1 = Y_0 T_0 / 2
        st.zdone = 1;
      }
      epi_bar<kEpiThreads>();   // dred free again; st.last visible to every epilogue thread
      // step 0 the last: Y_0 is not needed, T_J(H0) takes its pair now (else after the last Z update)
      if (st.last) fill_pair(base, n, n64, H);
    };

    // a4 for a new submatrix of slot s: X_0 = (A - mu I) / alpha in the main format, zero padded
    auto start_slot = [&](int s) {
      SlotState& st = sh.slot[s];
      for (;;) {
        if (tid == 128) {
          const int k = atomicAdd(g.next, 1);
          sh.fetch = (k < g.j1 - g.j0 && !sh.err) ? g.order[k] : -1;
        }
        epi_bar<kEpiThreads>();
        const int J = sh.fetch;
        epi_bar<kEpiThreads>();
        if (J < 0) {
          if (tid == 128) st.job = -1;
          break;
        }
        if constexpr (kMode == 1) {
          start_inverse(s, J);
          break;
        }
        if (g.cond && g.prep_status[J] == kSubOk && g.cond[J] > g.cond_max && g.sub_n[J] <= g.ill_max_n) continue;
        if (g.prep_status[J] != kSubOk) {
          if (tid == 128) {
            g.status[J] = g.prep_status[J];
            g.iters[J] = 0;
            g.rsteps[J] = 0;
            g.tS[J] = 0.0;
            g.tH[J] = 0.0;
          }
          continue;
        }
        const int n = g.sub_n[J], n64 = (n + 63) & ~63, R = (n + 127) & ~127;
        const float* A = g.A + g.a_off[J];
        const double alpha = scale_alpha(g.lam, g.lam_g, J, g.mu);
        const float inv = (float)(1.0 / alpha), fmu = (float)g.mu;
        uint16_t* hi = g.planes + (size_t)(sub0 + s) * kPps * plane_elems;
        uint16_t* lo = hi + plane_elems;
        const Fmt f = g.main_fmt;
        if (f.fmt == FMT_E4M3) {
          // one-byte view: X_0 * 2^7 in E4M3 over whole 128-byte K slices, and zeros in the K padding of
          // the other X plane and of T (their products write only the first n64 columns)
          const int k8 = k8_extent(n64);
          uint8_t* p8 = reinterpret_cast<uint8_t*>(hi);
          for (int e = etid; e < R * k8; e += kEpiThreads) {
            const int i = e / k8, j = e - i * k8;
            float x = 0.0f;
            if (i < n && j < n) x = (A[(size_t)i * n + j] - (i == j ? fmu : 0.0f)) * inv;
            p8[(size_t)i * 2 * g.LD + j] = (uint8_t)__nv_cvt_float_to_fp8(kF8Up * x, __NV_SATFINITE, __NV_E4M3);
            if (j >= n64) {
              p8[2 * 2 * plane_elems + (size_t)i * 2 * g.LD + j] = 0;   // X_1
              p8[4 * 2 * plane_elems + (size_t)i * 2 * g.LD + j] = 0;   // T
            }
          }
        } else {
          // four rows per warp pass, 8 consecutive columns per lane (all 32 loads in flight together, then
          // 16-byte stores of hi and lo); rows and columns n..n64 are the zero padding; rows from n64 on
          // only feed product rows that are never read back
          for (int i0 = 4 * (warp - 4); i0 < n64; i0 += 4 * kEpiWarps) {
            for (int j0 = 8 * lane; j0 < n64; j0 += 256) {
              float v[4][8];
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const int i = i0 + r;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  const int j = j0 + u;
                  v[r][u] = (i < n && j < n) ? (A[(size_t)i * n + j] - (i == j ? fmu : 0.0f)) * inv : 0.0f;
                }
              }
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const int i = i0 + r;
                if (i >= n64) break;
                uint32_t h[4], l[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) split2(v[r][2 * u], v[r][2 * u + 1], f.fmt, h[u], l[u]);
                *reinterpret_cast<uint4*>(hi + (size_t)i * g.LD + j0) = make_uint4(h[0], h[1], h[2], h[3]);
                if (f.terms > 1)
                  *reinterpret_cast<uint4*>(lo + (size_t)i * g.LD + j0) = make_uint4(l[0], l[1], l[2], l[3]);
              }
            }
          }
        }
        if (tid == 128) {
          st.job = J;
          st.n = n; st.n64 = n64; st.R = R;
          st.nrb = R / 128; st.ncb = (n64 + kTileN - 1) / kTileN; st.nks = n64 / 64;
          st.kind = 0; st.cur = 0;
          st.phase = 0; st.refine_left = g.refine_steps; st.steps = 0; st.rsteps = 0;
          st.status = kSubNotConv; st.last = 0;
          st.dprev = INFINITY;
          st.fcur = g.main_fmt; st.fnxt = g.main_fmt;
        }
        break;
      }
      tc::fence_proxy_async_global();
      tc::mbar_arrive(&sh.epi_done[s]);
    };

    // a7 for the finished submatrix of slot s: centre columns of T_J(D) = 1/2 (I - X) T_J(S)^-1 and the
    // FP64 partial traces
    auto finish_slot = [&](int s) {
      epi_bar<kEpiThreads>();   // the slot state written by thread 128 and the final X of every group are visible
      SlotState& st = sh.slot[s];
      const int J = st.job, n = st.n, b = g.nbf[J];
      // the final X_k, hi (+ lo) in the last product's output format
      const uint16_t* xh = g.planes + ((size_t)(sub0 + s) * kPps + 2 * st.cur) * plane_elems;
      const uint16_t* xl = xh + plane_elems;
      const Fmt xfmt = st.fcur;
      const double* Q = g.Q + g.c_off[J];
      const double* Sc = g.Sc + g.c_off[J];
      const double* Hc = g.Hc + g.c_off[J];
      double* Dc = g.Dc + g.c_off[J];
      // X Q with one row of X per lane (32 consecutive rows per warp), Q in FP32 in the staging buffers (idle
      // between products), zero padded to bp = 8 ceil(b / 8) columns and n64 rows so that the inner loop has
      // no conditions; the sums (hi, lo) then go through shared memory to the FP64 step, which runs
      // element by element. Larger cases take the same sums with Q read from global memory.
      const int n64 = st.n64, bp = (b + 7) & ~7;
      float* Qs = reinterpret_cast<float*>(stg);
      const size_t qs_bytes = (size_t)n64 * bp * sizeof(float);
      const bool fast = qs_bytes + (size_t)n * b * sizeof(float2) <= kStgTotal;
      float2* Ps = reinterpret_cast<float2*>(stg + qs_bytes);
      double ps = 0.0, ph = 0.0;
      if (fast) {
        for (int e = etid; e < n64 * bp; e += kEpiThreads) {
          const int k = e / bp, c = e - k * bp;
          Qs[e] = (k < n && c < b) ? (float)Q[(size_t)k * b + c] : 0.0f;
        }
        epi_bar<kEpiThreads>();
        for (int i0 = 32 * (warp - 4); i0 < n; i0 += kEpiThreads) {
          const int i = i0 + lane;
          const size_t ro = (size_t)(i < n ? i : 0) * g.LD;
          for (int cg = 0; cg < b; cg += 8) {
            float sh_[8], sl_[8];
            if (xfmt.fmt == FMT_BF16) {
              if (xfmt.terms > 1) xq_row<FMT_BF16, true>(xh + ro, xl + ro, n64, Qs + cg, bp, sh_, sl_);
              else xq_row<FMT_BF16, false>(xh + ro, xl + ro, n64, Qs + cg, bp, sh_, sl_);
            } else {
              if (xfmt.terms > 1) xq_row<FMT_F16, true>(xh + ro, xl + ro, n64, Qs + cg, bp, sh_, sl_);
              else xq_row<FMT_F16, false>(xh + ro, xl + ro, n64, Qs + cg, bp, sh_, sl_);
            }
            if (i < n) {
#pragma unroll
              for (int c = 0; c < 8; ++c)
                if (cg + c < b) Ps[(size_t)i * b + cg + c] = make_float2(sh_[c], sl_[c]);
            }
          }
        }
        epi_bar<kEpiThreads>();
        for (int e = etid; e < n * b; e += kEpiThreads) {
          const float2 p = Ps[e];
          const double dv = 0.5 * (Q[e] - ((double)p.x + (double)p.y));
          Dc[e] = dv;
          ps += dv * Sc[e];
          ph += dv * Hc[e];
        }
      } else {
        for (int e = etid; e < n * b; e += kEpiThreads) {
          const int i = e / b, c = e - i * b;
          float sum = 0.0f, cmp = 0.0f;
          for (int k = 0; k < n; ++k) {
            const float x = from_bits(xh[(size_t)i * g.LD + k], xfmt.fmt) +
                            (xfmt.terms > 1 ? from_bits(xl[(size_t)i * g.LD + k], xfmt.fmt) : 0.0f);
            const float qv = (float)Q[(size_t)k * b + c];
            const float p = x * qv;
            cmp += fmaf(x, qv, -p);
            two_sum(sum, cmp, p);
          }
          const double dv = 0.5 * (Q[e] - ((double)sum + (double)cmp));
          Dc[e] = dv;
          ps += dv * Sc[e];
          ph += dv * Hc[e];
        }
      }
      double px = 0.0;   // the trace of the final X: (n - Tr X) / 2 eigenvalues lie below mu
      for (int i = etid; i < n; i += kEpiThreads) {
        float x = from_bits(xh[(size_t)i * g.LD + i], xfmt.fmt);
        if (xfmt.terms > 1) x += from_bits(xl[(size_t)i * g.LD + i], xfmt.fmt);
        px += x;
      }
      for (int o = 16; o > 0; o >>= 1) {
        ps += __shfl_xor_sync(0xffffffffu, ps, o);
        ph += __shfl_xor_sync(0xffffffffu, ph, o);
        px += __shfl_xor_sync(0xffffffffu, px, o);
      }
      if (lane == 0) {
        sh.dred[0][warp - 4] = ps;
        sh.dred[1][warp - 4] = ph;
        sh.dred[2][warp - 4] = px;
      }
      epi_bar<kEpiThreads>();
      if (tid == 128) {
        double ts = 0.0, th = 0.0, tx = 0.0;
        for (int w = 0; w < kEpiWarps; ++w) {
          ts += sh.dred[0][w];
          th += sh.dred[1][w];
          tx += sh.dred[2][w];
        }
        if (g.nbelow) g.nbelow[J] = (int32_t)lrint(0.5 * (n - tx));
        int stt = st.status;
        if (stt == kSubOk && !(isfinite(ts) && isfinite(th))) stt = kSubNonFinite;
        g.tS[J] = ts;
        g.tH[J] = th;
        g.iters[J] = st.steps;
        g.rsteps[J] = st.rsteps;
        g.status[J] = stt;
      }
      epi_bar<kEpiThreads>();   // staging and dred free again
    };

    for (int c = 0; c < kSlots; ++c) start_slot(c);
    for (uint32_t i = 0;; ++i) {
      // every epilogue thread waits for the descriptor; a wait that ran out in any of them ends all
      const bool got = tc::mbar_wait(&sh.desc_full[i % kRing], (i / kRing) & 1, tc::globaltimer() + 8 * g.wait_ns);
      if (epi_bar_or<kEpiThreads>(!got || sh.err)) {
        if (tid == 128) sh.err = 1;
        break;
      }
      const Desc d = sh.ring[i % kRing];
      if (d.term) break;
      SlotState& st = sh.slot[d.slot];
      const int n = d.n, n64 = d.n64;
      // the sign iteration's epilogues are fixed by the product kind (no descriptor fields needed)
      const int epi = kMode == 0 ? (d.kind == 0 ? kEpiT : kEpiScale) : d.epi;
      const float escale = kMode == 0 ? 0.5f : (epi == kEpiA ? 1.0f : d.scale);
      float part = 0.0f;
      bool bad = false;   // a wait of this warp ran out: keep the barrier schedule, skip the work
      for (int mb = 0; mb < d.nrb; ++mb)
        for (int cb = 0; cb < d.ncb; ++cb) {
          const int nt = min(kTileN, n64 - kTileN * cb);
          const int buf = tcount & 1;
          if (!bad) bad = !tc::mbar_wait(&sh.accf[buf], (tcount >> 1) & 1, tc::globaltimer() + g.wait_ns);
          bad = __any_sync(0xffffffffu, bad);   // tcgen05.ld needs the whole warp
          tc::tc_fence_after();
          // an M = 64 tile: 16 rows per warp quarter, in its lanes 0-15
          const bool m64 = tail64(d, mb);
          const int rbase = 128 * mb + (m64 ? 16 : 32) * q;
          const int row = rbase + lane;
          const bool rok = !m64 || lane < 16;
          const bool live = rbase < n64 && !bad;   // rows >= n64 are never read back
          const int nch = nt / 32;
          const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * 256;
          uint32_t r[32];
          if (live && grp < nch) tc::tmem_ld32(taddr + 32 * grp, r);
          // E4M3 operand scales; and the factor of the inverse mode's Z before its first update
          const float sc = (d.f.fmt == FMT_E4M3 ? kF8Down : 1.0f) * (kMode == 1 && epi == kEpiT ? d.pscale : 1.0f);
          for (int c0 = grp; c0 < nch; c0 += kGroups) {
            const int col0 = kTileN * cb + 32 * c0;
            float v[32];
            if (live) {
              tc::tmem_wait_ld();
              // entries past n are written as zeros: the trimmed products leave the accumulator's columns
              // past n16 as they were, and the next products' K and N never reach past n16
              // a chunk inside the n columns that holds none of the warp's diagonal entries takes the short
              // path (warp-uniform test): rows past n through a zero factor, no test per entry
              const bool rin = rok && row < n;
              const bool inner = col0 + 32 <= n && col0 != (rbase & ~31);
              if (epi == kEpiT) {
                if (inner) {
                  const float s = rin ? sc : 0.0f;
                  float q4[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // four partial sums: a dependence chain of 8, not 32
#pragma unroll
                  for (int j = 0; j < 32; ++j) {
                    const float p = s * __uint_as_float(r[j]);   // P_ij, off the diagonal: (I - P)_ij = -p
                    q4[j & 3] = fmaf(p, p, q4[j & 3]);
                    v[j] = -p;                                   // (3I - P)_ij
                  }
                  part += (q4[0] + q4[1]) + (q4[2] + q4[3]);
                } else {
#pragma unroll
                  for (int j = 0; j < 32; ++j) {
                    const int col = col0 + j;
                    const bool in = rin && col < n;
                    const float e = (row == col ? 1.0f : 0.0f) - sc * __uint_as_float(r[j]);  // (I - P)_ij
                    if (in) part += e * e;
                    v[j] = in ? e + (row == col ? 2.0f : 0.0f) : 0.0f;                 // (3I - P)_ij
                  }
                }
              } else {
                const float m = escale * sc;
                if (col0 + 32 <= n) {
                  const float mr = rin ? m : 0.0f;
#pragma unroll
                  for (int j = 0; j < 32; ++j) v[j] = mr * __uint_as_float(r[j]);
                } else {
#pragma unroll
                  for (int j = 0; j < 32; ++j) v[j] = (rin && col0 + j < n) ? m * __uint_as_float(r[j]) : 0.0f;
                }
              }
              if (c0 + kGroups < nch) tc::tmem_ld32(taddr + 32 * (c0 + kGroups), r);   // overlaps this chunk's work
            }
            if (kMode == 1 && live && epi >= kEpiX) {
              // inverse mode: X or A_J in FP32, row-major n x n. The chunk goes through the warp's staging
              // buffer (row = lane, entry j at j ^ lane: no bank conflicts either way) so that each store
              // instruction writes 32 consecutive entries of one row
              const int J = sh.slot[d.slot].job;
              float* dst = epi == kEpiX ? g.Xout + (g.a_off[J] - g.a_base) : g.Aout + g.a_off[J];
              float* wf = reinterpret_cast<float*>(stg + (size_t)(warp - 4) * 4096);
              if (lane == 0) tc::bulk_wait_read<0>();   // this warp's previous store has read the buffer
              __syncwarp();
#pragma unroll
              for (int j = 0; j < 32; ++j) wf[lane * 32 + (j ^ lane)] = v[j];
              __syncwarp();
              const int nr = m64 ? 16 : 32;
              for (int rr = 0; rr < nr; ++rr) {
                const int orow = rbase + rr;
                if (orow < n && col0 + lane < n) dst[(size_t)orow * n + col0 + lane] = wf[rr * 32 + (lane ^ rr)];
              }
              __syncwarp();   // the staging is free again
            }
            if (kMode == 1 && epi == kEpiA) {
              // no operand to write
            } else if (d.fo.fmt == FMT_E4M3) {
              // E4M3 output (scaled by 2^7): this thread's 32 bytes of the row, two 16-byte stores into the
              // one-byte view of the plane (rows of 2 LD bytes)
              if (live) {
                uint32_t w8[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const uint32_t p0 = __nv_cvt_float2_to_fp8x2(make_float2(kF8Up * v[4 * j], kF8Up * v[4 * j + 1]),
                                                               __NV_SATFINITE, __NV_E4M3);
                  const uint32_t p1 = __nv_cvt_float2_to_fp8x2(make_float2(kF8Up * v[4 * j + 2], kF8Up * v[4 * j + 3]),
                                                               __NV_SATFINITE, __NV_E4M3);
                  w8[j] = p0 | (p1 << 16);
                }
                uint8_t* dst = reinterpret_cast<uint8_t*>(g.planes) + (size_t)d.zo * plane_elems * 2 +
                               (size_t)row * (2 * g.LD) + col0;
                reinterpret_cast<uint4*>(dst)[0] = make_uint4(w8[0], w8[1], w8[2], w8[3]);
                reinterpret_cast<uint4*>(dst)[1] = make_uint4(w8[4], w8[5], w8[6], w8[7]);
              }
            } else if (live) {
              // each warp stores its own 32 rows x 32 columns through its own 4 KB staging buffer (hi rows, then
              // lo rows; 64-byte swizzle: 16-byte unit c of row r at unit c ^ ((r >> 1) & 3)), with one TMA
              // tensor store issued by its lane 0 for both planes (a box two planes deep): no barrier between
              // warps, one store per chunk. An M = 64 tile has 16 rows per warp: its lo rows follow its 16 hi
              // rows, and the 16-row box reads them there.
              uint32_t h[16], l[16];
              split_pack(v, d.fo, h, l);
              uint8_t* wb = stg + (size_t)(warp - 4) * 4096;
              if (lane == 0) tc::bulk_wait_read<0>();   // this warp's previous store has read the buffer
              __syncwarp();
              if (rok) {
                uint4* dh = reinterpret_cast<uint4*>(wb + lane * 64);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                  dh[c ^ ((lane >> 1) & 3)] = make_uint4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3]);
                if (d.fo.terms > 1) {
                  uint4* dl = reinterpret_cast<uint4*>(wb + (m64 ? 1024 : 2048) + lane * 64);
#pragma unroll
                  for (int c = 0; c < 4; ++c)
                    dl[c ^ ((lane >> 1) & 3)] = make_uint4(l[4 * c], l[4 * c + 1], l[4 * c + 2], l[4 * c + 3]);
                }
              }
              tc::fence_proxy_async_smem();
              __syncwarp();
              if (lane == 0) {
                const CUtensorMap* ms = d.fo.terms > 1 ? (m64 ? &mapS16x2 : &mapS2) : (m64 ? &mapS16 : &mapS);
                tc::tma_store_3d(ms, wb, col0, rbase, d.zo);
                tc::bulk_commit();
              }
            }
          }
          tc::tc_fence_before();
          if (!bad) tc::mbar_arrive(&sh.acce[buf]);
          ++tcount;
        }
      if (lane == 0) tc::bulk_wait<0>();   // this warp's stores are written before anyone reads them
      tc::fence_proxy_async_global();
      // ---- end of the product: one uniform error decision, then the slot's next state
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) sh.red[i & 1][warp - 4] = part;
      if (epi_bar_or<kEpiThreads>(bad)) {
        if (tid == 128) sh.err = 1;
        break;
      }
      if (kMode == 1 && tid == 128) {
        // inverse mode: the next product of the slot
        switch (d.kind) {
          case 0: {
            float dsum = 0.0f;
            for (int w = 0; w < kEpiWarps; ++w) dsum += sh.red[i & 1][w];
            const float dd = sqrtf(dsum / (float)n);
            st.steps += 1;
            if (!isfinite(dd) || (dd > g.tol_inv && st.steps >= g.max_inv)) {
              st.status = kSubRefine;   // diverged or too slow: the FP64 preparation takes it
              st.last = 1;
            } else if (dd <= g.tol_inv) {
              st.last = 1;                // this step's Z update is the last product of the iteration
            }
            st.kind = st.last ? 2 : 1;
            break;
          }
          case 1:   // after Y's update: Z's, unless the step's Z update was made at the start
            if (st.ncb != 1) st.yc = st.yc == 0 ? 3 : 0;
            st.kind = st.zdone ? 0 : 2;
            st.zdone = 0;
            break;
          case 2: st.zc = st.zc == 1 ? 4 : 1; st.zs = 1.0f; st.kind = st.last ? 3 : 0; break;
          case 3: st.kind = 4; break;
          default: break;
        }
      }
      if (kMode == 1 && d.kind == 2 && st.last) {
        // the iteration's last Z update is done: T_J(H0) into Y's pair (Y was last read by this step's
        // V = Z Y) for A_J = X T_J(H0), written now so that it is not held through the iteration
        const int J = st.job;
        const double* H = g.ws + (g.a_off[J] - g.a_base) + g.chunk_n2;
        uint16_t* yp = g.planes + ((size_t)(sub0 + d.slot) * kPps + 2 * st.yc) * plane_elems;
        fill_pair(yp, n, n64, H);
      }
      if (kMode == 0 && tid == 128) {
        if (d.kind == 0) {
          // defect of X_step and the decision about the following steps
          float dsum = 0.0f;
          for (int w = 0; w < kEpiWarps; ++w) dsum += sh.red[i & 1][w];
          const float dd = sqrtf(dsum / (float)n);
          const int steps = st.steps + 1;
          if (st.phase == 1) st.rsteps += 1;   // this step ran in the refinement format
          int last_ = 0, status = kSubNotConv;
          Fmt nxt = st.fcur;
          if (!isfinite(dd)) {
            last_ = 1;
            status = kSubNonFinite;
          } else if (st.phase == 0) {
            // E4M3 iterates carry a rounding error of up to 2^-4 relative, which holds the defect at a floor
            // near 0.05, well above tol_ns: their phase ends at twice that floor, or when the defect has
            // stopped falling (below 0.25, where the exact iteration would at least halve it every step)
            const bool f8_end = st.fcur.fmt == FMT_E4M3 && (dd <= kF8Switch || (dd < 0.25f && dd > 0.5f * st.dprev));
            if (dd <= g.tol_ns || f8_end) {
              if (g.refine_steps == 0) {
                last_ = 1;
                status = dd <= g.tol_accept ? kSubOk : kSubNotConv;
              } else {
                st.phase = 1;
                st.refine_left = g.refine_steps;
                nxt = g.refine_fmt;
              }
            }
          } else if (--st.refine_left <= 0) {
            if (dd <= g.tol_accept) {
              last_ = 1;
              status = kSubOk;
            } else if (dd < st.dprev) {
              st.refine_left = 1;   // still converging: one more step (bounded by the step cap below)
            } else {
              last_ = 1;
              status = kSubNotConv;
            }
          }
          const int cap = g.budget ? min(g.max_iter, g.budget[st.job]) : g.max_iter;
          if (!last_ && steps >= cap) {
            last_ = 1;
            status = kSubNotConv;
          }
          st.dprev = dd;
          st.steps = steps;
          st.last = last_;
          st.status = status;
          st.fnxt = nxt;
          st.kind = 1;
        } else {
          // after X T: X_{k+1} is the current X (ping-pong unless written in place), in the next format
          if (d.ncb != 1) st.cur ^= 1;
          st.fcur = st.fnxt;
          st.kind = 0;
        }
      }
      if (d.last) {
        if constexpr (kMode == 1) {
          if (tid == 128) {
            const SlotState& sf = sh.slot[d.slot];
            g.prep_out[sf.job] = sf.status;
            const double n3 = (double)sf.n * sf.n * sf.n;
            // step 0 needs one product (Y_1), every further step three but the last two (no Y update); then X, A
            const double prods = 3.0 * sf.steps - 1.0;
            atomicAdd(&g.flops[0], 2.0 * n3 * prods);
            atomicAdd(&g.flops[1], 6.0 * n3 * prods);
          }
        } else {
          finish_slot(d.slot);
        }
        start_slot(d.slot);
      } else {
        tc::mbar_arrive(&sh.epi_done[d.slot]);
      }
    }
    if (sh.err && tid == 128) {
      // a wait ran out: the submatrices in flight are reported as timed out
      for (int s = 0; s < kSlots; ++s) {
        const int J = sh.slot[s].job;
        if (J >= 0 && kMode == 1) {
          g.prep_out[J] = kSubTimeout;
        } else if (J >= 0) {
          g.status[J] = kSubTimeout;
          g.iters[J] = sh.slot[s].steps;
          g.rsteps[J] = sh.slot[s].rsteps;
          g.tS[J] = 0.0;
          g.tH[J] = 0.0;
        }
      }
      atomicExch(g.err, 1);
    }
  }
  }

  // every role has left its loop, so sh.err is final; after a timeout wait (bounded) for this CTA's
  // TMA loads and MMAs still in flight before the shared and tensor memory are released
  __syncthreads();
  if (sh.err) {
    if (warp == 0 && lane == 0)
      for (int s = 0; s < kStages; ++s)
        if (armed[s]) tc::mbar_wait(&sh.full[s], arm_phase[s], tc::globaltimer() + 50000000ull);
    if (warp == 1 && lane == 0) {
      tc::mma_commit(&sh.idle);
      tc::mbar_wait(&sh.idle, 0, tc::globaltimer() + 50000000ull);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Every submatrix of the launch starts as "timed out": the sign kernel overwrites the status of each one it
// takes, so a submatrix that no block reached (every block gave up on a bounded wait) is reported as such
// instead of keeping the status of an earlier solve.
__global__ void k_status_pending(int32_t j0, int32_t count, const int32_t* __restrict__ list,
                                 int32_t* __restrict__ status) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
    status[list ? list[e] : j0 + e] = kSubTimeout;
}

}  // namespace

// ==================================================================================== host side

struct TcState {
  DevBuf planes, order, err;
  int R = 0, LD = 0, slots = 0;
  int64_t ord_j0 = -1, ord_j1 = -1;
  int32_t ord_large = 0;          // how many of the cached order (a prefix) have n above 192
  DevBuf inv_planes, inv_flops;   // inverse mode: its own plane layout (kPlanesInv per slot), flop sums
  int iR = 0, iLD = 0, islots = 0;
};

static TcState* state(nolsm_plan* plan) {
  if (!plan->tc) plan->tc = new TcState();
  return static_cast<TcState*>(plan->tc);
}

void tc_release(nolsm_plan* plan) {
  if (!plan->tc) return;
  TcState* s = static_cast<TcState*>(plan->tc);
  dev_free(plan, s->planes);
  dev_free(plan, s->order);
  dev_free(plan, s->err);
  dev_free(plan, s->inv_planes);
  dev_free(plan, s->inv_flops);
  delete s;
  plan->tc = nullptr;
}

int main_terms(int precision) {
  return precision == NOLSM_FP32 || precision == NOLSM_BF16X3 ? 3 : 1;
}

static bool formats(int precision, Fmt* main_fmt, Fmt* refine_fmt) {
  *refine_fmt = Fmt{FMT_F16, 3};
  switch (precision) {
    case NOLSM_FP32: *main_fmt = Fmt{FMT_F16, 3}; return true;
    case NOLSM_BF16X3: *main_fmt = Fmt{FMT_BF16, 3}; return true;
    case NOLSM_BF16: *main_fmt = Fmt{FMT_BF16, 1}; return true;
    case NOLSM_FP8E4M3: *main_fmt = Fmt{FMT_E4M3, 1}; return true;
    case NOLSM_FP16: *main_fmt = Fmt{FMT_F16, 1}; return true;
    default: return false;
  }
}

// The inverse kernel's register split (setmaxnreg) assumes the launch gives each of its 512 threads
// kRegsLaunch registers; with fewer, the epilogue warpgroups' increase could never be granted, so the launch
// is refused.
static nolsm_status check_register_split(const void* fn) {
  cudaFuncAttributes at{};
  NOLSM_CUDA_TRY(cudaFuncGetAttributes(&at, fn));
  if (at.numRegs != kRegsLaunch) {
    set_error("k_ns_tc was built with %d registers per thread; its register split needs exactly %d", at.numRegs,
              kRegsLaunch);
    return NOLSM_ERR_UNSUPPORTED;
  }
  return NOLSM_OK;
}

// ------------------------------------------------------------------ launch shapes and their tuner

using TcKernel = decltype(&k_ns_tc<0, 0>);
struct TcMaps { CUtensorMap mA, mB, mS, mA8, mB8, mS16, mS2, mS16x2; };

static TcKernel tc_kernel(int mode, int shape) {
  if (mode == 0) return shape == 0 ? &k_ns_tc<0, 0> : &k_ns_tc<0, 1>;
  return shape == 0 ? &k_ns_tc<1, 0> : &k_ns_tc<1, 1>;
}

// One launch of kernel (mode, shape) over the submatrices g.order[0, g.j1) (g.j0 = 0): one CTA per SM at most,
// kSlots submatrices in flight in each; the work counter is reset first.
static nolsm_status launch_shape(int mode, int shape, const TcMaps& m, const TcArgs& g, int sms, cudaStream_t st) {
  const TcKernel k = tc_kernel(mode, shape);
  const int threads = shape == 0 ? Shape<0>::kThreads : Shape<1>::kThreads;
  const int smem = shape == 0 ? Shape<0>::kSmemBytes : Shape<1>::kSmemBytes;
  NOLSM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  if (shape == 1) NOLSM_TRY(check_register_split(reinterpret_cast<const void*>(k)));
  NOLSM_CUDA_TRY(cudaMemsetAsync(g.next, 0, sizeof(int32_t), st));
  const int ctas = (int)std::min<int64_t>(sms, ((int64_t)g.j1 + kSlots - 1) / kSlots);
  k<<<ctas, threads, smem, st>>>(m.mA, m.mB, m.mS, m.mA8, m.mB8, m.mS16, m.mS2, m.mS16x2, g);
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}

// The launch shape of each (mode, precision, bucket) as measured in this process (-1: not yet), and the
// environment variable NOLSM_TC_SHAPE ("0" or "1") that fixes it instead.
static std::mutex g_shape_mu;
static int g_shape[2][8][2] = {{{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}},
                               {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}}};

static int env_shape() {
  const char* e = std::getenv("NOLSM_TC_SHAPE");
  if (e && (e[0] == '0' || e[0] == '1') && e[1] == 0) return e[0] - '0';
  return -1;
}

// The launch shape of one bucket of submatrices, order[0, count) (all with n above 192, or all at most 192):
// the one NOLSM_TC_SHAPE fixes, else the one measured faster for (mode, precision, bucket) in this process. The
// first time, both shapes run on the bucket's largest submatrices (32 per slot of every SM: with fewer, the
// start and the tail of the launch decide; the shapes differ by 3-40 % in steady state), timed with CUDA
// events on the stream, and the faster is kept (not when a bounded wait ran out in the measurement); the
// results of those runs are computed again by the launches that follow. pending(order, count) resets the
// statuses of the submatrices a launch takes.
template <typename Pending>
static nolsm_status bucket_shape(int mode, int precision, int bucket, bool fixed0, const TcMaps& m, TcArgs g,
                                 const int32_t* order, int32_t count, int sms, cudaStream_t st, Pending pending,
                                 int* out) {
  int shape = fixed0 ? 0 : env_shape();
  const int pi = precision & 7;
  if (shape < 0) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    shape = g_shape[mode][pi][bucket];
  }
  if (shape < 0) {
    g.j0 = 0;
    g.order = order;
    const int32_t sample = std::min<int32_t>(count, 32 * kSlots * sms);
    struct Events {   // destroyed on every way out
      cudaEvent_t e[2] = {nullptr, nullptr};
      ~Events() {
        for (cudaEvent_t x : e)
          if (x) cudaEventDestroy(x);
      }
    } ev;
    float ms[2] = {0.0f, 0.0f};
    NOLSM_CUDA_TRY(cudaEventCreate(&ev.e[0]));
    NOLSM_CUDA_TRY(cudaEventCreate(&ev.e[1]));
    for (int sh = 0; sh < 2; ++sh) {
      g.j1 = sample;
      NOLSM_TRY(pending(order, sample));
      NOLSM_CUDA_TRY(cudaEventRecord(ev.e[0], st));
      NOLSM_TRY(launch_shape(mode, sh, m, g, sms, st));
      NOLSM_CUDA_TRY(cudaEventRecord(ev.e[1], st));
      NOLSM_CUDA_TRY(cudaEventSynchronize(ev.e[1]));
      NOLSM_CUDA_TRY(cudaEventElapsedTime(&ms[sh], ev.e[0], ev.e[1]));
    }
    int32_t errf = 0;
    NOLSM_CUDA_TRY(cudaMemcpyAsync(&errf, g.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
    if (errf != 0) {
      shape = 0;
    } else {
      shape = ms[1] < ms[0] ? 1 : 0;
      std::lock_guard<std::mutex> lk(g_shape_mu);
      g_shape[mode][pi][bucket] = shape;
    }
  }
  *out = shape;
  return NOLSM_OK;
}

// Runs the submatrices order[0, count), largest first, of which the first n_large have n above 192: each bucket
// in its shape (bucket_shape), as one launch over both when the shapes agree (no second launch tail), else one
// launch per bucket.
template <typename Pending>
static nolsm_status run_buckets(int mode, int precision, bool fixed0, const TcMaps& m, TcArgs g, const int32_t* order,
                                int32_t n_large, int32_t count, int sms, cudaStream_t st, Pending pending) {
  if (count <= 0) return NOLSM_OK;
  int s1 = -1, s0 = -1;
  if (n_large > 0) NOLSM_TRY(bucket_shape(mode, precision, 1, fixed0, m, g, order, n_large, sms, st, pending, &s1));
  if (count > n_large)
    NOLSM_TRY(bucket_shape(mode, precision, 0, fixed0, m, g, order + n_large, count - n_large, sms, st, pending, &s0));
  g.j0 = 0;
  if (n_large == 0 || n_large == count || s1 == s0) {
    g.order = order;
    g.j1 = count;
    NOLSM_TRY(pending(order, count));
    return launch_shape(mode, n_large > 0 ? s1 : s0, m, g, sms, st);
  }
  g.order = order;
  g.j1 = n_large;
  NOLSM_TRY(pending(order, n_large));
  NOLSM_TRY(launch_shape(mode, s1, m, g, sms, st));
  g.order = order + n_large;
  g.j1 = count - n_large;
  NOLSM_TRY(pending(order + n_large, count - n_large));
  return launch_shape(mode, s0, m, g, sms, st);
}

int tc_shape_choice(int mode, int precision, int bucket) {
  if (mode < 0 || mode > 1 || bucket < 0 || bucket > 1) return -1;
  std::lock_guard<std::mutex> lk(g_shape_mu);
  return g_shape[mode][precision & 7][bucket];
}

nolsm_status solve_tc(nolsm_plan* plan, double mu, const nolsm_options& o, int64_t j0, int64_t j1, const SolveSpec& spec,
                      cudaStream_t st) {
  Fmt mf, rf;
  if (!formats(o.precision, &mf, &rf)) {
    set_error("precision %d is not available on the tensor-core path in this build", o.precision);
    return NOLSM_ERR_UNSUPPORTED;
  }
  if (mf.fmt == FMT_E4M3 && o.refine_steps < 1) {
    set_error("E4M3 needs at least one refinement step (the centre-column phase reads a 2-byte X)");
    return NOLSM_ERR_UNSUPPORTED;
  }
  NOLSM_TRY(ensure_results(plan));
  TcState* S = state(plan);
  int dev = 0, sms = 0;
  NOLSM_CUDA_TRY(cudaGetDevice(&dev));
  NOLSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int32_t maxn = 0;
  for (int64_t J = j0; J < j1; ++J) maxn = std::max(maxn, plan->h_sub_n[J]);
  const int LD = (maxn + 63) & ~63, R = (maxn + 127) & ~127;
  // one CTA per SM at most, each with kSlots submatrices in flight (one scratch sub-slot each)
  const int64_t work = spec.list ? spec.count : j1 - j0;
  if (work <= 0) return NOLSM_OK;
  const int ctas = (int)std::min<int64_t>(sms, (work + kSlots - 1) / kSlots);
  const int slots = ctas * kSlots;
  if (!S->planes.p || S->R < R || S->LD < LD || S->slots < slots) {
    const int nR = std::max(R, S->R), nLD = std::max(LD, S->LD), nS = std::max(slots, S->slots);
    dev_free(plan, S->planes);
    NOLSM_TRY(dev_alloc(plan, S->planes, sizeof(uint16_t) * (size_t)kPlanes * nS * nR * nLD));
    S->R = nR;
    S->LD = nLD;
    S->slots = nS;
  }
  if (!S->err.p) NOLSM_TRY(dev_alloc(plan, S->err, sizeof(int32_t) * 4));
  if (S->ord_j0 != j0 || S->ord_j1 != j1) {
    std::vector<int32_t> ord((size_t)(j1 - j0));
    for (int64_t J = j0; J < j1; ++J) ord[(size_t)(J - j0)] = (int32_t)J;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return plan->h_sub_n[a] > plan->h_sub_n[b]; });
    if (S->order.bytes < sizeof(int32_t) * ord.size()) {
      dev_free(plan, S->order);
      NOLSM_TRY(dev_alloc(plan, S->order, sizeof(int32_t) * (size_t)plan->n_mol));
    }
    NOLSM_CUDA_TRY(cudaMemcpyAsync(S->order.p, ord.data(), sizeof(int32_t) * ord.size(), cudaMemcpyHostToDevice, st));
    NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
    S->ord_j0 = j0;
    S->ord_j1 = j1;
    S->ord_large = 0;
    while (S->ord_large < (int32_t)ord.size() && plan->h_sub_n[ord[(size_t)S->ord_large]] > 192) ++S->ord_large;
  }
  CUtensorMap mA, mB, mS, mS16, mS2, mS16x2;
  if (!tmap::make_3d(&mS16, S->planes.p, 2, (uint64_t)S->LD, (uint64_t)S->R, (uint64_t)S->slots * kPlanes, 32, 16,
                     CU_TENSOR_MAP_SWIZZLE_64B) ||
      !tmap::make_3d(&mS16x2, S->planes.p, 2, (uint64_t)S->LD, (uint64_t)S->R, (uint64_t)S->slots * kPlanes, 32, 16,
                     CU_TENSOR_MAP_SWIZZLE_64B, 2) ||
      !tmap::make_3d(&mS2, S->planes.p, 2, (uint64_t)S->LD, (uint64_t)S->R, (uint64_t)S->slots * kPlanes, 32, 32,
                     CU_TENSOR_MAP_SWIZZLE_64B, 2) ||
      !tmap::make_3d(&mA, S->planes.p, 2, (uint64_t)S->LD, (uint64_t)S->R, (uint64_t)S->slots * kPlanes, 64, 128) ||
      !tmap::make_3d(&mB, S->planes.p, 2, (uint64_t)S->LD, (uint64_t)S->R, (uint64_t)S->slots * kPlanes, 64, 64) ||
      !tmap::make_3d(&mS, S->planes.p, 2, (uint64_t)S->LD, (uint64_t)S->R, (uint64_t)S->slots * kPlanes, 32, 32,
                     CU_TENSOR_MAP_SWIZZLE_64B)) {
    set_error("cuTensorMapEncodeTiled rejected the scratch layout (R %d, LD %d, slots %d)", S->R, S->LD, S->slots);
    return NOLSM_ERR_CUDA;
  }
  NOLSM_CUDA_TRY(cudaMemsetAsync(plan->counter.p, 0, sizeof(int32_t), st));
  NOLSM_CUDA_TRY(cudaMemsetAsync(S->err.p, 0, sizeof(int32_t), st));
  TcArgs g{};
  if (spec.list) {   // an explicit work list (reruns): in list order
    g.j0 = 0; g.j1 = spec.count;
    g.order = spec.list;
  } else {
    g.j0 = (int32_t)j0; g.j1 = (int32_t)j1;
    g.order = S->order.as<int32_t>();
  }
  g.sub_n = plan->sub_n.as<int32_t>(); g.nbf = plan->sub_b.as<int32_t>();
  g.a_off = plan->a_off.as<int64_t>(); g.c_off = plan->c_off.as<int64_t>();
  // the symmetric form iterates on M and its centre-column phase uses W_c = L^-1 E_c in place of Q
  const bool sym = prep_class(o) == kPrepSym;
  g.A = prepared(plan, prep_class(o)).A.as<float>();
  g.Q = sym ? plan->Wc.as<double>() : plan->Q.as<double>();
  g.Sc = plan->Sc.as<double>(); g.Hc = plan->Hc.as<double>();
  g.lam = spec.lam ? spec.lam : plan->lam.as<double>();
  g.lam_g = plan->lam.as<double>();
  g.prep_status = plan->prep_status.as<int32_t>();
  g.mu = mu;
  g.tol_ns = (float)o.tol_ns; g.tol_accept = (float)o.tol_accept;
  g.max_iter = o.max_iter; g.refine_steps = o.refine_steps;
  g.budget = spec.budget;
  g.main_fmt = mf; g.refine_fmt = rf;
  g.planes = S->planes.as<uint16_t>();
  g.R = S->R; g.LD = S->LD;
  g.next = plan->counter.as<int32_t>();
  g.err = S->err.as<int32_t>();
  g.Dc = plan->Dc.as<double>(); g.tS = plan->t_S.as<double>(); g.tH = plan->t_H.as<double>();
  g.iters = plan->iters.as<int32_t>(); g.status = plan->status.as<int32_t>();
  g.rsteps = plan->rsteps.as<int32_t>();
  g.nbelow = plan->nbelow.as<int32_t>();
  g.wait_ns = o.wait_ns > 0 ? (uint64_t)o.wait_ns : kWaitNs;
  g.cond = sym ? nullptr : prepared(plan, prep_class(o)).cond.as<float>();
  g.cond_max = cond_max(o.precision);
  g.ill_max_n = prepare_fp64_max_n();
  // one-byte views of the same planes (rows of 2 LD bytes) for E4M3 operands, both loaded K-major (E4M3 runs
  // in shape 0, whose B box is 256 rows)
  TcMaps m{mA, mB, mS, {}, {}, mS16, mS2, mS16x2};
  if (!tmap::make_3d(&m.mA8, S->planes.p, 1, 2 * (uint64_t)S->LD, (uint64_t)S->R, (uint64_t)S->slots * kPlanes, 128, 128) ||
      !tmap::make_3d(&m.mB8, S->planes.p, 1, 2 * (uint64_t)S->LD, (uint64_t)S->R, (uint64_t)S->slots * kPlanes, 128,
                     Shape<0>::kTileN)) {
    set_error("cuTensorMapEncodeTiled rejected the one-byte scratch layout");
    return NOLSM_ERR_CUDA;
  }
  // every submatrix of a launch starts as "timed out" (k_status_pending), the kernel overwrites what it takes
  int32_t* status = plan->status.as<int32_t>();
  auto pending = [&](const int32_t* list, int32_t count) -> nolsm_status {
    k_status_pending<<<(unsigned)std::min<int64_t>(1024, ((int64_t)count + 255) / 256), 256, 0, st>>>(0, count, list,
                                                                                                        status);
    NOLSM_LAUNCH_CHECK();
    return NOLSM_OK;
  };
  const bool f8 = mf.fmt == FMT_E4M3;
  if (spec.list) {   // reruns: one launch in list order, shape 0
    NOLSM_TRY(pending(spec.list, spec.count));
    NOLSM_TRY(launch_shape(0, 0, m, g, sms, st));
  } else {           // the largest-first order in its two buckets: n above 192, the rest
    NOLSM_TRY(run_buckets(0, o.precision, f8, m, g, S->order.as<int32_t>(), S->ord_large, (int32_t)(j1 - j0), sms, st,
                          pending));
  }
  plan->stats.launches += 2;
  if (sym) {   // D_c = L^-T U and the traces
    SymArgs a;
    a.j0 = (int32_t)j0;
    a.list = spec.list;
    a.sub_n = plan->sub_n.as<int32_t>(); a.nbf = plan->sub_b.as<int32_t>();
    a.a_off = plan->a_off.as<int64_t>(); a.c_off = plan->c_off.as<int64_t>();
    a.prep_status = plan->prep_status.as<int32_t>();
    a.L = plan->Lsym.as<float>();
    a.Sc = plan->Sc.as<double>(); a.Hc = plan->Hc.as<double>();
    a.Dc = plan->Dc.as<double>(); a.tS = plan->t_S.as<double>(); a.tH = plan->t_H.as<double>();
    a.status = plan->status.as<int32_t>();
    NOLSM_TRY(launch_sym_finish(a, (int)work, maxn, plan->max_b, st));
    plan->stats.launches += 1;
  }
  return NOLSM_OK;
}

// a2-a3 on the tensor cores for the chunk's submatrices order[0, count) (gathered into args.ws): A_J into
// Aout, T_J(S)^-1 into Xout, prep_out[J] = kSubOk or kSubRefine. Adds the products' flops to the stats.
nolsm_status launch_ns_inverse(nolsm_plan* plan, const NsInvArgs& a, cudaStream_t st) {
  if (a.count <= 0) return NOLSM_OK;
  TcState* S = state(plan);
  int dev = 0, sms = 0;
  NOLSM_CUDA_TRY(cudaGetDevice(&dev));
  NOLSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int LD = (a.max_n + 63) & ~63, R = (a.max_n + 127) & ~127;
  const int ctas = (int)std::min<int64_t>(sms, (a.count + kSlots - 1) / kSlots);
  const int slots = ctas * kSlots;
  if (!S->inv_planes.p || S->iR < R || S->iLD < LD || S->islots < slots) {
    const int nR = std::max(R, S->iR), nLD = std::max(LD, S->iLD), nS = std::max(slots, S->islots);
    dev_free(plan, S->inv_planes);
    NOLSM_TRY(dev_alloc(plan, S->inv_planes, sizeof(uint16_t) * (size_t)kPlanesInv * nS * nR * nLD));
    S->iR = nR;
    S->iLD = nLD;
    S->islots = nS;
  }
  if (!S->err.p) NOLSM_TRY(dev_alloc(plan, S->err, sizeof(int32_t) * 4));
  if (!S->inv_flops.p) NOLSM_TRY(dev_alloc(plan, S->inv_flops, sizeof(double) * 2));
  const uint64_t depth = (uint64_t)S->islots * kPlanesInv;
  CUtensorMap mA, mB, mS, mS16, mS2, mS16x2;
  if (!tmap::make_3d(&mS16, S->inv_planes.p, 2, (uint64_t)S->iLD, (uint64_t)S->iR, depth, 32, 16,
                     CU_TENSOR_MAP_SWIZZLE_64B) ||
      !tmap::make_3d(&mS16x2, S->inv_planes.p, 2, (uint64_t)S->iLD, (uint64_t)S->iR, depth, 32, 16,
                     CU_TENSOR_MAP_SWIZZLE_64B, 2) ||
      !tmap::make_3d(&mS2, S->inv_planes.p, 2, (uint64_t)S->iLD, (uint64_t)S->iR, depth, 32, 32,
                     CU_TENSOR_MAP_SWIZZLE_64B, 2) ||
      !tmap::make_3d(&mA, S->inv_planes.p, 2, (uint64_t)S->iLD, (uint64_t)S->iR, depth, 64, 128) ||
      !tmap::make_3d(&mB, S->inv_planes.p, 2, (uint64_t)S->iLD, (uint64_t)S->iR, depth, 64, 64) ||
      !tmap::make_3d(&mS, S->inv_planes.p, 2, (uint64_t)S->iLD, (uint64_t)S->iR, depth, 32, 32,
                     CU_TENSOR_MAP_SWIZZLE_64B)) {
    set_error("cuTensorMapEncodeTiled rejected the inverse scratch layout (R %d, LD %d, slots %d)", S->iR, S->iLD,
              S->islots);
    return NOLSM_ERR_CUDA;
  }
  NOLSM_CUDA_TRY(cudaMemsetAsync(plan->counter.p, 0, sizeof(int32_t), st));
  NOLSM_CUDA_TRY(cudaMemsetAsync(S->err.p, 0, sizeof(int32_t), st));
  NOLSM_CUDA_TRY(cudaMemsetAsync(S->inv_flops.p, 0, sizeof(double) * 2, st));
  TcArgs g{};
  g.j0 = 0; g.j1 = a.count;
  g.order = a.order;
  g.sub_n = plan->sub_n.as<int32_t>(); g.nbf = plan->sub_b.as<int32_t>();
  g.a_off = plan->a_off.as<int64_t>(); g.c_off = plan->c_off.as<int64_t>();
  g.main_fmt = Fmt{FMT_F16, 3}; g.refine_fmt = g.main_fmt;
  g.planes = S->inv_planes.as<uint16_t>();
  g.R = S->iR; g.LD = S->iLD;
  g.next = plan->counter.as<int32_t>();
  g.err = S->err.as<int32_t>();
  g.ws = a.ws; g.a_base = a.a_base; g.chunk_n2 = a.chunk_n2;
  g.Aout = a.Aout; g.Xout = a.Xout; g.prep_out = a.prep_out;
  g.tol_inv = a.tol_inv; g.max_inv = a.max_inv;
  g.wait_ns = kWaitNs;
  g.flops = S->inv_flops.as<double>();
  // the largest-first order in its two buckets (n above 192, the rest), each in its tuned shape; every
  // submatrix of a launch starts as "timed out" and the kernel overwrites what it takes. (The first call in a process
  // also counts the flops of the shape measurements.)
  TcMaps m{mA, mB, mS, mA, mB, mS16, mS2, mS16x2};
  auto pending = [&](const int32_t* list, int32_t count) -> nolsm_status {
    k_status_pending<<<(unsigned)std::min(1024, (count + 255) / 256), 256, 0, st>>>(0, count, list, a.prep_out);
    NOLSM_LAUNCH_CHECK();
    return NOLSM_OK;
  };
  NOLSM_TRY(run_buckets(1, NOLSM_FP16, false, m, g, a.order, a.n_large, a.count, sms, st, pending));
  double fl[2];
  NOLSM_CUDA_TRY(cudaMemcpyAsync(fl, S->inv_flops.p, sizeof(fl), cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  plan->stats.flops_prep_tensor += fl[0];
  plan->stats.flops_prep_tensor_issued += fl[1];
  plan->stats.launches += 2;
  return NOLSM_OK;
}

// ==================================================================================== no-allocation entry point
// Some callers cannot call cudaMalloc at the moment they need a sign iteration: an MD engine or other
// host framework that owns every byte of device memory through its own pool, or code that must not
// allocate while it runs (fixed memory budgets, allocation-free inner loops). For them the tensor-core
// kernel above can also run on scratch that lives in this file's static device array instead of a
// plan's workspaces. Every GPU that loads the library holds the array until the process exits.

namespace {

constexpr int kNaMaxN = 192;                  // largest submatrix dimension accepted
constexpr int kNaR = 256, kNaLD = 192;        // scratch plane shape: rows rounded to 128, columns to 64
constexpr int kNaSlots = 4 * kSlots;          // scratch sub-slots: 4 CTAs with kSlots each
constexpr int kNaMaxSub = 4096;               // submatrices per call
constexpr size_t kNaPlaneElems = (size_t)kNaR * kNaLD;
constexpr size_t kNaPlanesBytes = sizeof(uint16_t) * kPlanes * kNaSlots * kNaPlaneElems;
constexpr size_t kNaIntBytes = sizeof(int32_t) * (3 * (size_t)kNaMaxSub + 64);
constexpr size_t kNaBytes = kNaPlanesBytes + kNaIntBytes;   // about 4.8 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Identity work order, zero factorisation status, zero counters: what the kernel expects to find. Every
// caller status starts as "timed out": the kernel overwrites it for each submatrix it takes, so one that
// no block reached (all of them gave up on a wait) cannot keep a stale OK from an earlier call.
__global__ void k_noalloc_reset(unsigned char* base, int count, int32_t* status) {
  int32_t* ints = reinterpret_cast<int32_t*>(base + kNaPlanesBytes);
  int32_t* order = ints;
  int32_t* prep = ints + kNaMaxSub;
  int32_t* rst = ints + 2 * kNaMaxSub;
  int32_t* ctr = ints + 3 * kNaMaxSub;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    order[i] = i;
    prep[i] = kSubOk;
    rst[i] = 0;
    status[i] = kSubTimeout;
  }
  if (blockIdx.x == 0 && threadIdx.x < 64) ctr[threadIdx.x] = 0;
}

// device address of the static array per device ordinal, looked up by the first call on that device
std::atomic<void*> g_na_addr[64];

}  // namespace

}  // namespace nolsm

extern "C" nolsm_status nolsm_sign_noalloc(int32_t count, const int32_t* sub_n, const int32_t* nbf,
                                           const int64_t* a_off, const int64_t* c_off, const float* A, const double* Q,
                                           const double* Sc, const double* Hc, const double* lam, double mu,
                                           const nolsm_options* opts, nolsm_stream_t stream, double* Dc,
                                           double* t_S, double* t_H, int32_t* iters, int32_t* status) {
  using namespace nolsm;
  cudaStream_t st = (cudaStream_t)stream;
  if (!opts || !sub_n || !nbf || !a_off || !c_off || !A || !Q || !Sc || !Hc || !lam || !Dc || !t_S || !t_H ||
      !iters || !status || !std::isfinite(mu)) {
    set_error("nolsm_sign_noalloc: NULL argument or non-finite mu");
    return NOLSM_ERR_ARG;
  }
  if (count < 1 || count > kNaMaxSub) {
    set_error("nolsm_sign_noalloc: %d submatrices requested; this entry point takes 1..%d per call", count,
              kNaMaxSub);
    return NOLSM_ERR_UNSUPPORTED;
  }
  Fmt mf, rf;
  if (!formats(opts->precision, &mf, &rf) || mf.fmt == FMT_E4M3) {
    set_error("nolsm_sign_noalloc: precision %d is not available here (E4M3 needs the symmetric form)",
              opts->precision);
    return NOLSM_ERR_UNSUPPORTED;
  }
  if (opts->max_iter < 1 || opts->refine_steps < 0 || !(opts->tol_ns > 0) || !(opts->tol_accept > 0)) {
    set_error("nolsm_sign_noalloc: invalid options");
    return NOLSM_ERR_ARG;
  }
  // sizes are checked against the static scratch before anything is launched
  int32_t h_n[kNaMaxSub];
  NOLSM_CUDA_TRY(cudaMemcpyAsync(h_n, sub_n, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
  NOLSM_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) {
    if (h_n[i] < 1 || h_n[i] > kNaMaxN) {
      set_error("nolsm_sign_noalloc: submatrix %d has dimension %d; this entry point takes 1..%d", i, h_n[i],
                kNaMaxN);
      return NOLSM_ERR_UNSUPPORTED;
    }
  }
  // once per device: the device address of this file's static scratch array
  int dev = 0;
  NOLSM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("nolsm_sign_noalloc: device ordinal %d out of range", dev);
    return NOLSM_ERR_UNSUPPORTED;
  }
  void* addr = g_na_addr[dev].load(std::memory_order_acquire);
  if (!addr) {   // threads that race here look up the same address
    NOLSM_CUDA_TRY(cudaGetSymbolAddress(&addr, g_noalloc_scratch));
    g_na_addr[dev].store(addr, std::memory_order_release);
  }
  unsigned char* base = static_cast<unsigned char*>(addr);
  int32_t* ints = reinterpret_cast<int32_t*>(base + kNaPlanesBytes);

  CUtensorMap mA, mB, mS, mS16, mS2, mS16x2;
  if (!tmap::make_3d(&mS16, base, 2, kNaLD, kNaR, (uint64_t)kNaSlots * kPlanes, 32, 16, CU_TENSOR_MAP_SWIZZLE_64B) ||
      !tmap::make_3d(&mS16x2, base, 2, kNaLD, kNaR, (uint64_t)kNaSlots * kPlanes, 32, 16, CU_TENSOR_MAP_SWIZZLE_64B, 2) ||
      !tmap::make_3d(&mS2, base, 2, kNaLD, kNaR, (uint64_t)kNaSlots * kPlanes, 32, 32, CU_TENSOR_MAP_SWIZZLE_64B, 2) ||
      !tmap::make_3d(&mA, base, 2, kNaLD, kNaR, (uint64_t)kNaSlots * kPlanes, 64, 128) ||
      !tmap::make_3d(&mB, base, 2, kNaLD, kNaR, (uint64_t)kNaSlots * kPlanes, 64, 64) ||
      !tmap::make_3d(&mS, base, 2, kNaLD, kNaR, (uint64_t)kNaSlots * kPlanes, 32, 32, CU_TENSOR_MAP_SWIZZLE_64B)) {
    set_error("nolsm_sign_noalloc: cuTensorMapEncodeTiled rejected the static scratch layout");
    return NOLSM_ERR_CUDA;
  }
  k_noalloc_reset<<<(count + 255) / 256, 256, 0, st>>>(base, count, status);
  NOLSM_LAUNCH_CHECK();
  TcArgs g{};
  g.j0 = 0; g.j1 = count;
  g.order = ints;
  g.sub_n = sub_n; g.nbf = nbf; g.a_off = a_off; g.c_off = c_off;
  g.A = A; g.Q = Q; g.Sc = Sc; g.Hc = Hc; g.lam = lam; g.lam_g = lam;
  g.prep_status = ints + kNaMaxSub;
  g.mu = mu;
  g.tol_ns = (float)opts->tol_ns; g.tol_accept = (float)opts->tol_accept;
  g.max_iter = opts->max_iter; g.refine_steps = opts->refine_steps;
  g.budget = nullptr;
  g.main_fmt = mf; g.refine_fmt = rf;
  g.planes = reinterpret_cast<uint16_t*>(base);
  g.R = kNaR; g.LD = kNaLD;
  g.next = ints + 3 * kNaMaxSub;
  g.err = ints + 3 * kNaMaxSub + 32;
  g.Dc = Dc; g.tS = t_S; g.tH = t_H; g.iters = iters; g.status = status;
  g.rsteps = ints + 2 * kNaMaxSub;
  g.nbelow = nullptr;
  g.wait_ns = opts->wait_ns > 0 ? (uint64_t)opts->wait_ns : kWaitNs;
  NOLSM_CUDA_TRY(cudaFuncSetAttribute((k_ns_tc<0, 0>), cudaFuncAttributeMaxDynamicSharedMemorySize, Shape<0>::kSmemBytes));
  k_ns_tc<0, 0><<<std::min(kNaSlots / kSlots, (count + kSlots - 1) / kSlots), Shape<0>::kThreads, Shape<0>::kSmemBytes, st>>>(mA, mB, mS, mA, mB, mS16, mS2, mS16x2, g);
  NOLSM_LAUNCH_CHECK();
  return NOLSM_OK;
}
