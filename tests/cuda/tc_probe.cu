// Test-only probe of the tensor-core building blocks used by the sign-iteration kernel: TMA loads
// with 128-byte swizzle, K-major A and MN- or K-major B shared-memory descriptors, tcgen05.mma with
// one or three products accumulated in TMEM, and tcgen05.ld readback. One CTA computes
// C[128 x N] = A[128 x K] * B[K x N]. Every wait is bounded; on timeout the probe reports an error.
#include <cstdint>
#include <cstdio>

#include "tcgen05.cuh"
#include "tmap.cuh"

namespace {

__global__ void __launch_bounds__(128) k_probe(const __grid_constant__ CUtensorMap mA,
                                               const __grid_constant__ CUtensorMap mB, float* C, int K, int N,
                                               int terms, uint32_t idesc, int b_mn, uint32_t lboB, uint32_t sboB,
                                               int* err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* Ahi = sm;
  uint8_t* Alo = sm + 16384;
  uint8_t* Bhi = sm + 32768;
  uint8_t* Blo = Bhi + N * 128;
  __shared__ uint64_t bar_full, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar_full, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::fence_mbar_init();
    bad = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int two = terms > 1 ? 2 : 1;
  const uint32_t bytes = (uint32_t)two * (16384u + (uint32_t)N * 128u);
  const int nks = K / 64;
  for (int ks = 0; ks < nks; ++ks) {
    if (threadIdx.x == 0) {
      tc::mbar_arrive_expect_tx(&bar_full, bytes);
      for (int z = 0; z < two; ++z) {
        tc::tma_load_3d(z ? Alo : Ahi, &mA, &bar_full, 64 * ks, 0, z);
        if (b_mn) {
          for (int c = 0; c < N / 64; ++c) tc::tma_load_3d((z ? Blo : Bhi) + c * 8192, &mB, &bar_full, 64 * c, 64 * ks, z);
        } else {
          tc::tma_load_3d(z ? Blo : Bhi, &mB, &bar_full, 64 * ks, 0, z);
        }
      }
    }
    const uint64_t dl = tc::globaltimer() + 2000000000ull;
    if (!tc::mbar_wait(&bar_full, ks & 1, dl)) atomicExch(&bad, 1);
    __syncthreads();
    if (bad) break;
    if (threadIdx.x == 0) {
      tc::tc_fence_after();
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ah = tc::sdesc_sw128(tc::smem_u32(Ahi) + kk * 32, 16, 1024);
        const uint64_t al = tc::sdesc_sw128(tc::smem_u32(Alo) + kk * 32, 16, 1024);
        const uint32_t boff = b_mn ? kk * 2048 : kk * 32;
        const uint64_t bh = tc::sdesc_sw128(tc::smem_u32(Bhi) + boff, lboB, sboB);
        const uint64_t bl = tc::sdesc_sw128(tc::smem_u32(Blo) + boff, lboB, sboB);
        tc::mma_f16(tmem, ah, bh, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
        if (terms > 1) {
          tc::mma_f16(tmem, ah, bl, idesc, 1u);
          tc::mma_f16(tmem, al, bh, idesc, 1u);
        }
      }
      tc::mma_commit(&bar_mma);
    }
    if (!tc::mbar_wait(&bar_mma, ks & 1, dl)) atomicExch(&bad, 1);
    __syncthreads();
    if (bad) break;
  }
  tc::tc_fence_after();
  if (!bad) {
    for (int c0 = 0; c0 < N / 32; ++c0) {
      uint32_t r[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * c0, r);
      tc::tmem_wait_ld();
      const int row = 32 * warp + lane;
      for (int j = 0; j < 32; ++j) C[row * N + 32 * c0 + j] = __uint_as_float(r[j]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
  if (threadIdx.x == 0 && bad) *err = 1;
}

// Trimmed shapes: C = A[0:M, 0:Kuse] B[0:Kuse, 0:N] with M = 64 or 128, N a multiple of 16 (M = 128) or
// 8 (M = 64) up to the 64-column chunks loaded (Nl), Kuse a multiple of 16 up to K: the K = 16 steps past
// Kuse are not issued. Three-term split products, B MN-major. The raw accumulator (all 128 TMEM lanes x Nl
// columns) goes to C, so that the test sees where an M = 64 product's rows land.
__global__ void __launch_bounds__(128) k_probe_trim(const __grid_constant__ CUtensorMap mA,
                                                    const __grid_constant__ CUtensorMap mB, float* C, int K, int Nl,
                                                    int Kuse, uint32_t idesc, int* err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* Ahi = sm;
  uint8_t* Alo = sm + 16384;
  uint8_t* Bhi = sm + 32768;
  uint8_t* Blo = Bhi + Nl * 128;
  __shared__ uint64_t bar_full, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int bad;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar_full, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::fence_mbar_init();
    bad = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base;
  // zero the accumulator columns first, so that lanes the product does not write read back as 0
  {
    uint32_t z[32];
    for (int j = 0; j < 32; ++j) z[j] = 0u;
    for (int c0 = 0; c0 < Nl / 32; ++c0) tc::tmem_st32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * c0, z);
    tc::tmem_wait_st();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t bytes = 2u * (16384u + (uint32_t)Nl * 128u);
  const int nks = K / 64;
  bool first = true;
  for (int ks = 0; ks < nks; ++ks) {
    if (threadIdx.x == 0) {
      tc::mbar_arrive_expect_tx(&bar_full, bytes);
      for (int z = 0; z < 2; ++z) {
        tc::tma_load_3d(z ? Alo : Ahi, &mA, &bar_full, 64 * ks, 0, z);
        for (int c = 0; c < Nl / 64; ++c) tc::tma_load_3d((z ? Blo : Bhi) + c * 8192, &mB, &bar_full, 64 * c, 64 * ks, z);
      }
    }
    const uint64_t dl = tc::globaltimer() + 2000000000ull;
    if (!tc::mbar_wait(&bar_full, ks & 1, dl)) atomicExch(&bad, 1);
    __syncthreads();
    if (bad) break;
    if (threadIdx.x == 0) {
      tc::tc_fence_after();
      for (int kk = 0; kk < 4 && 64 * ks + 16 * kk < Kuse; ++kk) {
        const uint64_t ah = tc::sdesc_sw128(tc::smem_u32(Ahi) + kk * 32, 16, 1024);
        const uint64_t al = tc::sdesc_sw128(tc::smem_u32(Alo) + kk * 32, 16, 1024);
        const uint64_t bh = tc::sdesc_sw128(tc::smem_u32(Bhi) + kk * 2048, 8192, 1024);
        const uint64_t bl = tc::sdesc_sw128(tc::smem_u32(Blo) + kk * 2048, 8192, 1024);
        tc::mma_f16(tmem, ah, bh, idesc, first ? 0u : 1u);
        tc::mma_f16(tmem, ah, bl, idesc, 1u);
        tc::mma_f16(tmem, al, bh, idesc, 1u);
        first = false;
      }
      tc::mma_commit(&bar_mma);
    }
    if (!tc::mbar_wait(&bar_mma, ks & 1, dl)) atomicExch(&bad, 1);
    __syncthreads();
    if (bad) break;
  }
  tc::tc_fence_after();
  if (!bad) {
    const int lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < Nl / 32; ++c0) {
      uint32_t r[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * c0, r);
      tc::tmem_wait_ld();
      const int row = 32 * warp + lane;
      for (int j = 0; j < 32; ++j) C[row * Nl + 32 * c0 + j] = __uint_as_float(r[j]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
  if (threadIdx.x == 0 && bad) *err = 1;
}

}  // namespace

extern "C" int tc_probe_trim(const void* A, const void* B, float* C, int K, int Nl, int M, int N, int Kuse, int bf16,
                             int* err_dev) {
  if (K % 64 || Nl % 64 || Nl > 256 || K <= 0 || Kuse % 16 || Kuse <= 0 || Kuse > K) return -1;
  if ((M != 64 && M != 128) || N > Nl || N <= 0 || N % (M == 128 ? 16 : 8)) return -1;
  CUtensorMap mA, mB;
  if (!tmap::make_3d(&mA, const_cast<void*>(A), 2, K, 128, 2, 64, 128)) return -2;
  if (!tmap::make_3d(&mB, const_cast<void*>(B), 2, Nl, K, 2, 64, 64)) return -3;
  const uint32_t id = tc::idesc(bf16, bf16, 0, 1, (uint32_t)M, (uint32_t)N);
  const int smem = 1024 + 32768 + 2 * Nl * 128;
  cudaFuncSetAttribute(k_probe_trim, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_probe_trim<<<1, 128, smem>>>(mA, mB, C, K, Nl, Kuse, id, err_dev);
  if (cudaGetLastError() != cudaSuccess) return -4;
  if (cudaDeviceSynchronize() != cudaSuccess) return -5;
  return 0;
}

extern "C" int tc_probe_gemm(const void* A, const void* B, float* C, int K, int N, int terms, int bf16, int b_mn,
                             int lboB, int sboB, int* err_dev) {
  if (K % 64 || N % 64 || N > 256 || K <= 0) return -1;
  CUtensorMap mA, mB;
  const int two = terms > 1 ? 2 : 1;
  if (!tmap::make_3d(&mA, const_cast<void*>(A), 2, K, 128, two, 64, 128)) return -2;
  bool ok = b_mn ? tmap::make_3d(&mB, const_cast<void*>(B), 2, N, K, two, 64, 64)
                 : tmap::make_3d(&mB, const_cast<void*>(B), 2, K, N, two, 64, N);
  if (!ok) return -3;
  const uint32_t id = tc::idesc(bf16, bf16, 0, b_mn ? 1 : 0, 128, N);
  const int smem = 1024 + 32768 + 2 * N * 128;
  cudaFuncSetAttribute(k_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_probe<<<1, 128, smem>>>(mA, mB, C, K, N, terms, id, b_mn, (uint32_t)lboB, (uint32_t)sboB, err_dev);
  if (cudaGetLastError() != cudaSuccess) return -4;
  if (cudaDeviceSynchronize() != cudaSuccess) return -5;
  return 0;
}
