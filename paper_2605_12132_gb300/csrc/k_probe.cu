// Diagnostic: how the tcgen05 kind::f16 MMA rounds its FP32 accumulation.
//
// One CTA stages hand-picked bf16 operands in the same 64-byte-swizzled K-major layout the
// projection kernel uses, issues one MMA on K = 0..15 and then `reps` accumulating MMAs on
// K = 16..31 (M = 128, N = 256), and returns columns 0 and 1 of the first 12 rows.  Column 0
// multiplies by ones; column 1 by +1 on K < 16 and -1 on K >= 16.  The rows (u = ulp(1) = 2^-23):
//   0: 1 + 0.75u inside one MMA           1: 1, then +0.75u per chained MMA
//   2: -1, then -0.75u per chained MMA     3: 1 + 15 x 0.25u inside one MMA
//   4: 1 + 0.5u (tie) inside one MMA       5: 1 + u, then +0.5u per chained MMA
//   6: 1 - 1 + 2^-30 inside one MMA        7: 2^20 + 2^-10 - 2^20 inside one MMA
//   8: 1 + 15 x 2^-26 inside one MMA       9: 1, then +16 x 0.25u per chained MMA
//  10: 1 + 0.875u inside one MMA          11: 1 + 2 x 0.25u inside one MMA
// Round-to-nearest would give 1 + u for rows 0 and 1; the values returned tell the rounding mode
// and how many bits below the largest term survive the alignment.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fdetd.h"

namespace {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_sw64(const void* p) {
  uint64_t d = 0;
  d |= (uint64_t)((su32(p) >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// Ag: [128][32] bf16 rows (K contiguous), Bg: [256][32]; out: [128][2] FP32; status: 1 on timeout
__global__ void __launch_bounds__(128, 1) mma_rounding_kernel(const uint16_t* Ag, const uint16_t* Bg, float* out,
                                                              int reps, int* status) {
  extern __shared__ __align__(1024) unsigned char raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  unsigned char* A = base;          // 128 rows x 64 B
  unsigned char* B = base + 8192;   // 256 rows x 64 B
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 8192 + 16384);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // 64-byte swizzle: 16-byte chunk c of row r at r*64 + ((c ^ ((r >> 1) & 3)) << 4)
  for (int item = tid; item < 128 * 4; item += 128) {
    const int r = item >> 2, c = item & 3;
    *reinterpret_cast<uint4*>(A + r * 64 + ((c ^ ((r >> 1) & 3)) << 4)) =
        *reinterpret_cast<const uint4*>(Ag + r * 32 + c * 8);
  }
  for (int item = tid; item < 256 * 4; item += 128) {
    const int r = item >> 2, c = item & 3;
    *reinterpret_cast<uint4*>(B + r * 64 + ((c ^ ((r >> 1) & 3)) << 4)) =
        *reinterpret_cast<const uint4*>(Bg + r * 32 + c * 8);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tbase)), "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tbase;
  const uint32_t idesc =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  if (tid == 0) {
    mma(tmem, desc_sw64(A), desc_sw64(B), idesc, 0);
    for (int r = 0; r < reps; ++r) mma(tmem, desc_sw64(A + 32), desc_sw64(B + 32), idesc, 1);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
  }
  __syncwarp();
  bool ok = false;
  for (long it = 0; it < (1L << 24) && !ok; ++it) {
    uint32_t v;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(v)
                 : "r"(su32(bar)), "r"(0)
                 : "memory");
    ok = v != 0;
  }
  if (!ok && lane == 0) atomicExch(status, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  out[(warp * 32 + lane) * 2 + 0] = __uint_as_float(r0);
  out[(warp * 32 + lane) * 2 + 1] = __uint_as_float(r1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
  }
}

uint16_t to_bf16(float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  uint16_t u;
  memcpy(&u, &h, 2);
  return u;
}

}  // namespace

extern "C" int fdetd_probe_mma_rounding(float* host_out, int reps, void* stream) {
  if (!host_out || reps < 0 || reps > 64) return FDETD_ERR_ARG;
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return FDETD_ERR_UNSUPPORTED;
  std::vector<uint16_t> A(128 * 32, 0), B(256 * 32, 0);
  const float u = ldexpf(1.f, -23);
  for (int k = 0; k < 32; ++k) {
    B[0 * 32 + k] = to_bf16(1.f);
    B[1 * 32 + k] = to_bf16(k < 16 ? 1.f : -1.f);
  }
  auto set = [&](int r, int k, float v) { A[r * 32 + k] = to_bf16(v); };
  set(0, 0, 1.f), set(0, 1, 0.75f * u);
  set(1, 0, 1.f), set(1, 16, 0.75f * u);
  set(2, 0, -1.f), set(2, 16, -0.75f * u);
  set(3, 0, 1.f);
  for (int k = 1; k < 16; ++k) set(3, k, 0.25f * u);
  set(4, 0, 1.f), set(4, 1, 0.5f * u);
  set(5, 0, 1.f), set(5, 1, u), set(5, 16, 0.5f * u);
  set(6, 0, 1.f), set(6, 1, -1.f), set(6, 2, ldexpf(1.f, -30));
  set(7, 0, ldexpf(1.f, 20)), set(7, 1, ldexpf(1.f, -10)), set(7, 2, -ldexpf(1.f, 20));
  set(8, 0, 1.f);
  for (int k = 1; k < 16; ++k) set(8, k, ldexpf(1.f, -26));
  set(9, 0, 1.f);
  for (int k = 16; k < 32; ++k) set(9, k, 0.25f * u);
  set(10, 0, 1.f), set(10, 1, 0.875f * u);
  set(11, 0, 1.f), set(11, 1, ldexpf(1.f, -25)), set(11, 2, ldexpf(1.f, -25));
  cudaStream_t st = (cudaStream_t)stream;
  uint16_t *dA = nullptr, *dB = nullptr;
  float* dO = nullptr;
  int* dS = nullptr;
  int status = 0, rc = FDETD_OK;
  const int smem = 1024 + 8192 + 16384 + 64;
  cudaError_t e = cudaMalloc(&dA, A.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(&dB, B.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(&dO, 128 * 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dS, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dA, A.data(), A.size() * 2, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dB, B.data(), B.size() * 2, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dS, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mma_rounding_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) {
    mma_rounding_kernel<<<1, 128, smem, st>>>(dA, dB, dO, reps, dS);
    e = cudaGetLastError();
  }
  float O[128 * 2];
  if (e == cudaSuccess) e = cudaMemcpyAsync(O, dO, sizeof O, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, dS, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    rc = FDETD_ERR_CUDA;
  else if (status)
    rc = FDETD_ERR_TIMEOUT;
  else
    memcpy(host_out, O, 12 * 2 * sizeof(float));
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dO);
  cudaFree(dS);
  return rc;
}
