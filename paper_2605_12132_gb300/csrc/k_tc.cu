// Tensor-core (tcgen05 / TMEM / TMA) radial projection and back-projection with
// split-BF16 operands and FP32 accumulation.
//
// Each real FP32 operand x is represented by npieces bf16 terms x = x0 + x1 (+ x2)
// (x0 = bf16(x), x1 = bf16(x - x0), ...).  A product is accumulated as the sum of the
// piece products with ia + ib < npieces: 3 products for 2 pieces (BF16x3, ~16
// significant bits per operand) and 6 for 3 pieces (BF16x6, ~24 bits).
//
// Projection  (per mode, group, output block):  D[(z,part), j] = sum_r X[(z,part), r] P[j, r]
//   A = field rows (64 z x re/im, r contiguous): TMA stages the FP32 complex tile in shared
//       memory, four converter warps split it into swizzled bf16 pieces (forming the rotated
//       components tau*F on the way);
//   B = P pieces [j][r], K-major, loaded by TMA (64B swizzle);
//   M = 128, N = 256, K = 32 per pipeline stage; D in TMEM (128 lanes x 256 fp32 columns).
// Back-projection (per mode, group, output field): D[r, (z,part)] = sum_j Q[r, j] C[j, (z,part)]
//   A = Q pieces [r][j], K-major, TMA;  B = coefficient pieces [j][(z,part)], MN-major, TMA
//   (written pre-split by the spectral kernel).
// Warp roles: warps 0-3 convert (projection) and run the epilogue (TMEM -> registers ->
// global); warp 4 issues TMA; warp 5 issues tcgen05.mma (one elected thread) and commits
// to the stage's "empty" mbarrier.  Every mbarrier wait is bounded; on timeout the kernel
// records an error code, drains its own MMAs and frees TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace fdetd {

namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr uint32_t kTileBytes = 128 * 128;  // one bf16 piece of a 128 x 64 tile (16 KB)
constexpr long kSpinLimit = 1L << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Bounded wait for the phase with the given parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  // tcgen05 shared-memory matrix descriptor: start>>4 [0,14), LBO>>4 [16,30), SBO>>4 [32,46),
  // version 1 [46,48), layout SWIZZLE_128B (2) [61,64)
  uint64_t d = 0;
  d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor, kind::f16: D f32, A/B bf16, M = 128, N = BN
__host__ __device__ constexpr uint32_t idesc_bf16(bool b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn_major ? 1u : 0u) << 16) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcSmem {
  uint64_t fullA[4], fullB[4], fullS[4], empty[4], done;
  uint32_t tmem_base;
};

template <int NP>
struct Cfg {
  static constexpr int S = NP == 2 ? 3 : 2;                       // pipeline stages
  static constexpr uint32_t kStage = 2u * NP * kTileBytes;        // A and B pieces
  static constexpr size_t kSmem = (size_t)S * kStage + 1024 + sizeof(TcSmem) + 64;
};

// products (ia, ib) with ia + ib < NP
template <int NP>
__device__ __forceinline__ void product(int p, int& ia, int& ib) {
  if (NP == 2) {
    ia = p == 2 ? 1 : 0;
    ib = p == 1 ? 1 : 0;
  } else {
    const int A[6] = {0, 0, 1, 0, 1, 2}, B[6] = {0, 1, 0, 2, 1, 0};
    ia = A[p];
    ib = B[p];
  }
}

__device__ __forceinline__ void record_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

}  // namespace

struct TcProjArgs {
  const float2* fields;  // [nmodes][6][Nz][n]
  const float2* J;       // [nmodes][3][Nz][n] or null
  float* coef;           // [nmodes][9][n][Nz] complex (float pairs)
  int* err;
  int Nz, n, npad, kpad, ngroups;
};

struct TcBackArgs {
  float2* fields;
  int* err;
  int Nz, n, npad, kpad;
};

// Projection pipeline geometry: K tile of 32 (64-byte rows, 64B swizzle), N tile of 256.
constexpr int PBK = 32, PBN = 256;
constexpr uint32_t kPA = 128 * PBK * 2;      // one bf16 piece of the A tile (8 KB)
constexpr uint32_t kPB = PBN * PBK * 2;      // one bf16 piece of the B tile (16 KB)
constexpr uint32_t kPS = 64 * PBK * 8;       // FP32 complex staging tile: 64 z x 32 r (16 KB)

template <int NP>
struct PCfg {
  static constexpr int S = NP == 2 ? 3 : 2;
  static constexpr uint32_t kStage = kPS + NP * kPA + NP * kPB;
  static constexpr size_t kSmem = (size_t)S * kStage + 1024 + sizeof(TcSmem) + 64;
};

__device__ __forceinline__ uint64_t smem_desc_sw64(const void* p) {
  // K-major, 64-byte rows, SWIZZLE_64B (4): 8-row groups 512 B apart
  uint64_t d = 0;
  d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

__host__ __device__ constexpr uint32_t idesc_bf16_n(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int NP>
__global__ void __launch_bounds__(192, 1) tc_project_kernel(const __grid_constant__ CUtensorMap tmP,
                                                             const __grid_constant__ CUtensorMap tmF,
                                                             const __grid_constant__ CUtensorMap tmJ,
                                                             TcProjArgs a) {
  extern __shared__ __align__(1024) unsigned char raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  typedef PCfg<NP> C;
  TcSmem* sm = reinterpret_cast<TcSmem*>(base + C::S * C::kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, Nz = a.Nz;
  const int z0 = blockIdx.x * 64, j0 = blockIdx.y * PBN;
  const int md = blockIdx.z / (3 * a.ngroups), rem = blockIdx.z % (3 * a.ngroups);
  const int g = rem / 3, ob = rem % 3;
  const int gp = (g == 1) ? 1 : 0;
  // nonzero input blocks: E/J: e <- Ez ; a, c <- Er, Et.   B: b, d <- Bt, Br ; f <- Bz
  int blist[2], nb;
  if ((gp == 0 && ob == 0) || (gp == 1 && ob == 2)) {
    blist[0] = 2;
    nb = 1;
  } else {
    blist[0] = 0;
    blist[1] = 1;
    nb = 2;
  }
  const int ksteps = a.kpad / PBK;
  const int T = nb * ksteps;
  // stage layout: [staging FP32][A pieces][B pieces]
  auto stage_S = [&](int s) { return base + s * C::kStage; };
  auto stage_A = [&](int s) { return base + s * C::kStage + kPS; };
  auto stage_B = [&](int s) { return base + s * C::kStage + kPS + NP * kPA; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::S; ++s) {
      mbar_init(&sm->fullA[s], 4);
      mbar_init(&sm->fullB[s], 1);
      mbar_init(&sm->empty[s], 1);
    }
    for (int s = 0; s < C::S; ++s) mbar_init(&sm->fullS[s], 1);
    mbar_init(&sm->done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                 "r"(PBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp < 4) {
    // ---- converters: staged FP32 complex [64 z][32 r] -> A pieces, rows (z, re/im), K = r
    for (int t = 0; t < T; ++t) {
      const int s = t % C::S;
      const uint32_t ph = (uint32_t)(t / C::S) & 1u;
      if (!mbar_wait(&sm->fullS[s], ph)) {
        record_error(a.err, 1);
        break;
      }
      const int ib = blist[t / ksteps];
      const bool rot = (g == 1) ? (ib >= 1) : (ib == 1);
      const float* stg = reinterpret_cast<const float*>(stage_S(s));
      unsigned char* A = stage_A(s);
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int item = threadIdx.x + it * 128;  // 64 z x 4 chunks of 8 r
        const int zl = item >> 2, c = item & 3;
        const float4* src = reinterpret_cast<const float4*>(stg + zl * 64 + c * 16);
        float re[8], im[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 v = src[q];
          re[2 * q] = v.x;
          im[2 * q] = v.y;
          re[2 * q + 1] = v.z;
          im[2 * q + 1] = v.w;
        }
        if (rot) {  // tau = -i: (x, y) -> (y, -x)
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float x = re[q];
            re[q] = im[q];
            im[q] = -x;
          }
        }
        const int row_re = 2 * zl, row_im = 2 * zl + 1;
        const uint32_t off_re = row_re * 64 + ((c ^ ((row_re >> 1) & 3)) << 4);
        const uint32_t off_im = row_im * 64 + ((c ^ ((row_im >> 1) & 3)) << 4);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          uint32_t wr[4], wi[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 hr = __floats2bfloat162_rn(re[2 * q], re[2 * q + 1]);
            const __nv_bfloat162 hi = __floats2bfloat162_rn(im[2 * q], im[2 * q + 1]);
            wr[q] = *reinterpret_cast<const uint32_t*>(&hr);
            wi[q] = *reinterpret_cast<const uint32_t*>(&hi);
            re[2 * q] -= __low2float(hr);
            re[2 * q + 1] -= __high2float(hr);
            im[2 * q] -= __low2float(hi);
            im[2 * q + 1] -= __high2float(hi);
          }
          unsigned char* P = A + p * kPA;
          *reinterpret_cast<uint4*>(P + off_re) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
          *reinterpret_cast<uint4*>(P + off_im) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm->fullA[s]);
    }
  } else if (warp == 4) {
    if (lane == 0) {
      for (int t = 0; t < T; ++t) {
        const int s = t % C::S;
        const uint32_t ph = (uint32_t)(t / C::S) & 1u;
        if (!mbar_wait(&sm->empty[s], ph ^ 1u)) {
          record_error(a.err, 2);
          break;
        }
        const int ib = blist[t / ksteps];
        const int r0 = (t % ksteps) * PBK;
        // FP32 field tile: 64 z rows x 32 complex (64 floats)
        mbar_expect_tx(&sm->fullS[s], kPS);
        if (g == 2) {
          tma_load_2d(stage_S(s), &tmJ, &sm->fullS[s], 2 * r0, (md * 3 + ib) * Nz + z0);
        } else {
          const int field = (g == 1) ? (ib == 0 ? 4 : (ib == 1 ? 3 : 5)) : ib;
          tma_load_2d(stage_S(s), &tmF, &sm->fullS[s], 2 * r0, (md * 6 + field) * Nz + z0);
        }
        mbar_expect_tx(&sm->fullB[s], NP * kPB);
        for (int p = 0; p < NP; ++p) {
          const int y = (((md * 2 + gp) * NP + p) * 3 + ob) * a.npad + j0;
          tma_load_2d(stage_B(s) + p * kPB, &tmP, &sm->fullB[s], ib * a.kpad + r0, y);
        }
      }
    }
  } else {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_n(PBN);
      for (int t = 0; t < T; ++t) {
        const int s = t % C::S;
        const uint32_t ph = (uint32_t)(t / C::S) & 1u;
        if (!mbar_wait(&sm->fullA[s], ph) || !mbar_wait(&sm->fullB[s], ph)) {
          record_error(a.err, 3);
          break;
        }
        tc_fence_after();
        unsigned char* As = stage_A(s);
        unsigned char* Bs = stage_B(s);
#pragma unroll
        for (int k16 = 0; k16 < PBK / 16; ++k16) {
#pragma unroll
          for (int pr = 0; pr < (NP == 2 ? 3 : 6); ++pr) {
            int ia, ib;
            product<NP>(pr, ia, ib);
            const uint64_t ad = smem_desc_sw64(As + ia * kPA + k16 * 32);
            const uint64_t bd = smem_desc_sw64(Bs + ib * kPB + k16 * 32);
            mma_bf16(tmem, ad, bd, idesc, (t | k16 | pr) != 0);
          }
        }
        mma_commit(&sm->empty[s]);
      }
      mma_commit(&sm->done);
    }
  }

  // ---- epilogue: TMEM -> coef[md][g*3+ob][j][z] (complex, re/im from adjacent rows)
  if (warp < 4) {
    const bool got = mbar_wait(&sm->done, 0);
    if (!got) record_error(a.err, 4);
    tc_fence_after();
    if (got) {
      const int row = warp * 32 + lane;
      const int z = z0 + (row >> 1), part = row & 1;
      float* out = a.coef + (size_t)(md * 9 + g * 3 + ob) * n * 2 * Nz;
      for (int c0 = 0; c0 < PBN; c0 += 32) {
        if (j0 + c0 >= n) break;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int j = j0 + c0 + i;
          if (j < n) out[(size_t)j * 2 * Nz + 2 * z + part] = v[i];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PBN));
  }
}

template <int NP>
__global__ void __launch_bounds__(192, 1) tc_backproject_kernel(const __grid_constant__ CUtensorMap tmQ,
                                                                 const __grid_constant__ CUtensorMap tmS,
                                                                 TcBackArgs a) {
  extern __shared__ __align__(1024) unsigned char raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  typedef Cfg<NP> C;
  TcSmem* sm = reinterpret_cast<TcSmem*>(base + C::S * C::kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, Nz = a.Nz;
  const int z0 = blockIdx.x * 64, r0 = blockIdx.y * BM;
  const int md = blockIdx.z / 6, rem = blockIdx.z % 6;
  const int g = rem / 3, fb = rem % 3;
  // nonzero coefficient blocks: E: Er, Et <- a, c ; Ez <- e.   B: Bt, Br <- b, d ; Bz <- f
  int blist[2], nb;
  if (fb == 2) {
    blist[0] = (g == 0) ? 0 : 2;
    nb = 1;
  } else {
    blist[0] = (g == 0) ? 1 : 0;
    blist[1] = (g == 0) ? 2 : 1;
    nb = 2;
  }
  const int ksteps = a.kpad / BK;
  const int T = nb * ksteps;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::S; ++s) {
      mbar_init(&sm->fullB[s], 1);
      mbar_init(&sm->empty[s], 1);
    }
    mbar_init(&sm->done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp == 4) {
    if (lane == 0) {
      for (int t = 0; t < T; ++t) {
        const int s = t % C::S;
        const uint32_t ph = (uint32_t)(t / C::S) & 1u;
        if (!mbar_wait(&sm->empty[s], ph ^ 1u)) {
          record_error(a.err, 5);
          break;
        }
        const int cb = blist[t / ksteps];
        const int kk = (t % ksteps) * BK;
        unsigned char* As = base + s * C::kStage;
        unsigned char* Bs = As + NP * kTileBytes;
        mbar_expect_tx(&sm->fullB[s], 2 * NP * kTileBytes);
        for (int p = 0; p < NP; ++p) {
          const int ya = (((md * 2 + g) * NP + p) * 3 + fb) * a.npad + r0;
          tma_load_2d(As + p * kTileBytes, &tmQ, &sm->fullB[s], cb * a.kpad + kk, ya);
          const int yb = ((md * NP + p) * 6 + g * 3 + cb) * a.kpad + kk;
          tma_load_2d(Bs + p * kTileBytes, &tmS, &sm->fullB[s], 2 * z0, yb);
          tma_load_2d(Bs + p * kTileBytes + kTileBytes / 2, &tmS, &sm->fullB[s], 2 * z0 + 64, yb);
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(true);
      for (int t = 0; t < T; ++t) {
        const int s = t % C::S;
        const uint32_t ph = (uint32_t)(t / C::S) & 1u;
        if (!mbar_wait(&sm->fullB[s], ph)) {
          record_error(a.err, 6);
          break;
        }
        tc_fence_after();
        unsigned char* As = base + s * C::kStage;
        unsigned char* Bs = As + NP * kTileBytes;
#pragma unroll
        for (int k16 = 0; k16 < BK / 16; ++k16) {
#pragma unroll
          for (int pr = 0; pr < (NP == 2 ? 3 : 6); ++pr) {
            int ia, ib;
            product<NP>(pr, ia, ib);
            const uint64_t ad = smem_desc(As + ia * kTileBytes + k16 * 32, 16, 1024);
            // MN-major B: 64-element (128 B) rows along N, 16 K rows per MMA; N chunks 8 KB apart
            const uint64_t bd = smem_desc(Bs + ib * kTileBytes + k16 * 16 * 128, kTileBytes / 2, 1024);
            mma_bf16(tmem, ad, bd, idesc, (t | k16 | pr) != 0);
          }
        }
        mma_commit(&sm->empty[s]);
      }
      mma_commit(&sm->done);
    }
  }
  if (warp < 4) {
    const bool got = mbar_wait(&sm->done, 0);
    if (!got) record_error(a.err, 7);
    tc_fence_after();
    if (got) {
      const int r = r0 + warp * 32 + lane;
      const int field = g == 0 ? fb : (fb == 0 ? 4 : (fb == 1 ? 3 : 5));
      const bool rot = (g == 0) ? (fb == 1) : (fb >= 1);
      float2* out = a.fields + ((size_t)md * 6 + field) * Nz * n;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
        if (r < n) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int z = z0 + c0 / 2 + i;
            float2 o = make_float2(v[2 * i], v[2 * i + 1]);
            if (rot) o = make_float2(-o.y, o.x);  // 1/tau = i
            out[(size_t)z * n + r] = o;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  }
}

// ------------------------------------------------------------------ host side

struct TcPlan {
  int Nz = 0, n = 0, nmodes = 0, np = 0;
  int npadP = 0;  // projection: rows (j) of each coefficient block padded to the N tile (256)
  int npadQ = 0;  // back-projection: rows (r) of each field block padded to the M tile (128)
  int kpad = 0;   // columns of each block padded to 64
  __nv_bfloat16* d_P = nullptr;
  __nv_bfloat16* d_Q = nullptr;
  __nv_bfloat16* d_split = nullptr;
  int* d_err = nullptr;  // owned by the caller's plan
  CUtensorMap tmP, tmQ, tmS, tmF, tmJ;
  const void* mapped_fields = nullptr;
  const void* mapped_J = nullptr;
  size_t bytes = 0;
};

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

static bool make_map(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint32_t box_inner,
                     uint32_t box_outer, CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B,
                     CUtensorMapDataType ty = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) {
  auto enc = get_encode();
  if (!enc) return false;
  const uint64_t esz = ty == CU_TENSOR_MAP_DATA_TYPE_FLOAT32 ? 4 : 2;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * esz};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return enc(m, ty, 2, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static void split_bf16(double x, int np, uint16_t* out) {
  double r = x;
  for (int p = 0; p < np; ++p) {
    __nv_bfloat16 h = __float2bfloat16_rn((float)r);
    memcpy(&out[p], &h, 2);
    r -= (double)__bfloat162float(h);
  }
}

// Host matrices [nmodes][2][3n][3n] (FP64) -> padded bf16 pieces [nmodes][2][np][3 npad][3 kpad]
static std::vector<uint16_t> pack(const double* M, int nmodes, int n, int np, int npad, int kpad) {
  const int N3 = 3 * n;
  const size_t rows = (size_t)3 * npad, cols = (size_t)3 * kpad;
  std::vector<uint16_t> out((size_t)nmodes * 2 * np * rows * cols, 0);
  uint16_t pcs[3];
  for (int md = 0; md < nmodes; ++md)
    for (int g = 0; g < 2; ++g) {
      const double* src = M + (size_t)(md * 2 + g) * N3 * N3;
      for (int rb = 0; rb < 3; ++rb)
        for (int r = 0; r < n; ++r)
          for (int cb = 0; cb < 3; ++cb)
            for (int c = 0; c < n; ++c) {
              split_bf16(src[(size_t)(rb * n + r) * N3 + cb * n + c], np, pcs);
              for (int p = 0; p < np; ++p)
                out[((((size_t)(md * 2 + g) * np + p) * rows) + rb * npad + r) * cols + cb * kpad + c] = pcs[p];
            }
    }
  return out;
}

cudaError_t tc_create(TcPlan** outp, int Nz, int n, int nmodes, int np, const double* P, const double* Q, int* err,
                      char* msg, size_t msglen) {
  *outp = nullptr;
  if (np != 2 && np != 3) {
    snprintf(msg, msglen, "npieces must be 2 or 3");
    return cudaErrorInvalidValue;
  }
  if (Nz % 64) {
    snprintf(msg, msglen, "Nz must be a multiple of 64");
    return cudaErrorNotSupported;
  }
  if (n % 2) {
    snprintf(msg, msglen, "the tensor-core path needs an even Nr (16-byte field row stride for TMA)");
    return cudaErrorNotSupported;
  }
  int dev = 0, cc_major = 0, cc_minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (cc_major != 10 || cc_minor != 3) {
    snprintf(msg, msglen, "tcgen05 kernels are built for sm_103a (found sm_%d%d)", cc_major, cc_minor);
    return cudaErrorNotSupported;
  }
  if (!get_encode()) {
    snprintf(msg, msglen, "cuTensorMapEncodeTiled unavailable");
    return cudaErrorNotSupported;
  }
  TcPlan* t = new TcPlan();
  t->Nz = Nz;
  t->n = n;
  t->nmodes = nmodes;
  t->np = np;
  t->npadP = (n + PBN - 1) / PBN * PBN;
  t->npadQ = (n + BM - 1) / BM * BM;
  t->kpad = (n + BK - 1) / BK * BK;
  std::vector<uint16_t> hp = pack(P, nmodes, n, np, t->npadP, t->kpad);
  std::vector<uint16_t> hq = pack(Q, nmodes, n, np, t->npadQ, t->kpad);
  const size_t split_elems = (size_t)nmodes * np * 6 * t->kpad * 2 * Nz;
  cudaError_t e = cudaMalloc(&t->d_P, hp.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_Q, hq.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_split, split_elems * 2);
  if (e == cudaSuccess) e = cudaMemcpy(t->d_P, hp.data(), hp.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t->d_Q, hq.data(), hq.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(t->d_split, 0, split_elems * 2);
  if (e != cudaSuccess) {
    snprintf(msg, msglen, "allocation/upload failed");
    tc_destroy(t);
    return e;
  }
  t->d_err = err;
  t->bytes = hp.size() * 2 + hq.size() * 2 + split_elems * 2;
  const uint64_t cols = (uint64_t)3 * t->kpad;
  bool ok = make_map(&t->tmP, t->d_P, cols, (uint64_t)nmodes * 2 * np * 3 * t->npadP, PBK, PBN,
                     CU_TENSOR_MAP_SWIZZLE_64B) &&
            make_map(&t->tmQ, t->d_Q, cols, (uint64_t)nmodes * 2 * np * 3 * t->npadQ, BK, BM) &&
            make_map(&t->tmS, t->d_split, (uint64_t)2 * Nz, (uint64_t)nmodes * np * 6 * t->kpad, 64, BK);
  if (!ok) {
    snprintf(msg, msglen, "tensor map encoding failed");
    tc_destroy(t);
    return cudaErrorInvalidValue;
  }
  cudaError_t e1, e2;
  if (np == 2) {
    e1 = cudaFuncSetAttribute(tc_project_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PCfg<2>::kSmem);
    e2 = cudaFuncSetAttribute(tc_backproject_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Cfg<2>::kSmem);
  } else {
    e1 = cudaFuncSetAttribute(tc_project_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PCfg<3>::kSmem);
    e2 = cudaFuncSetAttribute(tc_backproject_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Cfg<3>::kSmem);
  }
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    snprintf(msg, msglen, "shared-memory opt-in failed");
    tc_destroy(t);
    return e1 != cudaSuccess ? e1 : e2;
  }
  *outp = t;
  return cudaSuccess;
}

void tc_destroy(TcPlan* t) {
  if (!t) return;
  if (t->d_P) cudaFree(t->d_P);
  if (t->d_Q) cudaFree(t->d_Q);
  if (t->d_split) cudaFree(t->d_split);
  delete t;
}

size_t tc_device_bytes(const TcPlan* t) { return t ? t->bytes : 0; }
__nv_bfloat16* tc_split_buffer(TcPlan* t) { return t->d_split; }
int tc_split_rows(const TcPlan* t) { return t->kpad; }

cudaError_t tc_project(TcPlan* t, const void* fields, const void* J, void* coef, cudaStream_t st) {
  // FP32 views of the caller's field and current arrays for the staging TMA: rows of 2 Nr floats
  if (fields != t->mapped_fields) {
    if (!make_map(&t->tmF, fields, (uint64_t)2 * t->n, (uint64_t)t->nmodes * 6 * t->Nz, 2 * PBK, 64,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_DATA_TYPE_FLOAT32))
      return cudaErrorInvalidValue;
    t->mapped_fields = fields;
  }
  if (J && J != t->mapped_J) {
    if (!make_map(&t->tmJ, J, (uint64_t)2 * t->n, (uint64_t)t->nmodes * 3 * t->Nz, 2 * PBK, 64,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_DATA_TYPE_FLOAT32))
      return cudaErrorInvalidValue;
    t->mapped_J = J;
  }
  TcProjArgs a;
  a.fields = (const float2*)fields;
  a.J = (const float2*)J;
  a.coef = (float*)coef;
  a.err = t->d_err;
  a.Nz = t->Nz;
  a.n = t->n;
  a.npad = t->npadP;
  a.kpad = t->kpad;
  a.ngroups = J ? 3 : 2;
  const CUtensorMap& mJ = J ? t->tmJ : t->tmF;
  dim3 grid(t->Nz / 64, t->npadP / PBN, t->nmodes * a.ngroups * 3);
  if (t->np == 2)
    tc_project_kernel<2><<<grid, 192, PCfg<2>::kSmem, st>>>(t->tmP, t->tmF, mJ, a);
  else
    tc_project_kernel<3><<<grid, 192, PCfg<3>::kSmem, st>>>(t->tmP, t->tmF, mJ, a);
  return cudaGetLastError();
}

cudaError_t tc_backproject(TcPlan* t, void* fields, cudaStream_t st) {
  TcBackArgs a;
  a.fields = (float2*)fields;
  a.err = t->d_err;
  a.Nz = t->Nz;
  a.n = t->n;
  a.npad = t->npadQ;
  a.kpad = t->kpad;
  dim3 grid(t->Nz / 64, t->npadQ / BM, t->nmodes * 6);
  if (t->np == 2)
    tc_backproject_kernel<2><<<grid, 192, Cfg<2>::kSmem, st>>>(t->tmQ, t->tmS, a);
  else
    tc_backproject_kernel<3><<<grid, 192, Cfg<3>::kSmem, st>>>(t->tmQ, t->tmS, a);
  return cudaGetLastError();
}

int tc_launches_per_step(const TcPlan*) { return 2; }

}  // namespace fdetd
