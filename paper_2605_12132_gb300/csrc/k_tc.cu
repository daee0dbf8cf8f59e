// Tensor-core (tcgen05 / TMEM / bulk async copies) radial projection and back-projection with
// split-BF16 operands and FP32 accumulation, as persistent grouped kernels.
//
// Each real FP32 operand x is represented by npieces bf16 terms x = x0 + x1 (+ x2)
// (x0 = bf16(x), x1 = bf16(x - x0), ...).  A product is accumulated as the sum of the
// piece products with ia + ib < npieces: 3 products for 2 pieces (BF16x3, ~16
// significant bits per operand) and 6 for 3 pieces (BF16x6, ~24 bits).
//
// The tensor core's FP32 accumulation truncates toward zero after every MMA and aligns the
// products to the largest exponent with two guard bits, so the error of a long accumulation
// chain grows with its length.  With NACC = 2 the leading product x0*y0 and the correction
// products (all at least 2^-8 smaller) accumulate in separate TMEM accumulators, which leaves
// one MMA per K step on the chain that carries the full magnitude; the epilogue adds the two
// in FP32 (round to nearest).
//
// Projection  (per mode, group, output block):  D[(z,part), j] = sum_r X[(z,part), r] P[j, r]
//   A = field rows (64 z x re/im, r contiguous): a TMA box (per-instance tensor map in the
//       kernel parameters) stages FP32 complex values in shared memory; eight converter warps
//       split them in place into 64B-swizzled bf16 pieces (forming tau*F on the way);
//   B = P pieces [j][r], K-major, pre-tiled and pre-swizzled at plan time (one bulk copy);
//   M = 128, N = TN (128 or 256), K = 32 per pipeline stage.
// Back-projection (per mode, group, output field): D[r, (z,part)] = sum_j Q[r, j] C[j, (z,part)]
//   A = Q pieces [r][j], K-major, pre-tiled (128B swizzle);  B = coefficient pieces [j][(z,part)],
//   MN-major, written pre-tiled and pre-split by the spectral kernel; M = 128 (r), N = TN.
//
// Both kernels are persistent: one CTA per SM walks a tile table (tiles of several instances in
// one launch), the pipeline stages run on across tile boundaries, and with NBUF = 2 the TMEM
// accumulators are double-buffered so the epilogue of one tile overlaps the MMAs of the next.
// Warp roles, projection: 0-7 convert, 8-15 epilogue (TMEM -> registers -> global; two warps per TMEM lane
// quarter, alternate 32-column chunks), 16 issues the TMA and bulk copies, 17 issues tcgen05.mma (one thread).
// Back-projection: 0-3 epilogue, 4 copies, 5 MMA.  With NBUF = 1 (BF16x6 at TN = 256: the leading and
// correction accumulators fill the 512 TMEM columns) the MMAs of the next tile wait for the drain.
// Every mbarrier wait is bounded; on timeout the kernel records an error code in the instance's
// flag, tells the other roles to stop through a shared abort flag, drains its own copies and
// MMAs, and frees TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace fdetd {

namespace {

constexpr long long kSpinLimit = 1LL << 26;

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
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity: at most `spin` polls (a kernel parameter, kSpinLimit
// unless a plan sets another limit).  Returns false on timeout (and raises the abort flag) or as soon as
// another role has raised it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, long long spin) {
  for (long long it = 0; it < spin; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}
// Bounded wait that ignores the abort flag (draining in-flight copies before exit).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_try(bar, parity)) return;
}

// bulk asynchronous copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// 2D TMA tile load (tensor map in kernel-parameter space), completing on `bar`
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// tcgen05 shared-memory matrix descriptor: start>>4 [0,14), LBO>>4 [16,30), SBO>>4 [32,46),
// version 1 [46,48), layout [61,64) (2 = SWIZZLE_128B, 4 = SWIZZLE_64B)
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)layout << 61;
  return d;
}
// K-major, 64-byte rows, SWIZZLE_64B: 8-row groups 512 B apart
__device__ __forceinline__ uint64_t desc_sw64(const void* p) { return smem_desc(p, 16, 512, 4); }

// instruction descriptor, kind::f16: D f32 (bit 4), A and B bf16 (bits 7, 10), B MN-major (bit 16),
// N >> 3 at bit 17, M >> 4 at bit 24 (M = 128)
__host__ __device__ constexpr uint32_t idesc_bf16(int N, bool b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn_major ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
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

// 32 columns of two accumulators, issued without waiting: the registers are written asynchronously and must
// not be read before tmem_wait2 on the same arrays, which the compiler sees as redefining them
__device__ __forceinline__ void tmem_ld2x32(uint32_t ta, uint32_t tb, uint32_t* a, uint32_t* b) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%"
      "48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
        "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]),
        "=r"(a[16]), "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]),
        "=r"(a[24]), "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31]),
        "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]),
        "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15]),
        "=r"(b[16]), "=r"(b[17]), "=r"(b[18]), "=r"(b[19]), "=r"(b[20]), "=r"(b[21]), "=r"(b[22]), "=r"(b[23]),
        "=r"(b[24]), "=r"(b[25]), "=r"(b[26]), "=r"(b[27]), "=r"(b[28]), "=r"(b[29]), "=r"(b[30]), "=r"(b[31])
      : "r"(ta), "r"(tb));
}
__device__ __forceinline__ void tmem_wait2(uint32_t* a, uint32_t* b) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                 "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]),
                 "+r"(a[15]), "+r"(a[16]), "+r"(a[17]), "+r"(a[18]), "+r"(a[19]), "+r"(a[20]), "+r"(a[21]),
                 "+r"(a[22]), "+r"(a[23]), "+r"(a[24]), "+r"(a[25]), "+r"(a[26]), "+r"(a[27]), "+r"(a[28]),
                 "+r"(a[29]), "+r"(a[30]), "+r"(a[31]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]),
                 "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]),
                 "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]), "+r"(b[16]), "+r"(b[17]),
                 "+r"(b[18]), "+r"(b[19]), "+r"(b[20]), "+r"(b[21]), "+r"(b[22]), "+r"(b[23]), "+r"(b[24]),
                 "+r"(b[25]), "+r"(b[26]), "+r"(b[27]), "+r"(b[28]), "+r"(b[29]), "+r"(b[30]), "+r"(b[31])
               :
               : "memory");
}

// the N extent of a projection tile starting at output j0 of an instance with n outputs: the rest of the
// instance rounded up to the MMA granularity of 16, at most the tile width TN
__host__ __device__ __forceinline__ int tile_n(int TN, int n, int j0) {
  const int r = ((n - j0) + 15) & ~15;
  return r < TN ? r : TN;
}

// products (ia, ib) with ia + ib < NP, leading product first
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

// Pipeline accounting (GroupParams.waits, 8 counters per kernel, summed over CTAs): clock cycles a role spent
// waiting on one kind of barrier, or busy, so that the idle time of the tensor pipe can be attributed.
enum {
  kWaitCta = 0,     // MMA issuer: whole residency of the CTA (the denominator)
  kWaitA = 1,       // MMA issuer: waiting for the A operand of a stage (projection: the converted pieces)
  kWaitB = 2,       // MMA issuer: waiting for the B operand of a stage (back-projection: both operands)
  kWaitTmem = 3,    // MMA issuer: waiting for the epilogue to free an accumulator
  kWaitStage = 4,   // producer: waiting for a free stage of the ring
  kWaitStaged = 5,  // converters: waiting for the staged FP32 tile
  kBusyConv = 6,    // converters: from the staged tile to the pieces' arrival
  kBusyEpi = 7      // epilogue: from a full accumulator to its release
};
__device__ __forceinline__ void add_waits(unsigned long long* w, int slot, long long cycles) {
  if (w) atomicAdd(w + slot, (unsigned long long)cycles);
}

// The projection's converter warps (0 .. kConvWarps-1) split the staged FP32 field tile (64 z x 32 complex =
// 256 items of 8 radii) into bf16 pieces; with eight of them each thread converts one item per stage.
constexpr int kConvWarps = 8, kConvThreads = 32 * kConvWarps, kConvItems = 256 / kConvThreads;
// epilogue warps: two per TMEM lane quarter, each draining every other 32-column chunk
constexpr int kEpiWarps = 8;
constexpr int kProjThreads = 32 * (kConvWarps + kEpiWarps + 2);   // + 1 copy, 1 MMA warp

// barrier + AND-reduction over the converter threads (named barrier 1)
__device__ __forceinline__ bool bar_and_conv(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kConvThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void bar_sync_conv() { asm volatile("bar.sync 1, %0;" ::"n"(kConvThreads) : "memory"); }

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return (unsigned char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

struct GBar {
  uint64_t fullS[8], fullA[8], fullB[8], empty[8], tfull[2], tempty[2], done;
  uint32_t tmem_base;
  int abort;
};

// tile record: x = instance, y = md | g << 8 | blk << 12, z = z0, w = j0 (projection) / r0 (back)
__device__ __forceinline__ void decode(const int4& t, int& md, int& g, int& blk) {
  md = t.y & 0xff;
  g = (t.y >> 8) & 0xf;
  blk = (t.y >> 12) & 0xf;
}

// input blocks feeding projection output block ob of group g (E/J: inputs Er, Et, Ez; B: Bt, Br, Bz)
__device__ __forceinline__ int proj_blocks(int g, int ob, int* bl) {
  const int gp = g == 1 ? 1 : 0;
  if ((gp == 0 && ob == 0) || (gp == 1 && ob == 2)) {
    bl[0] = 2;
    return 1;
  }
  bl[0] = 0;
  bl[1] = 1;
  return 2;
}
// coefficient blocks feeding back-projection field block fb of group g (E: e, a, c; B: b, d, f)
__device__ __forceinline__ int back_blocks(int g, int fb, int* bl) {
  if (fb == 2) {
    bl[0] = g == 0 ? 0 : 2;
    return 1;
  }
  bl[0] = g == 0 ? 1 : 0;
  bl[1] = g == 0 ? 2 : 1;
  return 2;
}

// ------------------------------------------------------------------ projection

template <int NP, int NACC, int NBUF, int TN>
struct PG {
  static constexpr uint32_t kA = NP * 8192u > 16384u ? NP * 8192u : 16384u;  // FP32 staging / A pieces
  static constexpr uint32_t kBp = TN * 64u;                                   // one piece of the B tile
  static constexpr uint32_t kStage = kA + NP * kBp;
  static constexpr int S0 = (int)((220u * 1024u) / kStage);
  static constexpr int S = S0 > 6 ? 6 : S0;
  static constexpr size_t kSmem = (size_t)S * kStage + 1024 + sizeof(GBar) + 64;
  static constexpr int kCols = NACC * NBUF * TN;
  static_assert(kCols <= 512 && (kCols & (kCols - 1)) == 0, "TMEM columns");
  static_assert(S >= 2, "pipeline depth");
};

template <int NP, int NACC, int NBUF, int TN>
__global__ void __launch_bounds__(kProjThreads, 1) tcg_project_kernel(const __grid_constant__ GroupParams gp,
                                                              const int4* __restrict__ tiles, int ntiles) {
  typedef PG<NP, NACC, NBUF, TN> C;
  constexpr int S = C::S;
  extern __shared__ __align__(1024) unsigned char raw[];
  unsigned char* base = align1024(raw);
  GBar* sb = reinterpret_cast<GBar*>(base + S * C::kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &sb->abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&sb->fullS[s], 1);
      mbar_init(&sb->fullA[s], kConvWarps);
      mbar_init(&sb->fullB[s], 1);
      mbar_init(&sb->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sb->tfull[b], 1);
      mbar_init(&sb->tempty[b], kEpiWarps);
    }
    mbar_init(&sb->done, 1);
    sb->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sb->tmem_base)),
                 "r"(C::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sb->tmem_base;
  auto stage_A = [&](int s) { return base + (size_t)s * C::kStage; };
  auto stage_B = [&](int s) { return base + (size_t)s * C::kStage + C::kA; };

  if (warp < kConvWarps) {
    // ---- converters: staged FP32 complex [64 z][32 r] -> A pieces in place, rows (z, re/im), K = r
    int q = 0;
    bool live = true;
    long long w_staged = 0, busy = 0;
    for (int ti = blockIdx.x; live && ti < ntiles; ti += gridDim.x) {
      const int4 tl = tiles[ti];
      int md, g, ob, bl[2];
      decode(tl, md, g, ob);
      const GInst& I = gp.inst[tl.x];
      const int n = I.n, nks = (n + 31) >> 5;
      const int T = proj_blocks(g, ob, bl) * nks;
      for (int t = 0; t < T; ++t, ++q) {
        const int s = q % S;
        const uint32_t ph = (uint32_t)(q / S) & 1u;
        const long long c0 = clock64();
        // all converter threads take the same decision, so none is left behind at a barrier
        const bool ok = bar_and_conv(mbar_wait(&sb->fullS[s], ph, abort, gp.spin));
        const long long c1 = clock64();
        w_staged += c1 - c0;
        if (!ok) {
          if (threadIdx.x == 0) record_error(I.err, 11);
          live = false;
          break;
        }
        const int ib = bl[t / nks];
        const int r0 = (t % nks) * 32;
        const bool rot = (g == 1) ? (ib >= 1) : (ib == 1);
        unsigned char* A = stage_A(s);
        const float* stg = reinterpret_cast<const float*>(A);
        float re[kConvItems][8], im[kConvItems][8];
#pragma unroll
        for (int it = 0; it < kConvItems; ++it) {
          const int item = threadIdx.x + it * kConvThreads;  // 64 z x 4 chunks of 8 r
          const int zl = item >> 2, c = item & 3;
          const float4* src = reinterpret_cast<const float4*>(stg + zl * 64 + c * 16);
          // read the four 16-byte pieces in an order rotated by rr = (c + zl): a warp's 32 reads then fall
          // on all eight 16-byte bank groups (4 wavefronts) instead of two; t[k] is re-rotated after
          const int rr = (c + zl) & 3;
          float4 t[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) t[k] = src[(k + rr) & 3];
          if (rr & 1) {
            const float4 x = t[3];
            t[3] = t[2];
            t[2] = t[1];
            t[1] = t[0];
            t[0] = x;
          }
          if (rr & 2) {
            float4 x = t[0];
            t[0] = t[2];
            t[2] = x;
            x = t[1];
            t[1] = t[3];
            t[3] = x;
          }
          // radii beyond Nr are zero-filled by the TMA box; masked here as well, on the last K stage only
          const bool full = r0 + 32 <= n;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float4 v = t[k];
            const bool in0 = full || r0 + c * 8 + 2 * k < n, in1 = full || r0 + c * 8 + 2 * k + 1 < n;
            re[it][2 * k] = in0 ? v.x : 0.f;
            im[it][2 * k] = in0 ? v.y : 0.f;
            re[it][2 * k + 1] = in1 ? v.z : 0.f;
            im[it][2 * k + 1] = in1 ? v.w : 0.f;
          }
          if (rot) {  // tau = -i: (x, y) -> (y, -x)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const float x = re[it][k];
              re[it][k] = im[it][k];
              im[it][k] = -x;
            }
          }
        }
        bar_sync_conv();  // every staged value is in registers before the pieces overwrite the staging
#pragma unroll
        for (int it = 0; it < kConvItems; ++it) {
          const int item = threadIdx.x + it * kConvThreads;
          const int zl = item >> 2, c = item & 3;
          const int row_re = 2 * zl, row_im = 2 * zl + 1;
          const uint32_t off_re = row_re * 64 + ((c ^ ((row_re >> 1) & 3)) << 4);
          const uint32_t off_im = row_im * 64 + ((c ^ ((row_im >> 1) & 3)) << 4);
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            uint32_t wr[4], wi[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const __nv_bfloat162 hr = __floats2bfloat162_rn(re[it][2 * k], re[it][2 * k + 1]);
              const __nv_bfloat162 hi = __floats2bfloat162_rn(im[it][2 * k], im[it][2 * k + 1]);
              wr[k] = *reinterpret_cast<const uint32_t*>(&hr);
              wi[k] = *reinterpret_cast<const uint32_t*>(&hi);
              if (p + 1 < NP) {  // the residual for the next piece (none after the last)
                re[it][2 * k] -= __low2float(hr);
                re[it][2 * k + 1] -= __high2float(hr);
                im[it][2 * k] -= __low2float(hi);
                im[it][2 * k + 1] -= __high2float(hi);
              }
            }
            // even z rows store re first, odd ones im first: each store instruction of a warp then
            // covers all eight 16-byte bank groups
            unsigned char* Pp = A + p * 8192;
            const bool odd = zl & 1;
            const uint4 vr = make_uint4(wr[0], wr[1], wr[2], wr[3]), vi = make_uint4(wi[0], wi[1], wi[2], wi[3]);
            *reinterpret_cast<uint4*>(Pp + (odd ? off_im : off_re)) = odd ? vi : vr;
            *reinterpret_cast<uint4*>(Pp + (odd ? off_re : off_im)) = odd ? vr : vi;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&sb->fullA[s]);
        busy += clock64() - c1;
      }
    }
    if (threadIdx.x == 0) {
      add_waits(gp.waits, kWaitStaged, w_staged);
      add_waits(gp.waits, kBusyConv, busy);
    }
  } else if (warp < kConvWarps + kEpiWarps) {
    // ---- epilogue: TMEM -> coef[md][g*3+ob][j][2 Nz] (complex, re/im from adjacent rows); TMEM lane quarter
    // = warp mod 4
    const int quarter = warp & 3;
    int it = 0;
    long long busy = 0;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x, ++it) {
      const int4 tl = tiles[ti];
      int md, g, ob;
      decode(tl, md, g, ob);
      const GInst& I = gp.inst[tl.x];
      const int b = NBUF == 2 ? (it & 1) : 0;
      const uint32_t use = (uint32_t)(NBUF == 2 ? (it >> 1) : it);
      if (!mbar_wait(&sb->tfull[b], use & 1u, abort, gp.spin)) {
        if (lane == 0) record_error(I.err, 14);
        break;
      }
      const long long c1 = clock64();
      tc_fence_after();
      const int n = I.n, Nz = I.Nz, z0 = tl.z, j0 = tl.w;
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * NACC * TN);
      // 32-column chunks that hold outputs j < n; NACC = 1 reads its single accumulator twice (the
      // second copy unused) so that both forms share one load instruction pair
      const int nch = (tile_n(TN, n, j0) + 31) >> 5;
      const int half = (warp - kConvWarps) >> 2;  // which of the two warps of this lane quarter
      const uint32_t corr = NACC == 2 ? (uint32_t)TN : 0u;
      // lanes 4g .. 4g+3 hold four consecutive rows (contiguous in memory along z, re/im); a 4 x 4 transpose
      // over each such group leaves lane 4g + q with column q of the block, so that it stores the four rows
      // as one 16-byte vector: 8 vector stores per 32 columns instead of 32 scalar ones
      const int q = lane & 3;
      float* const out4 = I.coef + (size_t)(md * 9 + g * 3 + ob) * n * 2 * Nz + 2 * z0 + quarter * 32 + (lane & ~3);
      for (int ch = half; ch < nch; ch += 2) {
        const int c0 = 32 * ch;
        uint32_t lead[32], cr[32];
        tmem_ld2x32(tbase + c0, tbase + corr + c0, lead, cr);  // both accumulators, one wait
        tmem_wait2(lead, cr);
#pragma unroll
        for (int b4 = 0; b4 < 8; ++b4) {
          float x[4];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int i = 4 * b4 + m;
            x[m] = NACC == 2 ? __uint_as_float(lead[i]) + __uint_as_float(cr[i]) : __uint_as_float(lead[i]);
          }
          transpose4(x, q);
          const int j = j0 + c0 + 4 * b4 + q;
          if (j < n) *reinterpret_cast<float4*>(out4 + (size_t)j * 2 * Nz) = make_float4(x[0], x[1], x[2], x[3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sb->tempty[b]);
      busy += clock64() - c1;
    }
    if (warp == kConvWarps && lane == 0) add_waits(gp.waits, kBusyEpi, busy);
  } else if (warp == kConvWarps + kEpiWarps) {
    // ---- producer: the FP32 field tile (TMA) and the pre-tiled P pieces (bulk copies)
    int q = 0;
    bool live = true;
    long long w_stage = 0;
    for (int ti = blockIdx.x; live && ti < ntiles; ti += gridDim.x) {
      const int4 tl = tiles[ti];
      int md, g, ob, bl[2];
      decode(tl, md, g, ob);
      const GInst& I = gp.inst[tl.x];
      const int n = I.n, Nz = I.Nz, nks = (n + 31) >> 5, z0 = tl.z, j0 = tl.w;
      const int T = proj_blocks(g, ob, bl) * nks;
      const uint32_t bbytes = (uint32_t)tile_n(TN, n, j0) * 64u;  // one B piece: ne rows of 32 K bf16
      for (int t = 0; t < T; ++t, ++q) {
        const int s = q % S;
        const uint32_t ph = (uint32_t)(q / S) & 1u;
        bool ok = true;
        const long long c0 = clock64();
        if (lane == 0) ok = mbar_wait(&sb->empty[s], ph ^ 1u, abort, gp.spin);
        w_stage += clock64() - c0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) record_error(I.err, 12);
          live = false;
          break;
        }
        const int ib = bl[t / nks], rs = t % nks, r0 = rs * 32;
        if (lane == 0) {
          // FP32 field tile: 64 z rows x 32 complex, one TMA box (radii beyond Nr are zero-filled); a single
          // 16 KB box arrives sooner than two 128-byte-swizzled halves, whose conflict-free reads did not pay
          mbar_expect_tx(&sb->fullS[s], 64u * 256u);
          const CUtensorMap* map = g == 2 ? &gp.jmap[tl.x] : &gp.fmap[tl.x];
          const int field = g == 2 ? ib : ((g == 1) ? (ib == 0 ? 4 : (ib == 1 ? 3 : 5)) : ib);
          tma_load_2d(stage_A(s), map, &sb->fullS[s], 2 * r0, (md * (g == 2 ? 3 : 6) + field) * Nz + z0);
          mbar_expect_tx(&sb->fullB[s], (uint32_t)NP * bbytes);
        }
        __syncwarp();
        if (lane < NP) {
          // P block (md, g, piece, ob, ib, rs, jb): 128 rows x 32 K, 8 KB; the tile's rows j0 .. j0 + ne - 1
          // are contiguous over consecutive jb blocks (whole 8-row swizzle atoms, ne a multiple of 16)
          const size_t blk = (((((size_t)(md * 2 + (g == 1 ? 1 : 0)) * NP + lane) * 3 + ob) * 3 + ib) * nks + rs) *
                                 I.njb +
                             (j0 >> 7);
          bulk_g2s(stage_B(s) + lane * C::kBp, I.P + blk * 8192, bbytes, &sb->fullB[s]);
        }
      }
    }
    if (lane == 0) add_waits(gp.waits, kWaitStage, w_stage);
    // after an abort: wait (bounded) for the copies already issued that no consumer will wait for
    if (!live && lane == 0) {
      for (int k = 1; k <= S; ++k) {
        const int qq = q - k;
        if (qq < 0) break;
        mbar_drain(&sb->fullS[qq % S], (uint32_t)(qq / S) & 1u);
        mbar_drain(&sb->fullB[qq % S], (uint32_t)(qq / S) & 1u);
      }
    }
  } else {
    // ---- MMA issuer
    if (lane == 0) {
      int q = 0, it = 0;
      bool live = true;
      const long long t_start = clock64();
      long long w_a = 0, w_b = 0, w_tmem = 0;
      for (int ti = blockIdx.x; live && ti < ntiles; ti += gridDim.x, ++it) {
        const int4 tl = tiles[ti];
        int md, g, ob, bl[2];
        decode(tl, md, g, ob);
        const GInst& I = gp.inst[tl.x];
        const int nks = (I.n + 31) >> 5;
        const int T = proj_blocks(g, ob, bl) * nks;
        const uint32_t idesc = idesc_bf16(tile_n(TN, I.n, tl.w), false);
        const int b = NBUF == 2 ? (it & 1) : 0;
        const uint32_t use = (uint32_t)(NBUF == 2 ? (it >> 1) : it);
        const long long c0 = clock64();
        const bool freed = mbar_wait(&sb->tempty[b], (use & 1u) ^ 1u, abort, gp.spin);
        w_tmem += clock64() - c0;
        if (!freed) {
          record_error(I.err, 15);
          break;
        }
        tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)(b * NACC * TN);
        for (int t = 0; t < T; ++t, ++q) {
          const int s = q % S;
          const uint32_t ph = (uint32_t)(q / S) & 1u;
          const long long c1 = clock64();
          const bool okA = mbar_wait(&sb->fullA[s], ph, abort, gp.spin);
          const long long c2 = clock64();
          const bool okB = okA && mbar_wait(&sb->fullB[s], ph, abort, gp.spin);
          w_a += c2 - c1;
          w_b += clock64() - c2;
          if (!okB) {
            record_error(I.err, 13);
            live = false;
            break;
          }
          tc_fence_after();
          unsigned char* As = stage_A(s);
          unsigned char* Bs = stage_B(s);
#pragma unroll
          for (int k16 = 0; k16 < 2; ++k16) {
#pragma unroll
            for (int pr = 0; pr < (NP == 2 ? 3 : 6); ++pr) {
              int ia, ibp;
              product<NP>(pr, ia, ibp);
              const int acc = (NACC == 2 && pr > 0) ? 1 : 0;
              const bool first = t == 0 && k16 == 0 && (pr == 0 || (NACC == 2 && pr == 1));
              mma_bf16(d0 + (uint32_t)(acc * TN), desc_sw64(As + ia * 8192 + k16 * 32),
                       desc_sw64(Bs + ibp * C::kBp + k16 * 32), idesc, first ? 0u : 1u);
            }
          }
          mma_commit(&sb->empty[s]);
        }
        if (live) mma_commit(&sb->tfull[b]);
      }
      mma_commit(&sb->done);
      mbar_drain(&sb->done, 0);
      add_waits(gp.waits, kWaitCta, clock64() - t_start);
      add_waits(gp.waits, kWaitA, w_a);
      add_waits(gp.waits, kWaitB, w_b);
      add_waits(gp.waits, kWaitTmem, w_tmem);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kCols));
  }
}

// ------------------------------------------------------------------ back-projection

template <int NP, int NACC, int NBUF, int TN>
struct BG {
  static constexpr uint32_t kA = 16384u;      // one piece of the Q tile: 128 r x 64 j
  static constexpr uint32_t kBp = TN * 128u;  // one piece of the coefficient tile: 64 j x TN (z, part)
  static constexpr uint32_t kStage = NP * (kA + kBp);
  static constexpr int S0 = (int)((220u * 1024u) / kStage);
  static constexpr int S = S0 > 6 ? 6 : S0;
  static constexpr size_t kSmem = (size_t)S * kStage + 1024 + sizeof(GBar) + 64;
  static constexpr int kCols = NACC * NBUF * TN;
  static_assert(kCols <= 512 && (kCols & (kCols - 1)) == 0, "TMEM columns");
  static_assert(S >= 2, "pipeline depth");
};

template <int NP, int NACC, int NBUF, int TN>
__global__ void __launch_bounds__(192, 1) tcg_backproject_kernel(const __grid_constant__ GroupParams gp,
                                                                  const int4* __restrict__ tiles, int ntiles) {
  typedef BG<NP, NACC, NBUF, TN> C;
  constexpr int S = C::S;
  extern __shared__ __align__(1024) unsigned char raw[];
  unsigned char* base = align1024(raw);
  GBar* sb = reinterpret_cast<GBar*>(base + S * C::kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &sb->abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&sb->fullB[s], 1);
      mbar_init(&sb->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sb->tfull[b], 1);
      mbar_init(&sb->tempty[b], 4);
    }
    mbar_init(&sb->done, 1);
    sb->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sb->tmem_base)),
                 "r"(C::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sb->tmem_base;
  auto stage_A = [&](int s) { return base + (size_t)s * C::kStage; };
  auto stage_B = [&](int s) { return base + (size_t)s * C::kStage + NP * C::kA; };
  unsigned long long* const waits = gp.waits ? gp.waits + 8 : nullptr;

  if (warp < 4) {
    // ---- epilogue: TMEM rows r, columns (z, part) -> fields[md][field][z][r]
    const int quarter = warp;
    int it = 0;
    long long busy = 0;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x, ++it) {
      const int4 tl = tiles[ti];
      int md, g, fb;
      decode(tl, md, g, fb);
      const GInst& I = gp.inst[tl.x];
      const int b = NBUF == 2 ? (it & 1) : 0;
      const uint32_t use = (uint32_t)(NBUF == 2 ? (it >> 1) : it);
      if (!mbar_wait(&sb->tfull[b], use & 1u, abort, gp.spin)) {
        if (lane == 0) record_error(I.err, 24);
        break;
      }
      const long long c1 = clock64();
      tc_fence_after();
      const int n = I.n, Nz = I.Nz, z0 = tl.z;
      const int r = tl.w + quarter * 32 + lane;
      const int field = g == 0 ? fb : (fb == 0 ? 4 : (fb == 1 ? 3 : 5));
      const bool rot = (g == 0) ? (fb == 1) : (fb >= 1);
      float2* out = I.fields + ((size_t)md * 6 + field) * Nz * n + r;
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * NACC * TN);
      for (int c0 = 0; c0 < TN; c0 += 32) {
        float v[32];
        tmem_ld32(tbase + c0, v);
        if (NACC == 2) {
          float w[32];
          tmem_ld32(tbase + TN + c0, w);
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] += w[i];
        }
        if (r < n) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int z = z0 + c0 / 2 + i;
            float2 o = make_float2(v[2 * i], v[2 * i + 1]);
            if (rot) o = make_float2(-o.y, o.x);  // 1/tau = i
            out[(size_t)z * n] = o;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sb->tempty[b]);
      busy += clock64() - c1;
    }
    if (warp == 0 && lane == 0) add_waits(waits, kBusyEpi, busy);
  } else if (warp == 4) {
    // ---- producer: pre-tiled Q pieces and coefficient pieces, one bulk copy each per piece
    if (lane == 0) {
      int q = 0;
      bool live = true;
      long long w_stage = 0;
      for (int ti = blockIdx.x; live && ti < ntiles; ti += gridDim.x) {
        const int4 tl = tiles[ti];
        int md, g, fb, bl[2];
        decode(tl, md, g, fb);
        const GInst& I = gp.inst[tl.x];
        const int ks = (I.n + 63) >> 6, nzb = I.Nz >> 6, nrb = (I.n + 127) >> 7;
        const int T = back_blocks(g, fb, bl) * ks;
        for (int t = 0; t < T; ++t, ++q) {
          const int s = q % S;
          const uint32_t ph = (uint32_t)(q / S) & 1u;
          const long long c0 = clock64();
          const bool freed = mbar_wait(&sb->empty[s], ph ^ 1u, abort, gp.spin);
          w_stage += clock64() - c0;
          if (!freed) {
            record_error(I.err, 21);
            live = false;
            break;
          }
          const int cb = bl[t / ks], kk = t % ks;
          mbar_expect_tx(&sb->fullB[s], (uint32_t)NP * (C::kA + C::kBp));
          for (int p = 0; p < NP; ++p) {
            // Q block (md, g, piece, fb, cb, ks, rb): 128 r x 64 j, 16 KB
            const size_t qa = (((((size_t)(md * 2 + g) * NP + p) * 3 + fb) * 3 + cb) * ks + kk) * nrb + (tl.w >> 7);
            bulk_g2s(stage_A(s) + p * C::kA, I.Q + qa * 16384, C::kA, &sb->fullB[s]);
            // coefficient block (md, piece, c, ks, zb): 64 j x 64 z x re/im, 16 KB; TN/128 consecutive zb
            const size_t sa = ((((size_t)md * NP + p) * 6 + g * 3 + cb) * ks + kk) * nzb + (tl.z >> 6);
            bulk_g2s(stage_B(s) + p * C::kBp, I.S + sa * 16384, C::kBp, &sb->fullB[s]);
          }
        }
      }
      add_waits(waits, kWaitStage, w_stage);
      if (!live) {
        for (int k = 1; k <= S; ++k) {
          const int qq = q - k;
          if (qq < 0) break;
          mbar_drain(&sb->fullB[qq % S], (uint32_t)(qq / S) & 1u);
        }
      }
    }
  } else {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TN, true);
      int q = 0, it = 0;
      bool live = true;
      const long long t_start = clock64();
      long long w_b = 0, w_tmem = 0;
      for (int ti = blockIdx.x; live && ti < ntiles; ti += gridDim.x, ++it) {
        const int4 tl = tiles[ti];
        int md, g, fb, bl[2];
        decode(tl, md, g, fb);
        const GInst& I = gp.inst[tl.x];
        const int ks = (I.n + 63) >> 6;
        const int T = back_blocks(g, fb, bl) * ks;
        const int b = NBUF == 2 ? (it & 1) : 0;
        const uint32_t use = (uint32_t)(NBUF == 2 ? (it >> 1) : it);
        const long long c0 = clock64();
        const bool freed = mbar_wait(&sb->tempty[b], (use & 1u) ^ 1u, abort, gp.spin);
        w_tmem += clock64() - c0;
        if (!freed) {
          record_error(I.err, 25);
          break;
        }
        tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)(b * NACC * TN);
        for (int t = 0; t < T; ++t, ++q) {
          const int s = q % S;
          const uint32_t ph = (uint32_t)(q / S) & 1u;
          const long long c1 = clock64();
          const bool okB = mbar_wait(&sb->fullB[s], ph, abort, gp.spin);
          w_b += clock64() - c1;
          if (!okB) {
            record_error(I.err, 23);
            live = false;
            break;
          }
          tc_fence_after();
          unsigned char* As = stage_A(s);
          unsigned char* Bs = stage_B(s);
#pragma unroll
          for (int k16 = 0; k16 < 4; ++k16) {
#pragma unroll
            for (int pr = 0; pr < (NP == 2 ? 3 : 6); ++pr) {
              int ia, ibp;
              product<NP>(pr, ia, ibp);
              const int acc = (NACC == 2 && pr > 0) ? 1 : 0;
              const bool first = t == 0 && k16 == 0 && (pr == 0 || (NACC == 2 && pr == 1));
              const uint64_t ad = smem_desc(As + ia * C::kA + k16 * 32, 16, 1024, 2);
              // MN-major B: 64-element (128 B) rows along N, 16 K rows per MMA; N chunks 8 KB apart
              const uint64_t bd = smem_desc(Bs + ibp * C::kBp + k16 * 16 * 128, 8192, 1024, 2);
              mma_bf16(d0 + (uint32_t)(acc * TN), ad, bd, idesc, first ? 0u : 1u);
            }
          }
          mma_commit(&sb->empty[s]);
        }
        if (live) mma_commit(&sb->tfull[b]);
      }
      mma_commit(&sb->done);
      mbar_drain(&sb->done, 0);
      add_waits(waits, kWaitCta, clock64() - t_start);
      add_waits(waits, kWaitB, w_b);
      add_waits(waits, kWaitTmem, w_tmem);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kCols));
  }
}

}  // namespace

// ------------------------------------------------------------------ host side

struct TcGroup {
  int np = 0;
  std::vector<TcPlan*> plans;
  GroupParams params;
  TcConfig cfg;
  int4* d_ptiles = nullptr;
  int4* d_btiles = nullptr;
  int nptiles = 0, nbtiles = 0;
  int grid_p = 0, grid_b = 0;
};

struct TcPlan {
  int Nz = 0, n = 0, nmodes = 0, np = 0;
  int njb = 0;  // projection: 128-row j blocks (n padded to 256)
  int nks = 0;  // projection: 32-wide r stages
  int ksb = 0;  // back-projection: 64-wide j stages
  int nrb = 0;  // back-projection: 128-row r blocks
  uint8_t* d_P = nullptr;
  uint8_t* d_Q = nullptr;
  __nv_bfloat16* d_split = nullptr;
  int* d_err = nullptr;  // owned by the caller's plan
  size_t bytes = 0;
  TcConfig cfg;
  long long spin = -1;   // pipeline wait limit of the single-instance launches (< 0: kSpinLimit)
  unsigned long long* waits = nullptr;  // pipeline cycle counters of the single-instance launches (or null)
  // one-instance groups used by tc_project / tc_backproject, without (0) and with (1) a current:
  // the tile tables depend only on the shapes, the pointers are kernel parameters
  TcGroup* self[2] = {nullptr, nullptr};
  int last = 0;
};

static void split_bf16(double x, int np, uint16_t* out) {
  double r = x;
  for (int p = 0; p < np; ++p) {
    __nv_bfloat16 h = __float2bfloat16_rn((float)r);
    memcpy(&out[p], &h, 2);
    r -= (double)__bfloat162float(h);
  }
}

// P [nmodes][2][3n][3n] (rows: output block ob, j; columns: input block ib, r) -> pieces in
// 8 KB blocks (md, g, piece, ob, ib, rs, jb) of 128 j rows x 32 r, 64B-swizzled rows.
static std::vector<uint8_t> tile_P(const double* P, int nmodes, int n, int np, int nks, int njb) {
  const int N3 = 3 * n;
  std::vector<uint8_t> out((size_t)nmodes * 2 * np * 9 * nks * njb * 8192, 0);
  uint16_t pcs[3];
  for (int md = 0; md < nmodes; ++md)
    for (int g = 0; g < 2; ++g) {
      const double* src = P + (size_t)(md * 2 + g) * N3 * N3;
      for (int ob = 0; ob < 3; ++ob)
        for (int ib = 0; ib < 3; ++ib)
          for (int j = 0; j < n; ++j)
            for (int r = 0; r < n; ++r) {
              const double v = src[(size_t)(ob * n + j) * N3 + ib * n + r];
              if (v == 0.0) continue;
              split_bf16(v, np, pcs);
              const int rs = r >> 5, rc = r & 31, jb = j >> 7, jr = j & 127;
              const size_t off = (size_t)jr * 64 + (((rc >> 3) ^ ((jr >> 1) & 3)) << 4) + (rc & 7) * 2;
              for (int p = 0; p < np; ++p) {
                const size_t blk = (((((size_t)(md * 2 + g) * np + p) * 3 + ob) * 3 + ib) * nks + rs) * njb + jb;
                memcpy(&out[blk * 8192 + off], &pcs[p], 2);
              }
            }
    }
  return out;
}

// Q [nmodes][2][3n][3n] (rows: field block fb, r; columns: coefficient block cb, j) -> pieces in
// 16 KB blocks (md, g, piece, fb, cb, ks, rb) of 128 r rows x 64 j, 128B-swizzled rows.
static std::vector<uint8_t> tile_Q(const double* Q, int nmodes, int n, int np, int ksb, int nrb) {
  const int N3 = 3 * n;
  std::vector<uint8_t> out((size_t)nmodes * 2 * np * 9 * ksb * nrb * 16384, 0);
  uint16_t pcs[3];
  for (int md = 0; md < nmodes; ++md)
    for (int g = 0; g < 2; ++g) {
      const double* src = Q + (size_t)(md * 2 + g) * N3 * N3;
      for (int fb = 0; fb < 3; ++fb)
        for (int cb = 0; cb < 3; ++cb)
          for (int r = 0; r < n; ++r)
            for (int j = 0; j < n; ++j) {
              const double v = src[(size_t)(fb * n + r) * N3 + cb * n + j];
              if (v == 0.0) continue;
              split_bf16(v, np, pcs);
              const int ks = j >> 6, jc = j & 63, rb = r >> 7, rr = r & 127;
              const size_t off = (size_t)rr * 128 + (((jc >> 3) ^ (rr & 7)) << 4) + (jc & 7) * 2;
              for (int p = 0; p < np; ++p) {
                const size_t blk = (((((size_t)(md * 2 + g) * np + p) * 3 + fb) * 3 + cb) * ksb + ks) * nrb + rb;
                memcpy(&out[blk * 16384 + off], &pcs[p], 2);
              }
            }
    }
  return out;
}

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

// FP32 view of a complex array with `rows` rows of n values (2 n floats), boxes of 32 complex x 64 rows
static bool encode_rows(CUtensorMap* m, const void* ptr, int n, long rows) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)2 * n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)2 * n * 4};
  cuuint32_t box[2] = {64, 64};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// (re-)encodes instance k's field / current maps for the pointers in params.inst[k]
static bool encode_instance(GroupParams& gp, int k, int nmodes) {
  const GInst& I = gp.inst[k];
  if (!encode_rows(&gp.fmap[k], I.fields, I.n, (long)nmodes * 6 * I.Nz)) return false;
  if (I.J && !encode_rows(&gp.jmap[k], I.J, I.n, (long)nmodes * 3 * I.Nz)) return false;
  return true;
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Orders tiles for the static round-robin schedule of the persistent kernels: sched 0 sorts by
// cost (K stages), longest first, so the last round of every CTA holds the short tiles; sched 1
// additionally walks each round in alternating direction (snake) so CTAs that drew long tiles in
// one round draw short ones in the next.
static void order_tiles(std::vector<std::pair<int, int4>>& t, int sched, int grid) {
  std::stable_sort(t.begin(), t.end(),
                   [](const std::pair<int, int4>& a, const std::pair<int, int4>& b) { return a.first > b.first; });
  if (sched == 1) {
    size_t round = 0;
    for (size_t r0 = 0; r0 < t.size(); r0 += grid, ++round)
      if (round & 1) std::reverse(t.begin() + r0, t.begin() + std::min(t.size(), r0 + (size_t)grid));
  }
}

static cudaError_t upload_tiles(const std::vector<std::pair<int, int4>>& t, int4** dptr) {
  if (*dptr) cudaFree(*dptr);
  *dptr = nullptr;
  std::vector<int4> h(t.size());
  for (size_t i = 0; i < t.size(); ++i) h[i] = t[i].second;
  cudaError_t e = cudaMalloc(dptr, std::max<size_t>(1, h.size()) * sizeof(int4));
  if (e == cudaSuccess && !h.empty()) e = cudaMemcpy(*dptr, h.data(), h.size() * sizeof(int4), cudaMemcpyHostToDevice);
  return e;
}

static cudaError_t build_tiles(TcGroup* G) {
  const TcConfig& c = G->cfg;
  std::vector<std::pair<int, int4>> pt, bt;
  for (size_t k = 0; k < G->plans.size(); ++k) {
    const TcPlan* t = G->plans[k];
    const bool hasJ = G->params.inst[k].J != nullptr;
    const int ngroups = hasJ ? 3 : 2;
    for (int md = 0; md < t->nmodes; ++md)
      for (int g = 0; g < ngroups; ++g)
        for (int ob = 0; ob < 3; ++ob) {
          const bool single = (g != 1 && ob == 0) || (g == 1 && ob == 2);
          for (int j0 = 0; j0 < t->n; j0 += c.tn_p) {
            const int cost = (single ? 1 : 2) * t->nks * tile_n(c.tn_p, t->n, j0);  // stages x MMA width
            for (int z0 = 0; z0 < t->Nz; z0 += 64)
              pt.push_back({cost, make_int4((int)k, md | g << 8 | ob << 12, z0, j0)});
          }
        }
    for (int md = 0; md < t->nmodes; ++md)
      for (int g = 0; g < 2; ++g)
        for (int fb = 0; fb < 3; ++fb) {
          const int cost = (fb == 2 ? 1 : 2) * t->ksb;
          for (int r0 = 0; r0 < t->n; r0 += 128)
            for (int z0 = 0; z0 < t->Nz; z0 += c.tn_b / 2)
              bt.push_back({cost, make_int4((int)k, md | g << 8 | fb << 12, z0, r0)});
        }
  }
  const int sms = num_sms();
  G->grid_p = (int)std::min<size_t>(pt.size(), (size_t)sms);
  G->grid_b = (int)std::min<size_t>(bt.size(), (size_t)sms);
  order_tiles(pt, c.sched_p, std::max(1, G->grid_p));
  order_tiles(bt, c.sched_b, std::max(1, G->grid_b));
  G->nptiles = (int)pt.size();
  G->nbtiles = (int)bt.size();
  cudaError_t e = upload_tiles(pt, &G->d_ptiles);
  if (e == cudaSuccess) e = upload_tiles(bt, &G->d_btiles);
  return e;
}

bool tc_config_valid(const TcPlan* const* plans, int count, const TcConfig& c) {
  if (c.tn_p != 128 && c.tn_p != 256) return false;
  if (c.tn_b != 128 && c.tn_b != 256) return false;
  if (c.sched_p < 0 || c.sched_p > 1 || c.sched_b < 0 || c.sched_b > 1) return false;
  for (int k = 0; k < count; ++k) {
    if (plans[k]->np == 3 && c.tn_b != 128) return false;  // 3 pieces of a 256-wide tile leave one stage
    if (plans[k]->Nz % (c.tn_b / 2)) return false;         // a back-projection tile spans tn_b / 2 z values
  }
  return true;
}

template <typename K>
static cudaError_t opt_in(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static cudaError_t opt_in_all() {
  static cudaError_t done = cudaErrorNotReady;
  if (done != cudaErrorNotReady) return done;
  cudaError_t e = cudaSuccess;
#define OPTP(NP, NA, NB, TN) \
  if (e == cudaSuccess) e = opt_in(tcg_project_kernel<NP, NA, NB, TN>, PG<NP, NA, NB, TN>::kSmem);
#define OPTB(NP, NA, NB, TN) \
  if (e == cudaSuccess) e = opt_in(tcg_backproject_kernel<NP, NA, NB, TN>, BG<NP, NA, NB, TN>::kSmem);
  OPTP(2, 1, 2, 128) OPTP(2, 1, 2, 256) OPTP(3, 2, 2, 128) OPTP(3, 2, 1, 256)
  OPTB(2, 1, 2, 128) OPTB(2, 1, 2, 256) OPTB(3, 2, 2, 128)
#undef OPTP
#undef OPTB
  done = e;
  return e;
}

static cudaError_t launch_project(const TcGroup* G, cudaStream_t st) {
  if (!G->nptiles) return cudaSuccess;
  const dim3 grid(G->grid_p);
  if (G->np == 2) {
    if (G->cfg.tn_p == 256)
      tcg_project_kernel<2, 1, 2, 256><<<grid, kProjThreads, PG<2, 1, 2, 256>::kSmem, st>>>(G->params, G->d_ptiles, G->nptiles);
    else
      tcg_project_kernel<2, 1, 2, 128><<<grid, kProjThreads, PG<2, 1, 2, 128>::kSmem, st>>>(G->params, G->d_ptiles, G->nptiles);
  } else {
    if (G->cfg.tn_p == 256)
      tcg_project_kernel<3, 2, 1, 256><<<grid, kProjThreads, PG<3, 2, 1, 256>::kSmem, st>>>(G->params, G->d_ptiles, G->nptiles);
    else
      tcg_project_kernel<3, 2, 2, 128><<<grid, kProjThreads, PG<3, 2, 2, 128>::kSmem, st>>>(G->params, G->d_ptiles, G->nptiles);
  }
  return cudaGetLastError();
}

static cudaError_t launch_backproject(const TcGroup* G, cudaStream_t st) {
  if (!G->nbtiles) return cudaSuccess;
  const dim3 grid(G->grid_b);
  if (G->np == 2) {
    if (G->cfg.tn_b == 256)
      tcg_backproject_kernel<2, 1, 2, 256>
          <<<grid, 192, BG<2, 1, 2, 256>::kSmem, st>>>(G->params, G->d_btiles, G->nbtiles);
    else
      tcg_backproject_kernel<2, 1, 2, 128>
          <<<grid, 192, BG<2, 1, 2, 128>::kSmem, st>>>(G->params, G->d_btiles, G->nbtiles);
  } else {
    tcg_backproject_kernel<3, 2, 2, 128>
        <<<grid, 192, BG<3, 2, 2, 128>::kSmem, st>>>(G->params, G->d_btiles, G->nbtiles);
  }
  return cudaGetLastError();
}

TcConfig tc_default_config(int np) {
  (void)np;
  TcConfig c;
  c.tn_p = 256;
  c.tn_b = 128;
  c.sched_p = 0;
  c.sched_b = 0;
  return c;
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
  cudaError_t e = opt_in_all();
  if (e != cudaSuccess) {
    snprintf(msg, msglen, "shared-memory opt-in failed");
    return e;
  }
  TcPlan* t = new TcPlan();
  t->Nz = Nz;
  t->n = n;
  t->nmodes = nmodes;
  t->np = np;
  t->njb = (n + 255) / 256 * 2;
  t->nks = (n + 31) / 32;
  t->ksb = (n + 63) / 64;
  t->nrb = (n + 127) / 128;
  t->cfg = tc_default_config(np);
  std::vector<uint8_t> hp = tile_P(P, nmodes, n, np, t->nks, t->njb);
  std::vector<uint8_t> hq = tile_Q(Q, nmodes, n, np, t->ksb, t->nrb);
  const size_t split_bytes = (size_t)nmodes * np * 6 * t->ksb * (Nz / 64) * 16384;
  e = cudaMalloc(&t->d_P, hp.size());
  if (e == cudaSuccess) e = cudaMalloc(&t->d_Q, hq.size());
  if (e == cudaSuccess) e = cudaMalloc(&t->d_split, split_bytes);
  if (e == cudaSuccess) e = cudaMemcpy(t->d_P, hp.data(), hp.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t->d_Q, hq.data(), hq.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(t->d_split, 0, split_bytes);
  if (e != cudaSuccess) {
    snprintf(msg, msglen, "allocation/upload failed");
    tc_destroy(t);
    return e;
  }
  t->d_err = err;
  t->bytes = hp.size() + hq.size() + split_bytes;
  *outp = t;
  return cudaSuccess;
}

void tc_destroy(TcPlan* t) {
  if (!t) return;
  for (TcGroup*& g : t->self)
    if (g) tc_group_destroy(g);
  if (t->d_P) cudaFree(t->d_P);
  if (t->d_Q) cudaFree(t->d_Q);
  if (t->d_split) cudaFree(t->d_split);
  delete t;
}

size_t tc_device_bytes(const TcPlan* t) { return t ? t->bytes : 0; }
__nv_bfloat16* tc_split_buffer(TcPlan* t) { return t->d_split; }
int tc_split_kstages(const TcPlan* t) { return t->ksb; }
int tc_pieces(const TcPlan* t) { return t->np; }
TcConfig tc_plan_config(const TcPlan* t) { return t->cfg; }

cudaError_t tc_plan_set_config(TcPlan* t, const TcConfig& c) {
  const TcPlan* pl[1] = {t};
  if (!tc_config_valid(pl, 1, c)) return cudaErrorInvalidValue;
  t->cfg = c;
  for (TcGroup*& g : t->self)
    if (g) {
      tc_group_destroy(g);
      g = nullptr;
    }
  return cudaSuccess;
}

cudaError_t tc_group_create(TcGroup** out, TcPlan* const* plans, const void* const* fields, const void* const* J,
                            int count, const TcConfig& cfg) {
  *out = nullptr;
  if (count < 1 || count > kMaxGroupInstances) return cudaErrorInvalidValue;
  const int np = plans[0]->np;
  for (int k = 0; k < count; ++k)
    if (plans[k]->np != np) return cudaErrorInvalidValue;
  if (!tc_config_valid(plans, count, cfg)) return cudaErrorInvalidValue;
  TcGroup* G = new TcGroup();
  G->np = np;
  G->cfg = cfg;
  memset(&G->params, 0, sizeof(G->params));
  for (int k = 0; k < count; ++k) {
    TcPlan* t = plans[k];
    G->plans.push_back(t);
    GInst& I = G->params.inst[k];
    I.fields = (float2*)fields[k];
    I.J = (const float2*)J[k];
    I.coef = nullptr;  // set by tc_group_set_coef
    I.P = t->d_P;
    I.Q = t->d_Q;
    I.S = (const uint8_t*)t->d_split;
    I.err = t->d_err;
    I.Nz = t->Nz;
    I.n = t->n;
    I.njb = t->njb;
    if (!encode_instance(G->params, k, t->nmodes)) {
      delete G;
      return cudaErrorInvalidValue;
    }
  }
  G->params.count = count;
  G->params.spin = kSpinLimit;
  cudaError_t e = build_tiles(G);
  if (e != cudaSuccess) {
    tc_group_destroy(G);
    return e;
  }
  *out = G;
  return cudaSuccess;
}

void tc_group_set_coef(TcGroup* G, int k, void* coef) { G->params.inst[k].coef = (float*)coef; }
// the back-projection writes through GInst.fields; the projection's tensor map is left as it is
void tc_group_set_fields(TcGroup* G, int k, void* fields) { G->params.inst[k].fields = (float2*)fields; }

void tc_group_destroy(TcGroup* G) {
  if (!G) return;
  if (G->d_ptiles) cudaFree(G->d_ptiles);
  if (G->d_btiles) cudaFree(G->d_btiles);
  delete G;
}

cudaError_t tc_group_project(TcGroup* G, cudaStream_t st) { return launch_project(G, st); }
cudaError_t tc_group_backproject(TcGroup* G, cudaStream_t st) { return launch_backproject(G, st); }
int tc_group_tiles(const TcGroup* G, int which) { return which == 0 ? G->nptiles : G->nbtiles; }

// one-instance group of a plan; built once per current on/off, pointers updated per call
static cudaError_t self_group(TcPlan* t, const void* fields, const void* J, void* coef) {
  const int h = J ? 1 : 0;
  if (!t->self[h]) {
    TcPlan* pl[1] = {t};
    const void* f[1] = {fields};
    const void* j[1] = {J};
    cudaError_t e = tc_group_create(&t->self[h], pl, f, j, 1, t->cfg);
    if (e != cudaSuccess) return e;
  }
  GroupParams& gp = t->self[h]->params;
  gp.spin = t->spin < 0 ? kSpinLimit : t->spin;
  gp.waits = t->waits;
  GInst& I = gp.inst[0];
  const bool moved = I.fields != (float2*)fields || I.J != (const float2*)J;
  I.fields = (float2*)fields;
  I.J = (const float2*)J;
  I.coef = (float*)coef;
  if (moved && !encode_instance(gp, 0, t->nmodes)) return cudaErrorInvalidValue;
  t->last = h;
  return cudaSuccess;
}

cudaError_t tc_prepare(TcPlan* t, const void* fields, const void* J, void* coef) {
  return self_group(t, fields, J, coef);
}

cudaError_t tc_project(TcPlan* t, const void* fields, const void* J, void* coef, cudaStream_t st) {
  // building the tile tables uploads synchronously, which a stream capture does not allow
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
  if (capturing && !t->self[J ? 1 : 0]) return cudaErrorStreamCaptureUnsupported;
  cudaError_t e = self_group(t, fields, J, coef);
  if (e != cudaSuccess) return e;
  return launch_project(t->self[t->last], st);
}

cudaError_t tc_backproject(TcPlan* t, void* fields, cudaStream_t st) {
  TcGroup* G = t->self[t->last];
  if (!G) return cudaErrorInvalidValue;
  G->params.inst[0].fields = (float2*)fields;
  G->params.spin = t->spin < 0 ? kSpinLimit : t->spin;
  G->params.waits = t->waits;
  return launch_backproject(G, st);
}

void tc_set_wait_limit(TcPlan* t, long long polls) { t->spin = polls < 0 ? -1 : polls; }
void tc_set_waits(TcPlan* t, unsigned long long* counters) { t->waits = counters; }
void tc_group_set_waits(TcGroup* G, unsigned long long* counters) { G->params.waits = counters; }

int tc_launches_per_step(const TcPlan*) { return 2; }

}  // namespace fdetd
