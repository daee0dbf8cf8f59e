// Spectral kernel for FP32 data, Nz = 2^LOGN in 64..4096, specialised on LOGN.
//
// Computes what the general spectral kernel (k_spectral.cu) computes for one (mode, family, j): the
// forward z-DFT of the family's coefficient columns, the exact midpoint update of every (kz, j) point
// (Eq. maxwellAM_solution2 with the 3x3 exponential of the family), the inverse z-DFT.  The transform is
// the same in-place decimation-in-frequency FFT with the same stage radices (the factor left over by
// radix 8 first, then radix 8), the same twiddle tables and the same position order of the per-kz tables,
// but every stride, padded offset and loop bound is a compile-time constant of LOGN, and each thread
// owns exactly one radix-8 butterfly per column and stage (Nz / 8 threads), so a stage is straight-line
// code: one base address per butterfly, immediate offsets, no bounds predicates.
//
// The update uses the structure of the families' matrices.  With g = e - s- a (TM) the square of
//   M_TM = [[0, 0, -lam], [0, 0, -s+], [1, -s-, 0]]
// is M_TM^2 v = (-lam g_v, -s+ g_v, -w^2 v_2), and with k = f - s+ d (TE) the square of
//   M_TE = [[0, -s+, 1], [-s-, 0, 0], [-mu, 0, 0]]
// is M_TE^2 v = (-w^2 v_0, -s- k_v, -mu k_v), w^2 = kappa^2 + lam (mu), s+ s- = -kappa^2.  Substituted into
//   x <- x + A1 M x + A2 M^2 x - dt (x_J + B1 M x_J + B2 M^2 x_J)
// (A = t dt, B = t dt / 2; A1 = sin(w t) / w, A2 = (1 - cos w t) / w^2) this gives, per (kz, j):
//   TM, x_J = (eJ, aJ, 0), gJ = eJ - s- aJ,  h = A1 b + A2 g - dt B2 gJ:
//     e' = e - dt eJ - lam h,   a' = a - dt aJ - s+ h,   b' = b - A2 (w^2 b) + A1 g - dt B1 gJ
//   TE, x_J = (cJ, 0, 0), h = A1 c + A2 k - dt B1 cJ:
//     c' = c - A2 (w^2 c) + A1 k - dt cos(w dt / 2) cJ,   d' = d - s- h,   f' = f - mu h.
// Coefficients that multiply the state (A1, A2, lam, kappa^2, s+-) are double-float (hi + lo), so that
// their rounding does not bias every step the same way; the current's coefficients are FP32.
#include "common.cuh"
#include "fft_small.cuh"
#include "kernels.h"

namespace fdetd {

namespace {

template <int LOGN>
struct Shape {
  static constexpr int N = 1 << LOGN;
  static constexpr int NT = N / 8;                  // threads: one radix-8 butterfly per column and stage
  static constexpr int S = (LOGN + 2) / 3;          // stages
  static constexpr int LR0 = LOGN - 3 * (S - 1);    // log2 of the first stage's radix (1, 2 or 3)
  static constexpr int PC = pad16(N);               // padded column length
  __host__ __device__ static constexpr int R(int s) { return s == 0 ? (1 << LR0) : 8; }
  // stride of stage s: a power of 8 (1 for the last stage)
  __host__ __device__ static constexpr int L(int s) { return N >> (LR0 + 3 * s); }
  // offset of stage s's twiddles in the table (stages back to back, (R_s - 1) L_s entries each)
  __host__ __device__ static constexpr int TWO(int s) { return s == 0 ? 0 : TWO(s - 1) + (R(s - 1) - 1) * L(s - 1); }
  static constexpr int TW = TWO(S - 1);
  // blocks per SM that keep 128 registers a thread (a block narrower than a warp still holds a warp)
  static constexpr int MINB = NT >= 512 ? 1 : (NT >= 32 ? 512 / NT : 16);
};

// Offset of element r of a butterfly of stride L from the padded address of its first element: L is a
// power of 8, so r L either keeps the low four bits of the position (L >= 16), or, for L = 8 inside a
// block of 64 and L = 1 inside an aligned run of 8, crosses a 16-element boundary at fixed r.
template <int L>
__device__ __forceinline__ constexpr int boff(int r) {
  return L >= 16 ? r * (L + L / 8) : (L == 8 ? 8 * r + 2 * (r >> 1) : r);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void l2_prefetch(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((uint64_t)src), "r"(bytes) : "memory");
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
// double-float coefficient times complex data, and its complex-coefficient form
__device__ __forceinline__ float2 dmul(df c, float2 x) { return f2(rmul(c, x.x), rmul(c, x.y)); }
__device__ __forceinline__ float2 dcmul(df re, df im, float2 x) {
  return f2(rmul(re, x.x) - rmul(im, x.y), rmul(re, x.y) + rmul(im, x.x));
}

// One in-place stage (forward, or its adjoint) of the first ncol columns.
template <int LOGN, int s, bool INV>
__device__ __forceinline__ void stage(float2* sm, const float2* tw, int ncol) {
  typedef Shape<LOGN> SH;
  constexpr int R = SH::R(s), L = SH::L(s), M = R * L, PB = 8 / R, NT = SH::NT;
#pragma unroll
  for (int u = 0; u < PB; ++u) {
    const int beta = threadIdx.x + u * NT;
    const int blk = beta / L, n1 = beta % L;
    const int p0 = blk * M + n1;
    const int base = pad16(p0);
    float2 w[R];
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = tw[SH::TWO(s) + (r - 1) * L + n1];
    // columns rolled: the butterfly's code once, not five times (instruction-cache footprint)
#pragma unroll 1
    for (int a = 0; a < ncol; ++a) {
      float2* col = sm + a * SH::PC + base;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = col[boff<L>(r)];
      if (INV) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmulconj(v[r], w[r]);
        dft_small<R, true>(v);
      } else {
        dft_small<R, false>(v);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r]);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) col[boff<L>(r)] = v[r];
    }
  }
  __syncthreads();
}

// forward stages 1 .. s (stage 0 runs column by column as the columns arrive, first_stage)
template <int LOGN, int s>
struct Forward {
  static __device__ __forceinline__ void run_after_first(float2* sm, const float2* tw, int ncol) {
    Forward<LOGN, s - 1>::run_after_first(sm, tw, ncol);
    stage<LOGN, s, false>(sm, tw, ncol);
  }
};
template <int LOGN>
struct Forward<LOGN, 0> {
  static __device__ __forceinline__ void run_after_first(float2*, const float2*, int) {}
};

// Forward stage 0 of column a once its copy group (and, for a = 0, the twiddles) has landed; the copies of
// the columns after it stay in flight.  Columns a >= ncol have empty groups and no work.
template <int LOGN, int a>
__device__ __forceinline__ void first_stage(float2* sm, const float2* tw, int ncol) {
  if constexpr (a < 5) {
    cp_wait<4 - a>();
    __syncthreads();
    if (a < ncol) stage<LOGN, 0, false>(sm + a * Shape<LOGN>::PC, tw, 1);
    first_stage<LOGN, a + 1>(sm, tw, ncol);
  }
}
// adjoint stages s .. 1 (stage 0's adjoint writes to global memory)
template <int LOGN, int s>
struct Inverse {
  static __device__ __forceinline__ void run(float2* sm, const float2* tw) {
    stage<LOGN, s, true>(sm, tw, 3);
    Inverse<LOGN, s - 1>::run(sm, tw);
  }
};
template <int LOGN>
struct Inverse<LOGN, 0> {
  static __device__ __forceinline__ void run(float2*, const float2*) {}
};

__device__ __forceinline__ void load8(const float2* p, float2* v) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 t = q[i];
    v[2 * i] = f2(t.x, t.y);
    v[2 * i + 1] = f2(t.z, t.w);
  }
}
__device__ __forceinline__ void store8(float2* p, const float2* v) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
}

// Current coefficients of the half step: B1 = sin(w dt/2) / w = sqrt(A2 / 2), ch = cos(w dt/2) = A1 / (2 B1),
// B2 = (1 - ch) / w^2 = B1^2 / (1 + ch) (half-angle identities; FP32 suffices for the source term).
__device__ __forceinline__ void half_step(const PhaseF& p, float& B1, float& B2, float& ch) {
  const float a2 = p.A2.h + p.A2.l;
  B1 = sqrtf(0.5f * fmaxf(a2, 0.f));
  ch = B1 > 0.f ? __fdividef(p.A1.h + p.A1.l, 2.f * B1) : 1.f;
  B2 = B1 > 0.f ? __fdividef(B1 * B1, 1.f + ch) : 0.f;
}

// The last forward stage (radix 8, stride 1: positions 8t .. 8t+7), the update of those eight kz and the
// first inverse stage, in registers.
template <int LOGN, bool HASJ>
__device__ __forceinline__ void fused_last(float2* sm, int fam, const PhaseF* __restrict__ phase,
                                           const ZSymK* __restrict__ zs, df lam, float dt, float inv) {
  typedef Shape<LOGN> SH;
  constexpr int NT = SH::NT;
  const int t = threadIdx.x;
  const int base = pad16(8 * t);
  float2 x[3][8];
  // the first kz's records are requested before the column transforms so that their latency overlaps them;
  // the records of kz r + 1 are loaded while kz r is updated
  PhaseF ph_next = phase[t];
  ZSymK z_next = zs[t];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    load8(sm + a * SH::PC + base, x[a]);
    dft_small<8, false>(x[a]);
  }
  float2 j0[8], j1[8];
  if (HASJ) {
    load8(sm + 3 * SH::PC + base, j0);
    dft_small<8, false>(j0);
    if (fam == 0) {
      load8(sm + 4 * SH::PC + base, j1);
      dft_small<8, false>(j1);
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const PhaseF ph = ph_next;
    const ZSymK z = z_next;
    if (r < 7) {
      ph_next = phase[(r + 1) * NT + t];
      z_next = zs[(r + 1) * NT + t];
    }
    const df A1 = ph.A1, A2 = ph.A2;
    float B1 = 0.f, B2 = 0.f, ch = 1.f;
    if (HASJ) half_step(ph, B1, B2, ch);
    const df smr = {-z.spr.h, -z.spr.l}, smi = z.spi;   // s- = (-Re s+, Im s+)
    if (fam == 0) {
      const float2 e = x[0][r], a = x[1][r], b = x[2][r];
      const float2 g = csub(e, dcmul(smr, smi, a));
      float2 h = cadd(dmul(A1, b), dmul(A2, g));
      float2 ne = e, na = a;
      float2 w2b = cadd(dmul(z.k2, b), dmul(lam, b));
      float2 nb = cadd(csub(b, dmul(A2, w2b)), dmul(A1, g));
      if (HASJ) {
        const float2 eJ = j0[r], aJ = j1[r];
        // FP32 s- for the current's term
        const float2 gJ = f2(eJ.x - (smr.h * aJ.x - smi.h * aJ.y), eJ.y - (smr.h * aJ.y + smi.h * aJ.x));
        const float dB1 = dt * B1, dB2 = dt * B2;
        h.x -= dB2 * gJ.x;
        h.y -= dB2 * gJ.y;
        ne = f2(fmaf(-dt, eJ.x, e.x), fmaf(-dt, eJ.y, e.y));
        na = f2(fmaf(-dt, aJ.x, a.x), fmaf(-dt, aJ.y, a.y));
        nb.x -= dB1 * gJ.x;
        nb.y -= dB1 * gJ.y;
      }
      ne = csub(ne, dmul(lam, h));
      na = csub(na, dcmul(z.spr, z.spi, h));
      x[0][r] = f2(ne.x * inv, ne.y * inv);
      x[1][r] = f2(na.x * inv, na.y * inv);
      x[2][r] = f2(nb.x * inv, nb.y * inv);
    } else {
      const float2 c = x[0][r], d = x[1][r], f = x[2][r];
      const float2 k = csub(f, dcmul(z.spr, z.spi, d));
      float2 h = cadd(dmul(A1, c), dmul(A2, k));
      const float2 w2c = cadd(dmul(z.k2, c), dmul(lam, c));
      float2 nc = cadd(csub(c, dmul(A2, w2c)), dmul(A1, k));
      if (HASJ) {
        const float2 cJ = j0[r];
        const float dB1 = dt * B1, dch = dt * ch;
        h.x -= dB1 * cJ.x;
        h.y -= dB1 * cJ.y;
        nc.x -= dch * cJ.x;
        nc.y -= dch * cJ.y;
      }
      const float2 nd = csub(d, dcmul(smr, smi, h));
      const float2 nf = csub(f, dmul(lam, h));
      x[0][r] = f2(nc.x * inv, nc.y * inv);
      x[1][r] = f2(nd.x * inv, nd.y * inv);
      x[2][r] = f2(nf.x * inv, nf.y * inv);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dft_small<8, true>(x[a]);
    store8(sm + a * SH::PC + base, x[a]);
  }
  __syncthreads();
}

// The adjoint of stage 0 for the three field columns, writing natural z order to global memory (or the
// back-projection's bf16 split pieces).
template <int LOGN, bool SPLIT>
__device__ __forceinline__ void stage0_out(const float2* sm, const float2* tw, float2* const* dst,
                                           const SplitColumn* sc) {
  typedef Shape<LOGN> SH;
  constexpr int R = SH::R(0), L = SH::L(0), PB = 8 / R, NT = SH::NT;
  // split pieces from full warps with a radix of 4 or 8: a 4 x 4 transpose across each group of four lanes
  // (consecutive n1) and four outputs r leaves every lane with four consecutive z, one 16-byte store per piece
  constexpr bool VEC = SPLIT && NT >= 32 && (R == 4 || R == 8);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // the split stores are kept rolled: unrolled, they push the kernel out of the instruction cache
#pragma unroll 1
    for (int u = 0; u < PB; ++u) {
      const int n1 = threadIdx.x + u * NT;
      const float2* col = sm + a * SH::PC + pad16(n1);
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = col[boff<L>(r)];
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmulconj(v[r], tw[(r - 1) * L + n1]);
      dft_small<R, true>(v);
      if constexpr (VEC) {
        const int q = threadIdx.x & 3;
#pragma unroll
        for (int h = 0; h < R / 4; ++h) {
          float xr[4], xi[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            xr[k] = v[4 * h + k].x;
            xi[k] = v[4 * h + k].y;
          }
          transpose4(xr, q);
          transpose4(xi, q);
          // lane q now holds z = (n1 - q) + k + (4 h + q) L, k = 0 .. 3
          split_store4(sc[a], (n1 & ~3) + (4 * h + q) * L, xr, xi);
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int z = n1 + r * L;
          if (!SPLIT)
            dst[a][z] = v[r];
          else
            split_store(sc[a], z, v[r].x, v[r].y);
        }
      }
    }
  }
}

// coefficient array of column a of family fam (TM: e, a, b, eJ, aJ; TE: c, d, f, cJ) in the layout
// [md][9][n][Nz] with E group (e, a, c) = 0, 1, 2, B group (b, d, f) = 3, 4, 5, J (eJ, aJ, cJ) = 6, 7, 8
__device__ __forceinline__ int column_of(int fam, int a) {
  if (fam == 0) return a < 2 ? a : (a == 2 ? 3 : a + 3);
  return a == 0 ? 2 : (a < 3 ? a + 3 : 8);
}

template <int LOGN, bool HASJ, bool SPLIT>
__global__ void __launch_bounds__(Shape<LOGN>::NT, Shape<LOGN>::MINB) spectral32_kernel(SpectralArgs args) {
  typedef Shape<LOGN> SH;
  constexpr int N = SH::N, NT = SH::NT, SLOTS = HASJ ? 5 : 3;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm + SLOTS * SH::PC;
  const int n = args.n;
  const int j = blockIdx.x, fam = blockIdx.y, md = blockIdx.z;
  const int ncol = HASJ ? (fam == 0 ? 5 : 4) : 3;
  // phase accounting (args.phases): thread 0's clock at the end of each phase; every phase ends at a barrier
  long long ck[6];
  ck[0] = clock64();
  const float2* coef = reinterpret_cast<const float2*>(args.coef);
  const PhaseF* phase = reinterpret_cast<const PhaseF*>(args.phase) + ((size_t)(md * 2 + fam) * n + j) * N;
  if (threadIdx.x == 0) l2_prefetch(phase, (uint32_t)(N * sizeof(PhaseF)));
  // the twiddles and the family's columns into the padded layout, 16 bytes per copy, one commit group per
  // column (group 0 also holds the twiddles; groups past ncol are empty): the first stage of column a runs
  // while the columns after it are still arriving
  constexpr int PER = N / 2;
  const float2* twg = reinterpret_cast<const float2*>(args.twiddle);
  for (int i = threadIdx.x; i < (SH::TW + 1) / 2; i += NT) cp16(tws + 2 * i, twg + 2 * i);
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    if (a < ncol) {
      const float2* col = coef + ((size_t)(md * 9 + column_of(fam, a)) * n + j) * N;
#pragma unroll
      for (int i = threadIdx.x; i < PER; i += NT) cp16(sm + a * SH::PC + pad16(2 * i), col + 2 * i);
    }
    cp_commit();
  }

  static_assert(SH::S >= 2, "at least two stages");
  first_stage<LOGN, 0>(sm, tws, ncol);
  ck[1] = clock64();
  Forward<LOGN, SH::S - 2>::run_after_first(sm, tws, ncol);
  ck[2] = clock64();
  const df lam = reinterpret_cast<const df*>(args.lam)[(md * 2 + fam) * n + j];
  fused_last<LOGN, HASJ>(sm, fam, phase, reinterpret_cast<const ZSymK*>(args.zsymk), lam, (float)args.dt,
                         1.0f / (float)N);
  ck[3] = clock64();
  Inverse<LOGN, SH::S - 2>::run(sm, tws);
  ck[4] = clock64();

  float2* out = reinterpret_cast<float2*>(args.coef);
  float2* dst[3];
  SplitColumn sc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dst[a] = out + ((size_t)(md * 9 + column_of(fam, a)) * n + j) * N;
    if (SPLIT) sc[a] = split_column(args.split_out, args.npieces, md, column_of(fam, a), j, args.split_kstages, N);
  }
  stage0_out<LOGN, SPLIT>(sm, tws, dst, sc);
  if (args.phases && threadIdx.x == 0) {
    ck[5] = clock64();
    // [0] residency, [1] loads and first stage, [2] other forward stages, [3] last forward stage + update +
    // first inverse stage, [4] other inverse stages, [5] output stage, [6] blocks
    atomicAdd(args.phases + 0, (unsigned long long)(ck[5] - ck[0]));
    for (int k = 1; k <= 5; ++k) atomicAdd(args.phases + k, (unsigned long long)(ck[k] - ck[k - 1]));
    atomicAdd(args.phases + 6, 1ull);
  }
}

template <int LOGN, bool HASJ, bool SPLIT>
cudaError_t launch_l(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  typedef Shape<LOGN> SH;
  const size_t smem = spectral32_smem_bytes(SH::N, HASJ);
  auto k = spectral32_kernel<LOGN, HASJ, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<dim3(a.n, 2, nmodes), SH::NT, smem, st>>>(a);
  return cudaGetLastError();
}

template <bool HASJ, bool SPLIT>
cudaError_t launch_j(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  switch (a.logNz) {
    case 6: return launch_l<6, HASJ, SPLIT>(a, nmodes, st);
    case 7: return launch_l<7, HASJ, SPLIT>(a, nmodes, st);
    case 8: return launch_l<8, HASJ, SPLIT>(a, nmodes, st);
    case 9: return launch_l<9, HASJ, SPLIT>(a, nmodes, st);
    case 10: return launch_l<10, HASJ, SPLIT>(a, nmodes, st);
    case 11: return launch_l<11, HASJ, SPLIT>(a, nmodes, st);
    case 12: return launch_l<12, HASJ, SPLIT>(a, nmodes, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

size_t spectral32_smem_bytes(int Nz, bool hasJ) {
  int logN = 0;
  while ((1 << logN) < Nz) ++logN;
  const int S = (logN + 2) / 3, LR0 = logN - 3 * (S - 1);
  size_t tw = 0;
  for (int s = 0; s + 1 < S; ++s) {
    const int R = s == 0 ? (1 << LR0) : 8;
    tw += (size_t)(R - 1) * (size_t)(Nz >> (LR0 + 3 * s));
  }
  tw = (tw + 1) & ~(size_t)1;  // whole 16-byte copies
  return ((size_t)(hasJ ? 5 : 3) * pad16(Nz) + tw) * sizeof(float2);
}

bool spectral32_supported(int Nz) { return Nz >= 64 && Nz <= 4096 && (Nz & (Nz - 1)) == 0; }

cudaError_t launch_spectral32(const SpectralArgs& a, int nmodes, bool split_out, cudaStream_t st) {
  if (!spectral32_supported(a.Nz) || !a.zsymk) return cudaErrorNotSupported;
  if (a.hasJ) return split_out ? launch_j<true, true>(a, nmodes, st) : launch_j<true, false>(a, nmodes, st);
  return split_out ? launch_j<false, true>(a, nmodes, st) : launch_j<false, false>(a, nmodes, st);
}

}  // namespace fdetd
