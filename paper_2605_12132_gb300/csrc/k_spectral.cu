// Spectral kernel: for one radial eigen-index j of one family (TM or TE) of one
// mode, transform the coefficient columns along periodic z, apply the exact
// per-kz 3x3 exponential with the midpoint current term, transform back.
//
// Per (kz, j) the TM family x = (e, a, b) evolves with
//   M_TM = [[0, 0, -lam], [0, 0, -s+], [1, -s-, 0]]
// and the TE family x = (c, d, f) with
//   M_TE = [[0, -s+, 1], [-s-, 0, 0], [-mu, 0, 0]],
// both with eigenvalues {0, +-i w}, w^2 = kappa^2 + lam (mu), so
//   exp(t M) = I + A1(t) M + A2(t) M^2,  A1 = sin(wt)/w, A2 = (1 - cos wt)/w^2.
// The step is the midpoint form of Eq. maxwellAM_solution2:
//   x <- exp(dt M) x - dt exp(dt M / 2) x_J,
// with x_J = (eJ, aJ, 0) for TM and (cJ, 0, 0) for TE (the current enters the
// Ampere equations only).  s+/s- are the DFT symbols of the periodic staggered
// z stencil D_z^(+/-) (Eq. spatial_derivativeSt along z).
//
// The z transform is an in-place mixed-radix FFT in shared memory (radix 8 for FP32,
// radix 4 for FP64, the leftover factor as the first stage): decimation in frequency forward, so
// kz comes out digit-reversed and the per-kz tables are stored in that order, and the
// adjoint stages in reverse order for the inverse, which restores natural z order.
// Each butterfly writes back where it read, so a stage needs one barrier.  The last
// forward stage, the rotation and the first inverse stage are fused in registers.
#include <vector>

#include "common.cuh"
#include "fft_small.cuh"
#include "kernels.h"

namespace fdetd {

namespace {

template <typename C, typename K>
__device__ __forceinline__ void apply_tm(const C& e, const C& a, const C& b, C& y0, C& y1, C& y2, K lam, K spr,
                                         K spi, K smr, K smi) {
  y0 = cscale(lam, b);
  y0.x = -y0.x;
  y0.y = -y0.y;
  y1 = ccoef(spr, spi, b);
  y1.x = -y1.x;
  y1.y = -y1.y;
  y2 = csub(e, ccoef(smr, smi, a));
}

template <typename C, typename K>
__device__ __forceinline__ void apply_te(const C& c, const C& d, const C& f, C& y0, C& y1, C& y2, K mu, K spr,
                                         K spi, K smr, K smi) {
  y0 = csub(f, ccoef(spr, spi, d));
  y1 = ccoef(smr, smi, c);
  y1.x = -y1.x;
  y1.y = -y1.y;
  y2 = cscale(mu, c);
  y2.x = -y2.x;
  y2.y = -y2.y;
}

__device__ __forceinline__ void phase_unpack(const PhaseD& p, double& A1, double& A2, double& B1, double& B2) {
  A1 = p.A1;
  A2 = p.A2;
  B1 = p.B1;
  B2 = p.B2;
}
// FP32 record holds A1, A2 as double-float; the half-step pair follows from half-angle identities:
// sin(th/2) = w sqrt(A2/2) -> B1 = sqrt(A2/2);  cos(th/2) = A1 / (2 B1);  B2 = B1^2 / (1 + cos(th/2)).
__device__ __forceinline__ void phase_unpack(const PhaseF& p, df& A1, df& A2, float& B1, float& B2) {
  A1 = p.A1;
  A2 = p.A2;
  const float a2 = p.A2.h + p.A2.l;
  B1 = sqrtf(0.5f * fmaxf(a2, 0.f));
  // B1 and B2 scale only the current's term: the fast reciprocal-based division (2 ulp) suffices
  const float c = B1 > 0.f ? __fdividef(p.A1.h + p.A1.l, 2.f * B1) : 1.f;
  B2 = B1 > 0.f ? __fdividef(B1 * B1, 1.f + c) : 0.f;
}
// s- = (-Re s+, Im s+)
__device__ __forceinline__ void zsym_unpack(const ZSymD& z, double& spr, double& spi, double& smr, double& smi) {
  spr = z.spr;
  spi = z.spi;
  smr = -z.spr;
  smi = z.spi;
}
__device__ __forceinline__ void zsym_unpack(const ZSymF& z, df& spr, df& spi, df& smr, df& smi) {
  spr = z.spr;
  spi = z.spi;
  smr.h = -z.spr.h;
  smr.l = -z.spr.l;
  smi = z.spi;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// bulk prefetch of `bytes` (multiple of 16, 16-byte aligned) from global memory into L2
__device__ __forceinline__ void l2_prefetch(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((uint64_t)src), "r"(bytes) : "memory");
}

// Kernel modes: FUSED transforms the family's field and current columns together; SOURCE
// transforms only the current columns and writes the midpoint source term (with the 1/Nz of the
// inverse transform) in kz space; MAIN transforms the field columns and adds that precomputed
// source (used when five columns do not fit in shared memory).
enum { FUSED = 0, MAIN = 1, SOURCE = 2 };

// Column slots a kernel of the given mode keeps in shared memory (the twiddles follow them when they are
// staged): the one count both the kernel's layout and the launcher's sizing use.
__host__ __device__ __forceinline__ constexpr int spectral_slots(int mode, bool hasJ) {
  return mode == FUSED ? (hasJ ? 5 : 3) : (mode == MAIN ? 3 : 2);
}

// ---------------------------------------------------------------- in-place transforms
// N = 2^logN = RF R^(S-1): a first stage of radix RF (the factor left over by radix R), then radix-R
// stages.  Forward: decimation in frequency; stage s has radix R_s and stride L_s = N / (R_0 ... R_s)
// (sub-transform length M_s = R_s L_s); the last stage has stride 1.  Butterfly (block, n1) of stage
// s reads the R_s elements block M_s + n1 + L_s n2, takes their DFT and multiplies output k2 by
// W_{M_s}^{n1 k2}; it writes them back where it read them, so a stage needs one barrier, after it.  The forward output at position p is the DFT at kz(p), the digit reversal
// of p (spectral_positions); the rotation tables are stored in that order.  The inverse applies the
// adjoint stages in reverse order (conjugated twiddle, then the inverse DFT), which returns natural
// order.  The twiddle table of stage s holds W_{M_s}^{n1 k2} at (k2 - 1) L_s + n1 (k2 >= 1), stages
// back to back, so the threads of a warp (consecutive n1) read consecutive entries.  The per-kz
// tables hold the record of position b RL + r (last stage of radix RL) at r (N / RL) + b, so the
// threads of a warp (consecutive b) read consecutive records.  Columns sit in shared memory in the
// padded layout pad16 (fft_small.cuh).

// 16-byte asynchronous global -> shared copy, and the wait for all of a thread's copies
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// RR consecutive complex values at p (16-byte aligned when the values are 8-byte floats)
template <int RR, typename C>
__device__ __forceinline__ void load_run(const C* p, C* v) {
  if constexpr (sizeof(C) == 8 && RR % 2 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < RR / 2; ++i) {
      const float4 t = q[i];
      v[2 * i].x = t.x;
      v[2 * i].y = t.y;
      v[2 * i + 1].x = t.z;
      v[2 * i + 1].y = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < RR; ++i) v[i] = p[i];
  }
}
template <int RR, typename C>
__device__ __forceinline__ void store_run(C* p, const C* v) {
  if constexpr (sizeof(C) == 8 && RR % 2 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < RR / 2; ++i) q[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
  } else {
#pragma unroll
    for (int i = 0; i < RR; ++i) p[i] = v[i];
  }
}

template <int RR> struct Log2R { static constexpr int v = RR == 8 ? 3 : (RR == 4 ? 2 : 1); };

// One radix-R stage (not the last) over columns 0 .. narr-1, forward (INV = false) or adjoint.
// Two butterflies per thread and iteration, both read before either is written.
template <int R, bool INV, int NT, typename C>
__device__ __forceinline__ void stage_inplace(C* s, int Pc, int narr, int logN, int logL, const C* tw) {
  constexpr int LR = Log2R<R>::v;
  const int lnb = logN - LR, total = narr << lnb;
  const int bmask = (1 << lnb) - 1, lmask = (1 << logL) - 1;
  for (int b0 = threadIdx.x; b0 < total; b0 += 2 * NT) {
    C v[2][R];
    int ad[2][R], n1s[2];
    bool ok[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int bi = b0 + u * NT;
      ok[u] = bi < total;
      const int bb = ok[u] ? bi : b0;
      const int a = bb >> lnb, rem = bb & bmask, n1 = rem & lmask;
      const int p0 = ((rem >> logL) << (logL + LR)) + n1;
      n1s[u] = n1;
#pragma unroll
      for (int r = 0; r < R; ++r) ad[u][r] = a * Pc + pad16(p0 + (r << logL));
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (ok[u]) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[u][r] = s[ad[u][r]];
      }
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (ok[u]) {
        C w[R];
#pragma unroll
        for (int r = 1; r < R; ++r) w[r] = tw[((r - 1) << logL) + n1s[u]];
        if (INV) {
#pragma unroll
          for (int r = 1; r < R; ++r) v[u][r] = cmulconj(v[u][r], w[r]);
          dft_small<R, true>(v[u]);
        } else {
          dft_small<R, false>(v[u]);
#pragma unroll
          for (int r = 1; r < R; ++r) v[u][r] = cmul(v[u][r], w[r]);
        }
      }
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (ok[u]) {
#pragma unroll
        for (int r = 0; r < R; ++r) s[ad[u][r]] = v[u][r];
      }
  }
  __syncthreads();
}

// The adjoint of stage 0 (one block, stride N / R) for the three field columns, writing the natural
// order result z = n1 + L n2 to global memory (or its bf16 split pieces).  The column index is a
// compile-time loop index, so the column descriptors stay in registers.
template <int R, int NT, bool SPLIT_OUT, typename C, int NCOL = 3>
__device__ __forceinline__ void stage0_inv_to_global(const C* s, int Pc, int logN, const C* tw, C* const* dst,
                                                     const SplitColumn* sc) {
  constexpr int LR = Log2R<R>::v;
  const int logL = logN - LR, L = 1 << logL;
#pragma unroll
  for (int a = 0; a < NCOL; ++a) {
    // the bf16 split stores are kept rolled: unrolled, they push the kernel out of the instruction cache
#pragma unroll 1
    for (int n1 = threadIdx.x; n1 < L; n1 += NT) {
      C v[R], w[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = s[a * Pc + pad16(n1 + (r << logL))];
#pragma unroll
      for (int r = 1; r < R; ++r) w[r] = tw[((r - 1) << logL) + n1];
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmulconj(v[r], w[r]);
      dft_small<R, true>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int z = n1 + (r << logL);
        if (!SPLIT_OUT)
          dst[a][z] = v[r];
        else
          split_store(sc[a], z, (float)v[r].x, (float)v[r].y);
      }
    }
  }
}

// A single-stage transform leaves the result in shared memory: copy it out in natural order.
template <int NT, bool SPLIT_OUT, typename C>
__device__ __forceinline__ void copy_out(const C* s, int Pc, int N, C* const* dst, const SplitColumn* sc) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    for (int z = threadIdx.x; z < N; z += NT) {
      const C v = s[a * Pc + pad16(z)];
      if (!SPLIT_OUT)
        dst[a][z] = v;
      else
        split_store(sc[a], z, (float)v.x, (float)v.y);
    }
}

// Exact midpoint update of one (kz, j) point: Horner form of
//   x + A1 M x + A2 M^2 x - dt (xJ + B1 M xJ + B2 M^2 xJ):
//   p = x - dt xJ,  q = A1 x - dt B1 xJ,  u = A2 x - dt B2 xJ,  r = p + M (q + M u),
// x_J = (eJ, aJ, 0) for TM, (cJ, 0, 0) for TE; the result is scaled by `inv` (1/Nz of the inverse DFT).
template <typename T, typename K, typename C>
__device__ __forceinline__ void rotate_point(C& x0, C& x1, C& x2, C j0, C j1, bool hasJ, int fam, K lam, K spr,
                                             K spi, K smr, K smi, K A1, K A2, T B1, T B2, T dt, T inv) {
  C y0, y1, y2, z0, z1, z2;
  const T dB1 = dt * B1, dB2 = dt * B2;
  C u0 = cscale(A2, x0), u1 = cscale(A2, x1), u2 = cscale(A2, x2);
  C q0 = cscale(A1, x0), q1 = cscale(A1, x1), q2 = cscale(A1, x2);
  C p0 = x0, p1 = x1;
  if (hasJ) {
    u0.x -= dB2 * j0.x; u0.y -= dB2 * j0.y;
    u1.x -= dB2 * j1.x; u1.y -= dB2 * j1.y;
    q0.x -= dB1 * j0.x; q0.y -= dB1 * j0.y;
    q1.x -= dB1 * j1.x; q1.y -= dB1 * j1.y;
    p0.x -= dt * j0.x; p0.y -= dt * j0.y;
    p1.x -= dt * j1.x; p1.y -= dt * j1.y;
  }
  if (fam == 0) {
    apply_tm(u0, u1, u2, y0, y1, y2, lam, spr, spi, smr, smi);
    y0 = cadd(y0, q0); y1 = cadd(y1, q1); y2 = cadd(y2, q2);
    apply_tm(y0, y1, y2, z0, z1, z2, lam, spr, spi, smr, smi);
  } else {
    apply_te(u0, u1, u2, y0, y1, y2, lam, spr, spi, smr, smi);
    y0 = cadd(y0, q0); y1 = cadd(y1, q1); y2 = cadd(y2, q2);
    apply_te(y0, y1, y2, z0, z1, z2, lam, spr, spi, smr, smi);
  }
  C r0 = cadd(p0, z0), r1 = cadd(p1, z1), r2 = cadd(x2, z2);
  r0.x *= inv; r0.y *= inv;
  r1.x *= inv; r1.y *= inv;
  r2.x *= inv; r2.y *= inv;
  x0 = r0;
  x1 = r1;
  x2 = r2;
}

// The last forward stage (radix RL, stride 1: butterfly b holds positions b RL .. b RL + RL - 1), the
// exact rotation of those RL kz values and the first inverse stage (the adjoint of the same butterfly),
// in registers per butterfly.  The current columns' last stage is done here too: their values at
// these positions are needed only by this butterfly.  MAIN adds the precomputed source term instead.
template <int RL, int MODE, int NT, typename T, typename K, typename PH, typename ZS, typename C>
__device__ __forceinline__ void fused_last_stage(C* s, int Pc, int N, bool hasJ, int fam, const PH* phase,
                                                 const ZS* zs, K lam, T dt, T inv, const C* src, size_t sstride) {
  const int nb = N / RL;
  for (int b = threadIdx.x; b < nb; b += NT) {
    const int p0 = b * RL, pa = pad16(p0);
    // up to radix 4 (FP32) the butterfly's table records are loaded first, to overlap their latency
    // with the transforms; radix 8 or FP64 would not leave the registers for it
    constexpr bool PRE = RL <= 4 && sizeof(T) == 4;
    PH ph[PRE ? RL : 1];
    ZS zr[PRE ? RL : 1];
    if constexpr (PRE) {
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        ph[r] = phase[r * nb + b];
        zr[r] = zs[r * nb + b];
      }
    }
    C v[3][RL], jv[2][RL];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      load_run<RL>(s + a * Pc + pa, v[a]);
      dft_small<RL, false>(v[a]);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int r = 0; r < RL; ++r) jv[c][r] = cmake<C>(0, 0);
    if (hasJ) {
      load_run<RL>(s + 3 * Pc + pa, jv[0]);
      dft_small<RL, false>(jv[0]);
      if (fam == 0) {
        load_run<RL>(s + 4 * Pc + pa, jv[1]);
        dft_small<RL, false>(jv[1]);
      }
    }
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      K spr, spi, smr, smi, A1, A2;
      T B1, B2;
      if constexpr (PRE) {
        zsym_unpack(zr[r], spr, spi, smr, smi);
        phase_unpack(ph[r], A1, A2, B1, B2);
      } else {
        zsym_unpack(zs[r * nb + b], spr, spi, smr, smi);
        phase_unpack(phase[r * nb + b], A1, A2, B1, B2);
      }
      rotate_point<T, K, C>(v[0][r], v[1][r], v[2][r], jv[0][r], jv[1][r], hasJ, fam, lam, spr, spi, smr, smi, A1,
                            A2, B1, B2, dt, inv);
      if (MODE == MAIN && src) {
        const int q = r * nb + b;
        v[0][r] = cadd(v[0][r], src[q]);
        v[1][r] = cadd(v[1][r], src[sstride + q]);
        v[2][r] = cadd(v[2][r], src[2 * sstride + q]);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dft_small<RL, true>(v[a]);
      store_run<RL>(s + a * Pc + pa, v[a]);
    }
  }
  __syncthreads();
}

// SOURCE: the current columns' last forward stage and the midpoint source term
// -dt exp(dt M / 2) x_J / Nz per position, written to global memory in position order.
template <int RL, int NT, typename T, typename K, typename PH, typename ZS, typename C>
__device__ __forceinline__ void source_last_stage(const C* s, int Pc, int N, int fam, const PH* phase, const ZS* zs,
                                                  K lam, T dt, T inv, C* src, size_t sstride) {
  const int nb = N / RL;
  for (int b = threadIdx.x; b < nb; b += NT) {
    const int p0 = b * RL, pa = pad16(p0);
    C j0v[RL], j1v[RL];
    load_run<RL>(s + pa, j0v);
    dft_small<RL, false>(j0v);
#pragma unroll
    for (int r = 0; r < RL; ++r) j1v[r] = cmake<C>(0, 0);
    if (fam == 0) {
      load_run<RL>(s + Pc + pa, j1v);
      dft_small<RL, false>(j1v);
    }
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int q = r * nb + b;
      K spr, spi, smr, smi, A1, A2;
      T B1, B2;
      zsym_unpack(zs[q], spr, spi, smr, smi);
      phase_unpack(phase[q], A1, A2, B1, B2);
      C y0, y1, y2, z0, z1, z2;
      const C j0 = j0v[r], j1 = j1v[r], j2 = cmake<C>(0, 0);
      if (fam == 0) {
        apply_tm(j0, j1, j2, y0, y1, y2, lam, spr, spi, smr, smi);
        apply_tm(y0, y1, y2, z0, z1, z2, lam, spr, spi, smr, smi);
      } else {
        apply_te(j0, j1, j2, y0, y1, y2, lam, spr, spi, smr, smi);
        apply_te(y0, y1, y2, z0, z1, z2, lam, spr, spi, smr, smi);
      }
      const T f = -dt * inv;
      const C jj[3] = {j0, j1, j2}, yy[3] = {y0, y1, y2}, zz[3] = {z0, z1, z2};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C w = cadd(jj[c], cadd(cscale(B1, yy[c]), cscale(B2, zz[c])));
        w.x *= f;
        w.y *= f;
        src[c * sstride + q] = w;
      }
    }
  }
}

}  // namespace

// coefficient array of column a of family fam: E group (e, a, c) = 0, 1, 2; B group (b, d, f) = 3, 4, 5;
// J (eJ, aJ, cJ) = 6, 7, 8.  TM columns: e, a, b, eJ, aJ; TE: c, d, f, cJ.  SOURCE: the J columns alone.
__device__ __forceinline__ int column_index(int mode, int fam, int a) {
  if (mode == SOURCE) return fam == 0 ? 6 + a : 8;
  if (fam == 0) return a < 2 ? a : (a == 2 ? 3 : a + 3);
  return a == 0 ? 2 : (a < 3 ? a + 3 : 8);
}

// T: data real type; K: coefficient type (double or df); PH / ZS: table records; R: radix of all
// stages but the last; NT: threads; TW_SMEM: twiddle tables copied to shared memory (else read
// through L1).
template <typename T, typename K, typename PH, typename ZS, int R, int NT, bool SPLIT_OUT, int MODE, bool TW_SMEM>
__global__ void __launch_bounds__(NT, (NT <= 256 ? 2 : 1)) spectral_kernel(SpectralArgs args) {
  typedef typename cplx<T>::type C;
  constexpr int LR = Log2R<R>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int Nz = args.Nz, L = args.logNz, n = args.n;
  const int j = blockIdx.x, fam = blockIdx.y, md = blockIdx.z;
  const bool hasJ = MODE == FUSED ? args.hasJ : false;
  const int narr = MODE == SOURCE ? (fam == 0 ? 2 : 1) : (hasJ ? (fam == 0 ? 5 : 4) : 3);
  const C* coef = reinterpret_cast<const C*>(args.coef);
  const C* twg = reinterpret_cast<const C*>(args.twiddle);
  const int Pc = pad16(Nz);
  const int slots = spectral_slots(MODE, args.hasJ);
  const C* tw = TW_SMEM ? s + (size_t)slots * Pc : twg;
  const PH* phase = reinterpret_cast<const PH*>(args.phase) + ((size_t)(md * 2 + fam) * n + j) * Nz;
  if (threadIdx.x == 0) {
    // the rotation reads this column's phase records (and, in MAIN mode, the source term) from global
    // memory: start pulling them into L2 now, while the columns arrive and the forward stages run
    l2_prefetch(phase, (uint32_t)(Nz * sizeof(PH)));
    if (MODE == MAIN && args.src)
      for (int c = 0; c < 3; ++c)
        l2_prefetch(reinterpret_cast<const C*>(args.src) + (((size_t)(md * 2 + fam) * 3 + c) * n + j) * Nz,
                    (uint32_t)(Nz * sizeof(C)));
  }
  // the family's columns (contiguous Nz values each) into the padded layout, 16 bytes per copy
  {
    constexpr int EPC = 16 / (int)sizeof(C);
    const int lper = L - (EPC == 2 ? 1 : 0), per = 1 << lper;
    for (int i = threadIdx.x; i < narr * per; i += NT) {
      const int a = i >> lper, e = (i & (per - 1)) * EPC;
      const C* col = coef + ((size_t)(md * 9 + column_index(MODE, fam, a)) * n + j) * Nz;
      cp_async16(s + a * Pc + pad16(e), col + e);
    }
    if (TW_SMEM) {
      C* tws = s + (size_t)slots * Pc;
      for (int i = threadIdx.x; i < args.tw_count / EPC; i += NT) cp_async16(tws + i * EPC, twg + i * EPC);
    }
    cp_async_wait_all();
    __syncthreads();
  }
  const ZS* zs = reinterpret_cast<const ZS*>(args.zsym);
  const K lam = reinterpret_cast<const K*>(args.lam)[(md * 2 + fam) * n + j];
  const T dt = (T)args.dt;
  const T inv = (T)1 / (T)Nz;
  C* src = reinterpret_cast<C*>(args.src) + ((size_t)(md * 2 + fam) * 3 * n + j) * Nz;  // [md][fam][3][n][Nz]
  const size_t sstride = (size_t)n * Nz;
  // stages: the leftover factor first (radix RF = 2^(L mod LR), RF = R when that is 1), then radix R;
  // a transform shorter than R is one stage of radix Nz
  const int nfull = L / LR, rem = L % LR;
  const int S = rem && nfull ? nfull + 1 : (nfull ? nfull : 1);
  const int LRF = S == 1 ? L : (rem ? rem : LR);  // log2 of the first stage's radix
  // forward stages but the last
  const C* t = tw;
  for (int st = 0; st < S - 1; ++st) {
    const int logLs = L - LRF - LR * st;
    if (st > 0 || LRF == LR) {
      stage_inplace<R, false, NT>(s, Pc, narr, L, logLs, t);
      t += (size_t)(R - 1) << logLs;
    } else if (LRF == 1) {
      stage_inplace<2, false, NT>(s, Pc, narr, L, logLs, t);
      t += (size_t)1 << logLs;
    } else {
      stage_inplace<4, false, NT>(s, Pc, narr, L, logLs, t);
      t += (size_t)3 << logLs;
    }
  }
  // the last stage: radix R, or the single stage of a short transform
  const int LRL = S == 1 ? L : LR;
  if (MODE == SOURCE) {
    if (LRL == 1)
      source_last_stage<2, NT, T>(s, Pc, Nz, fam, phase, zs, lam, dt, inv, src, sstride);
    else if (LRL == 2)
      source_last_stage<4, NT, T>(s, Pc, Nz, fam, phase, zs, lam, dt, inv, src, sstride);
    else
      source_last_stage<R, NT, T>(s, Pc, Nz, fam, phase, zs, lam, dt, inv, src, sstride);
    return;
  }
  if (LRL == 1)
    fused_last_stage<2, MODE, NT, T>(s, Pc, Nz, hasJ, fam, phase, zs, lam, dt, inv, src, sstride);
  else if (LRL == 2)
    fused_last_stage<4, MODE, NT, T>(s, Pc, Nz, hasJ, fam, phase, zs, lam, dt, inv, src, sstride);
  else
    fused_last_stage<R, MODE, NT, T>(s, Pc, Nz, hasJ, fam, phase, zs, lam, dt, inv, src, sstride);
  // remaining inverse stages (adjoints in reverse order), the one of stage 0 writing to global memory
  for (int st = S - 2; st >= 1; --st) {
    const int logLs = L - LRF - LR * st;
    t -= (size_t)(R - 1) << logLs;
    stage_inplace<R, true, NT>(s, Pc, 3, L, logLs, t);
  }
  C* out = reinterpret_cast<C*>(args.coef);
  C* dst[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) dst[a] = out + ((size_t)(md * 9 + column_index(MODE, fam, a)) * n + j) * Nz;
  SplitColumn sc[3];
  if (SPLIT_OUT) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      sc[a] = split_column(args.split_out, args.npieces, md, column_index(MODE, fam, a), j, args.split_kstages, Nz);
  }
  if (S == 1)
    copy_out<NT, SPLIT_OUT>(s, Pc, Nz, dst, sc);
  else if (LRF == LR)
    stage0_inv_to_global<R, NT, SPLIT_OUT>(s, Pc, L, tw, dst, sc);
  else if (LRF == 1)
    stage0_inv_to_global<2, NT, SPLIT_OUT>(s, Pc, L, tw, dst, sc);
  else
    stage0_inv_to_global<4, NT, SPLIT_OUT>(s, Pc, L, tw, dst, sc);
}

// ---------------------------------------------------------------- column-split form
// For z lengths whose three field columns do not fit in shared memory (FP64 at Nz = 8192): the same
// transform and update in three kernels over one column at a time.  (1) every coefficient column (fields
// and current) is transformed forward in place, the last stage included, and left in global memory in
// position order; (2) the update of every (kz, j) point reads the family's columns at that position;
// (3) every field column is transformed back (the adjoints in reverse order) to natural order, or to the
// back-projection's split pieces.  Same butterflies, tables and update arithmetic as the fused kernel, so
// the results are bitwise those of the fused form.

// stage schedule of a length-2^L transform with radix R: first-stage radix 2^LRF, S stages, last radix 2^LRL
struct StageSchedule {
  int S, LRF, LRL;
  __device__ StageSchedule(int L, int LR) {
    const int nfull = L / LR, rem = L % LR;
    S = rem && nfull ? nfull + 1 : (nfull ? nfull : 1);
    LRF = S == 1 ? L : (rem ? rem : LR);
    LRL = S == 1 ? L : LR;
  }
};

// the last stage (stride 1, no twiddles) of one column, forward or adjoint: runs of RL consecutive positions
template <int RL, bool INV, int NT, typename C>
__device__ __forceinline__ void stage_last_column(C* s, int N) {
  for (int b = threadIdx.x; b < N / RL; b += NT) {
    C v[RL];
    load_run<RL>(s + pad16(b * RL), v);
    dft_small<RL, INV>(v);
    store_run<RL>(s + pad16(b * RL), v);
  }
  __syncthreads();
}
template <int R, bool INV, int NT, typename C>
__device__ __forceinline__ void stage_last_any(C* s, int N, int LRL) {
  if (LRL == 1)
    stage_last_column<2, INV, NT>(s, N);
  else if (LRL == 2)
    stage_last_column<4, INV, NT>(s, N);
  else if (LRL == 3)
    stage_last_column<8, INV, NT>(s, N);
  else
    stage_last_column<R, INV, NT>(s, N);
}

template <typename C, int NT>
__device__ __forceinline__ void load_column(C* s, const C* col, int L) {
  constexpr int EPC = 16 / (int)sizeof(C);
  const int per = 1 << (L - (EPC == 2 ? 1 : 0));
  for (int i = threadIdx.x; i < per; i += NT) cp_async16(s + pad16(i * EPC), col + i * EPC);
  cp_async_wait_all();
  __syncthreads();
}

// (1) forward transform of coefficient column blockIdx.y (0 .. 8) of (mode blockIdx.z, j blockIdx.x), in place
template <typename T, int R, int NT>
__global__ void __launch_bounds__(NT, 1) spectral_fwd_column(SpectralArgs args) {
  typedef typename cplx<T>::type C;
  constexpr int LR = Log2R<R>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int Nz = args.Nz, L = args.logNz, n = args.n;
  C* col = reinterpret_cast<C*>(args.coef) + ((size_t)(blockIdx.z * 9 + blockIdx.y) * n + blockIdx.x) * Nz;
  const C* t = reinterpret_cast<const C*>(args.twiddle);
  load_column<C, NT>(s, col, L);
  const StageSchedule sc(L, LR);
  const int Pc = pad16(Nz);
  for (int st = 0; st < sc.S - 1; ++st) {
    const int logLs = L - sc.LRF - LR * st;
    if (st > 0 || sc.LRF == LR) {
      stage_inplace<R, false, NT>(s, Pc, 1, L, logLs, t);
      t += (size_t)(R - 1) << logLs;
    } else if (sc.LRF == 1) {
      stage_inplace<2, false, NT>(s, Pc, 1, L, logLs, t);
      t += (size_t)1 << logLs;
    } else {
      stage_inplace<4, false, NT>(s, Pc, 1, L, logLs, t);
      t += (size_t)3 << logLs;
    }
  }
  stage_last_any<R, false, NT>(s, Nz, sc.LRL);
  for (int z = threadIdx.x; z < Nz; z += NT) col[z] = s[pad16(z)];
}

// (2) the exact midpoint update of every (kz, j) point of (mode, family) = (blockIdx.z / 2, blockIdx.z % 2),
// j = blockIdx.y, positions blockIdx.x * blockDim.x + threadIdx.x, scaled by 1 / Nz
template <typename T, typename K, typename PH, typename ZS>
__global__ void spectral_update_columns(SpectralArgs args, int RL) {
  typedef typename cplx<T>::type C;
  const int Nz = args.Nz, n = args.n, j = blockIdx.y, md = blockIdx.z >> 1, fam = blockIdx.z & 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Nz) return;
  const int nb = Nz / RL, q = (p % RL) * nb + p / RL;  // table index of position p
  C* coef = reinterpret_cast<C*>(args.coef);
  auto at = [&](int c) { return coef + ((size_t)(md * 9 + c) * n + j) * Nz + p; };
  // TM: e, a, b (columns 0, 1, 3), current eJ, aJ (6, 7); TE: c, d, f (2, 4, 5), current cJ (8)
  C* x0 = at(fam == 0 ? 0 : 2);
  C* x1 = at(fam == 0 ? 1 : 4);
  C* x2 = at(fam == 0 ? 3 : 5);
  const bool hasJ = args.hasJ;
  const C zero = cmake<C>(0, 0);
  const C j0 = hasJ ? *at(fam == 0 ? 6 : 8) : zero;
  const C j1 = hasJ && fam == 0 ? *at(7) : zero;
  K spr, spi, smr, smi, A1, A2;
  T B1, B2;
  zsym_unpack(reinterpret_cast<const ZS*>(args.zsym)[q], spr, spi, smr, smi);
  phase_unpack(reinterpret_cast<const PH*>(args.phase)[((size_t)(md * 2 + fam) * n + j) * Nz + q], A1, A2, B1, B2);
  const K lam = reinterpret_cast<const K*>(args.lam)[(md * 2 + fam) * n + j];
  C v0 = *x0, v1 = *x1, v2 = *x2;
  rotate_point<T, K, C>(v0, v1, v2, j0, j1, hasJ, fam, lam, spr, spi, smr, smi, A1, A2, B1, B2, (T)args.dt,
                        (T)1 / (T)Nz);
  *x0 = v0;
  *x1 = v1;
  *x2 = v2;
}

// (3) inverse transform of field coefficient column blockIdx.y (0 .. 5) of (mode blockIdx.z, j blockIdx.x)
template <typename T, int R, int NT, bool SPLIT_OUT>
__global__ void __launch_bounds__(NT, 1) spectral_inv_column(SpectralArgs args) {
  typedef typename cplx<T>::type C;
  constexpr int LR = Log2R<R>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int Nz = args.Nz, L = args.logNz, n = args.n, c = blockIdx.y, md = blockIdx.z, j = blockIdx.x;
  C* col = reinterpret_cast<C*>(args.coef) + ((size_t)(md * 9 + c) * n + j) * Nz;
  const C* tw = reinterpret_cast<const C*>(args.twiddle);
  load_column<C, NT>(s, col, L);
  const StageSchedule sc(L, LR);
  const int Pc = pad16(Nz);
  stage_last_any<R, true, NT>(s, Nz, sc.LRL);
  // twiddles of stages 1 .. S-2 follow stage 0's
  const C* t = tw + ((size_t)((1 << sc.LRF) - 1) << (L - sc.LRF));
  for (int st = 1; st < sc.S - 1; ++st) t += (size_t)(R - 1) << (L - sc.LRF - LR * st);
  for (int st = sc.S - 2; st >= 1; --st) {
    const int logLs = L - sc.LRF - LR * st;
    t -= (size_t)(R - 1) << logLs;
    stage_inplace<R, true, NT>(s, Pc, 1, L, logLs, t);
  }
  SplitColumn spl[3];
  C* dst[3] = {col, col, col};
  if (SPLIT_OUT) spl[0] = split_column(args.split_out, args.npieces, md, c, j, args.split_kstages, Nz);
  if (sc.S == 1) {
    for (int z = threadIdx.x; z < Nz; z += NT) {
      const C v = s[pad16(z)];
      if (!SPLIT_OUT)
        col[z] = v;
      else
        split_store(spl[0], z, (float)v.x, (float)v.y);
    }
  } else if (sc.LRF == LR) {
    stage0_inv_to_global<R, NT, SPLIT_OUT, C, 1>(s, Pc, L, tw, dst, spl);
  } else if (sc.LRF == 1) {
    stage0_inv_to_global<2, NT, SPLIT_OUT, C, 1>(s, Pc, L, tw, dst, spl);
  } else {
    stage0_inv_to_global<4, NT, SPLIT_OUT, C, 1>(s, Pc, L, tw, dst, spl);
  }
}

template <typename T, typename K, typename PH, typename ZS, int R, int NT, bool SPLIT>
static cudaError_t launch_columns_nt(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  typedef typename cplx<T>::type C;
  const size_t smem = (size_t)pad16(a.Nz) * sizeof(C);
  auto kf = spectral_fwd_column<T, R, NT>;
  auto ki = spectral_inv_column<T, R, NT, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kf<<<dim3(a.n, a.hasJ ? 9 : 6, nmodes), NT, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int LR = Log2R<R>::v, L = a.logNz;
  const int RL = L <= LR ? a.Nz : R;  // radix of the last stage (the table order)
  spectral_update_columns<T, K, PH, ZS><<<dim3((a.Nz + 255) / 256, a.n, 2 * nmodes), 256, 0, st>>>(a, RL);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ki<<<dim3(a.n, 6, nmodes), NT, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, typename K, typename PH, typename ZS, int R, bool SPLIT>
static cudaError_t launch_columns(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  const int need = a.Nz / R;
  if (need <= 128) return launch_columns_nt<T, K, PH, ZS, R, 128, SPLIT>(a, nmodes, st);
  if (need <= 256) return launch_columns_nt<T, K, PH, ZS, R, 256, SPLIT>(a, nmodes, st);
  return launch_columns_nt<T, K, PH, ZS, R, 512, SPLIT>(a, nmodes, st);
}

template <typename T, typename K, typename PH, typename ZS, int R, int NT, bool SPLIT, int MODE, bool TW_SMEM>
static cudaError_t launch_one(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  typedef typename cplx<T>::type C;
  const size_t smem = ((size_t)spectral_slots(MODE, a.hasJ) * pad16(a.Nz) + (TW_SMEM ? (size_t)a.tw_count : 0)) *
                      sizeof(C);
  auto k = spectral_kernel<T, K, PH, ZS, R, NT, SPLIT, MODE, TW_SMEM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.n, 2, nmodes);
  k<<<grid, NT, smem, st>>>(a);
  return cudaGetLastError();
}

// Threads by transform length: Nz / R (one radix-R butterfly per thread per column and stage),
// at least 128 and at most 512.
template <typename T, typename K, typename PH, typename ZS, int R, bool SPLIT, int MODE, bool TW_SMEM>
static cudaError_t launch_sized(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  const int need = a.Nz / R;
  if (need <= 128) return launch_one<T, K, PH, ZS, R, 128, SPLIT, MODE, TW_SMEM>(a, nmodes, st);
  if (need <= 256) return launch_one<T, K, PH, ZS, R, 256, SPLIT, MODE, TW_SMEM>(a, nmodes, st);
  return launch_one<T, K, PH, ZS, R, 512, SPLIT, MODE, TW_SMEM>(a, nmodes, st);
}

static size_t fused_bytes(int Nz, int precision, bool hasJ, int tw_count) {
  return ((size_t)spectral_slots(FUSED, hasJ) * pad16(Nz) + (size_t)tw_count) * (precision == 0 ? 16 : 8);
}

template <typename T, typename K, typename PH, typename ZS, int R, bool SPLIT>
static cudaError_t launch_prec(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  if (fused_bytes(a.Nz, prec, a.hasJ, a.tw_count) <= 227 * 1024)
    return launch_sized<T, K, PH, ZS, R, SPLIT, FUSED, true>(a, nmodes, st);
  // two kernels: the current's source term first, then the field columns alone (twiddles via L1)
  if (a.hasJ) {
    if (!a.src) return cudaErrorInvalidValue;
    cudaError_t e = launch_sized<T, K, PH, ZS, R, SPLIT, SOURCE, false>(a, nmodes, st);
    if (e != cudaSuccess) return e;
    return launch_sized<T, K, PH, ZS, R, SPLIT, MAIN, false>(a, nmodes, st);
  }
  SpectralArgs b = a;
  b.src = nullptr;
  return launch_sized<T, K, PH, ZS, R, SPLIT, MAIN, false>(b, nmodes, st);
}

cudaError_t launch_spectral(const SpectralArgs& a, int nmodes, int precision, bool split_out, cudaStream_t st) {
  if (precision == 0) return launch_prec<double, double, PhaseD, ZSymD, 4, false>(a, nmodes, st);
  if (split_out) return launch_prec<float, df, PhaseF, ZSymF, 8, true>(a, nmodes, st);
  return launch_prec<float, df, PhaseF, ZSymF, 8, false>(a, nmodes, st);
}

cudaError_t launch_spectral_columns(const SpectralArgs& a, int nmodes, int precision, bool split_out,
                                    cudaStream_t st) {
  if (!spectral_columns_supported(a.Nz, precision)) return cudaErrorNotSupported;
  if (precision == 0) return launch_columns<double, double, PhaseD, ZSymD, 4, false>(a, nmodes, st);
  if (split_out) return launch_columns<float, df, PhaseF, ZSymF, 8, true>(a, nmodes, st);
  return launch_columns<float, df, PhaseF, ZSymF, 8, false>(a, nmodes, st);
}

bool spectral_columns_supported(int Nz, int precision) {
  return Nz >= 2 && (Nz & (Nz - 1)) == 0 && (size_t)pad16(Nz) * (precision == 0 ? 16 : 8) <= 227 * 1024;
}

bool spectral_needs_source(int Nz, int precision, int tw_count) {
  return fused_bytes(Nz, precision, true, tw_count) > 227 * 1024;
}

// Smallest shared-memory footprint a plan needs: the three field columns of the two-kernel path
// (padded layout, twiddles through L1).  The fused path is used whenever it fits.
size_t spectral_smem_bytes(int Nz, int precision, bool hasJ) {
  (void)hasJ;
  return (size_t)spectral_slots(MAIN, false) * pad16(Nz) * (precision == 0 ? 16 : 8);
}


// Stage radices of the transform, first to last.  Nz = 2^logN: the leftover factor 2^(logN mod log2 R) first
// (when it is not 1), then R (8 for FP32, 4 for FP64); a transform shorter than R is a single stage.  Other
// 7-smooth Nz: the odd factors first (7s, 5s, 3s), then the power-of-two part the same way, so the last stage
// keeps the largest power-of-two radix.  Empty when Nz has a prime factor above 7.
static std::vector<int> stage_radices(int Nz, int precision) {
  const int LR = precision == 0 ? 2 : 3;
  std::vector<int> r;
  int rest = Nz;
  for (int p : {7, 5, 3})
    while (rest % p == 0) {
      r.push_back(p);
      rest /= p;
    }
  int logN = 0;
  while ((1 << logN) < rest) ++logN;
  if ((1 << logN) != rest) return std::vector<int>();
  const int nfull = logN / LR, rem = logN % LR;
  if (!nfull) {
    if (rest > 1 || r.empty()) r.push_back(1 << logN);
    return r;
  }
  if (rem) r.push_back(1 << rem);
  for (int k = 0; k < nfull; ++k) r.push_back(1 << LR);
  return r;
}

int spectral_radices(int Nz, int precision, int* rad) {
  const std::vector<int> r = stage_radices(Nz, precision);
  if ((int)r.size() > MixedRadices::kMax) return 0;
  for (size_t k = 0; k < r.size(); ++k) rad[k] = r[k];
  return (int)r.size();
}

// Twiddle tables of the in-place stages in stage order: stage s < S-1 (radix R_s, stride L_s,
// length M_s = R_s L_s) holds exp(-2 pi i n1 k2 / M_s) at (k2 - 1) L_s + n1 for n1 < L_s, 1 <= k2 < R_s.
int spectral_twiddles(int Nz, int precision, double* re, double* im) {
  const std::vector<int> rad = stage_radices(Nz, precision);
  const double pi = 3.14159265358979323846;
  int M = Nz, cnt = 0;
  for (size_t s = 0; s + 1 < rad.size(); ++s) {
    const int R = rad[s], L = M / R;
    for (int k2 = 1; k2 < R; ++k2)
      for (int n1 = 0; n1 < L; ++n1) {
        // reduce the angle exactly: n1 k2 / M of a full turn
        const long long num = ((long long)n1 * k2) % (long long)M;
        const double ang = -2.0 * pi * (double)num / (double)M;
        if (re) {
          re[cnt] = cos(ang);
          im[cnt] = sin(ang);
        }
        ++cnt;
      }
    M = L;
  }
  return cnt;
}

// kz index of the record at table index i: position p = b RL + r for i = r (Nz / RL) + b (RL the last
// stage's radix); the forward transform leaves at p = sum_s k2_s L_s (digit k2_s of stage s) the
// value of kz = sum_s k2_s R_0 ... R_{s-1}.
void spectral_positions(int Nz, int precision, int* kz) {
  const std::vector<int> rad = stage_radices(Nz, precision);
  const int RL = rad.back(), nb = Nz / RL;
  for (int i = 0; i < Nz; ++i) {
    const int p = (i % nb) * RL + i / nb;
    int M = Nz, rest = p, k = 0, mult = 1;
    for (int R : rad) {
      const int L = M / R;
      k += (rest / L) * mult;
      rest %= L;
      mult *= R;
      M = L;
    }
    kz[i] = k;
  }
}

}  // namespace fdetd
