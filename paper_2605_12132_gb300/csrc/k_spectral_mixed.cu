// Spectral kernel for z lengths that are not powers of two: Nz = 2^a 3^b 5^c 7^d (a multiple of 64).
//
// Computes what the power-of-two kernels compute for one (mode, family, j): forward z-DFT of the family's
// coefficient columns, the exact midpoint update of every (kz, j) (Eq. maxwellAM_solution2 with the family's
// 3x3 exponential), inverse z-DFT.  The transform is the same in-place decimation-in-frequency FFT with a
// runtime list of stage radices (3, 5, 7 first, then the power-of-two part: a leftover 2 or 4, then 8s, so
// the last stage has radix 8): stage s of radix R_s and stride L_s = N / (R_0 ... R_s) takes the DFT of the
// R_s elements blk M_s + n1 + L_s n2 (M_s = R_s L_s) and multiplies output k2 by W_{M_s}^{n1 k2}, in place;
// the forward output at position p holds kz = the mixed-radix digit reversal of p, and the per-kz tables
// are stored in that order (spectral_positions).  Twiddle tables, record layout and the update are those of
// the power-of-two kernel (k_spectral.cu); the small DFTs of odd radix use the symmetric form
//   X[m], X[R-m] = v0 + sum_k cos(2 pi m k / R) (v_k + v_{R-k})  -+ i sum_k sin(2 pi m k / R) (v_k - v_{R-k})
// (upper signs forward).  One kernel, columns in shared memory (the family's field and current columns and
// the twiddles must fit: FP32 up to Nz = 4096, FP64 up to about 2500).
#include "common.cuh"
#include "fft_small.cuh"
#include "kernels.h"

namespace fdetd {

namespace {

// cos and sin of 2 pi j / R for the odd radices (j = 0 .. R-1)
template <int R>
__device__ __forceinline__ double root_cos(int j) {
  if (R == 3) return j == 0 ? 1.0 : -0.5;
  if (R == 5) {
    const double c[5] = {1.0, 0.30901699437494742410, -0.80901699437494742410, -0.80901699437494742410,
                         0.30901699437494742410};
    return c[j];
  }
  const double c[7] = {1.0, 0.62348980185873353053, -0.22252093395631440429, -0.90096886790241912624,
                       -0.90096886790241912624, -0.22252093395631440429, 0.62348980185873353053};
  return c[j];
}
template <int R>
__device__ __forceinline__ double root_sin(int j) {
  if (R == 3) return j == 0 ? 0.0 : (j == 1 ? 0.86602540378443864676 : -0.86602540378443864676);
  if (R == 5) {
    const double s[5] = {0.0, 0.95105651629515357212, 0.58778525229247312917, -0.58778525229247312917,
                         -0.95105651629515357212};
    return s[j];
  }
  const double s[7] = {0.0, 0.78183148246802980871, 0.97492791218182360702, 0.43388373911755812048,
                       -0.43388373911755812048, -0.97492791218182360702, -0.78183148246802980871};
  return s[j];
}

// DFT of R = 3, 5, 7 points in registers (W = exp(-+2 pi i / R)), natural order in and out
template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_odd(C* v) {
  typedef decltype(v[0].x) T;
  constexpr int H = (R - 1) / 2;
  C t[H], u[H];
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    t[k - 1] = cadd(v[k], v[R - k]);
    u[k - 1] = csub(v[k], v[R - k]);
  }
  const C v0 = v[0];
  C x0 = v0;
#pragma unroll
  for (int k = 0; k < H; ++k) x0 = cadd(x0, t[k]);
#pragma unroll
  for (int m = 1; m <= H; ++m) {
    C a = v0, b = cmake<C>(0, 0);
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      const T c = (T)root_cos<R>((m * k) % R), s = (T)root_sin<R>((m * k) % R);
      a.x += c * t[k - 1].x;
      a.y += c * t[k - 1].y;
      b.x += s * u[k - 1].x;
      b.y += s * u[k - 1].y;
    }
    // forward: X[m] = a - i b, X[R-m] = a + i b; inverse: the conjugate pair
    const C mib = rot90<false>(b);  // -i b
    v[m] = INV ? csub(a, mib) : cadd(a, mib);
    v[R - m] = INV ? cadd(a, mib) : csub(a, mib);
  }
  v[0] = x0;
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_any(C* v) {
  if constexpr (R == 2 || R == 4 || R == 8)
    dft_small<R, INV>(v);
  else
    dft_odd<R, INV>(v);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory"); }

// one in-place stage (forward or adjoint) of radix R and stride L over ncol columns of length N
template <int R, bool INV, int NT, typename C>
__device__ __forceinline__ void mstage(C* s, int Pc, int ncol, int N, int L, const C* tw) {
  const int nb = N / R, total = ncol * nb;
  for (int i = threadIdx.x; i < total; i += NT) {
    const int a = i / nb, beta = i - a * nb;
    const int blk = beta / L, n1 = beta - blk * L;
    const int p0 = blk * R * L + n1;
    C v[R];
    int ad[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ad[r] = a * Pc + pad16(p0 + r * L);
      v[r] = s[ad[r]];
    }
    if (INV) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmulconj(v[r], tw[(r - 1) * L + n1]);
      dft_any<R, true>(v);
    } else {
      dft_any<R, false>(v);
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[(r - 1) * L + n1]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) s[ad[r]] = v[r];
  }
  __syncthreads();
}

template <bool INV, int NT, typename C>
__device__ __forceinline__ void mstage_any(int R, C* s, int Pc, int ncol, int N, int L, const C* tw) {
  switch (R) {
    case 2: mstage<2, INV, NT>(s, Pc, ncol, N, L, tw); break;
    case 3: mstage<3, INV, NT>(s, Pc, ncol, N, L, tw); break;
    case 4: mstage<4, INV, NT>(s, Pc, ncol, N, L, tw); break;
    case 5: mstage<5, INV, NT>(s, Pc, ncol, N, L, tw); break;
    case 7: mstage<7, INV, NT>(s, Pc, ncol, N, L, tw); break;
    default: mstage<8, INV, NT>(s, Pc, ncol, N, L, tw); break;
  }
}

// multiply a value by a table coefficient (double or double-float) and the update of one (kz, j) point
template <typename K, typename T>
__device__ __forceinline__ T kmul(K c, T x) { return rmul(c, x); }

// The exact midpoint update of one (kz, j) point (Horner form of x + A1 M x + A2 M^2 x - dt (x_J + B1 M x_J +
// B2 M^2 x_J)), scaled by inv = 1 / Nz; M = M_TM on (e, a, b) or M_TE on (c, d, f).
template <typename T, typename K, typename C>
__device__ __forceinline__ void update_point(C& x0, C& x1, C& x2, C j0, C j1, bool hasJ, int fam, K lam, K spr,
                                             K spi, K smr, K smi, K A1, K A2, T B1, T B2, T dt, T inv) {
  auto cs = [](K c, C x) { C r; r.x = kmul(c, x.x); r.y = kmul(c, x.y); return r; };
  auto cc = [](K re, K im, C x) {
    C r;
    r.x = kmul(re, x.x) - kmul(im, x.y);
    r.y = kmul(re, x.y) + kmul(im, x.x);
    return r;
  };
  auto apply = [&](C v0, C v1, C v2, C& y0, C& y1, C& y2) {
    if (fam == 0) {  // M_TM = [[0, 0, -lam], [0, 0, -s+], [1, -s-, 0]]
      y0 = cs(lam, v2); y0.x = -y0.x; y0.y = -y0.y;
      y1 = cc(spr, spi, v2); y1.x = -y1.x; y1.y = -y1.y;
      y2 = csub(v0, cc(smr, smi, v1));
    } else {         // M_TE = [[0, -s+, 1], [-s-, 0, 0], [-mu, 0, 0]]
      y0 = csub(v2, cc(spr, spi, v1));
      y1 = cc(smr, smi, v0); y1.x = -y1.x; y1.y = -y1.y;
      y2 = cs(lam, v0); y2.x = -y2.x; y2.y = -y2.y;
    }
  };
  const T dB1 = dt * B1, dB2 = dt * B2;
  C u0 = cs(A2, x0), u1 = cs(A2, x1), u2 = cs(A2, x2);
  C q0 = cs(A1, x0), q1 = cs(A1, x1), q2 = cs(A1, x2);
  C p0 = x0, p1 = x1;
  if (hasJ) {
    u0.x -= dB2 * j0.x; u0.y -= dB2 * j0.y;
    u1.x -= dB2 * j1.x; u1.y -= dB2 * j1.y;
    q0.x -= dB1 * j0.x; q0.y -= dB1 * j0.y;
    q1.x -= dB1 * j1.x; q1.y -= dB1 * j1.y;
    p0.x -= dt * j0.x; p0.y -= dt * j0.y;
    p1.x -= dt * j1.x; p1.y -= dt * j1.y;
  }
  C y0, y1, y2, z0, z1, z2;
  apply(u0, u1, u2, y0, y1, y2);
  y0 = cadd(y0, q0); y1 = cadd(y1, q1); y2 = cadd(y2, q2);
  apply(y0, y1, y2, z0, z1, z2);
  C r0 = cadd(p0, z0), r1 = cadd(p1, z1), r2 = cadd(x2, z2);
  x0.x = r0.x * inv; x0.y = r0.y * inv;
  x1.x = r1.x * inv; x1.y = r1.y * inv;
  x2.x = r2.x * inv; x2.y = r2.y * inv;
}

__device__ __forceinline__ void unpack(const PhaseD& p, double& A1, double& A2, double& B1, double& B2) {
  A1 = p.A1; A2 = p.A2; B1 = p.B1; B2 = p.B2;
}
__device__ __forceinline__ void unpack(const PhaseF& p, df& A1, df& A2, float& B1, float& B2) {
  A1 = p.A1;
  A2 = p.A2;
  const float a2 = p.A2.h + p.A2.l;
  B1 = sqrtf(0.5f * fmaxf(a2, 0.f));
  const float c = B1 > 0.f ? __fdividef(p.A1.h + p.A1.l, 2.f * B1) : 1.f;
  B2 = B1 > 0.f ? __fdividef(B1 * B1, 1.f + c) : 0.f;
}
__device__ __forceinline__ void unpack(const ZSymD& z, double& spr, double& spi, double& smr, double& smi) {
  spr = z.spr; spi = z.spi; smr = -z.spr; smi = z.spi;
}
__device__ __forceinline__ void unpack(const ZSymF& z, df& spr, df& spi, df& smr, df& smi) {
  spr = z.spr; spi = z.spi; smr.h = -z.spr.h; smr.l = -z.spr.l; smi = z.spi;
}

// Kernel modes: FUSED transforms the family's field and current columns together; SOURCE transforms only
// the current columns and writes the midpoint source term -dt exp(dt M / 2) x_J / Nz per table index; MAIN
// transforms the field columns and adds that precomputed source (when five columns do not fit in shared
// memory).
enum { MFUSED = 0, MMAIN = 1, MSOURCE = 2 };

// the last forward stage (radix RL, stride 1), the update of those RL kz and the first inverse stage
template <int RL, int MODE, int NT, typename T, typename K, typename PH, typename ZS, typename C>
__device__ __forceinline__ void mfused(C* s, int Pc, int N, bool hasJ, int fam, const PH* phase, const ZS* zs, K lam,
                                       T dt, T inv, const C* src, size_t sstride) {
  const int nb = N / RL;
  for (int b = threadIdx.x; b < nb; b += NT) {
    const int p0 = b * RL;
    C v[3][RL], jv[2][RL];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int r = 0; r < RL; ++r) v[a][r] = s[a * Pc + pad16(p0 + r)];
      dft_any<RL, false>(v[a]);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int r = 0; r < RL; ++r) jv[c][r] = cmake<C>(0, 0);
    if (MODE == MFUSED && hasJ) {
      const int nj = fam == 0 ? 2 : 1;
      for (int c = 0; c < nj; ++c) {
#pragma unroll
        for (int r = 0; r < RL; ++r) jv[c][r] = s[(3 + c) * Pc + pad16(p0 + r)];
        dft_any<RL, false>(jv[c]);
      }
    }
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int q = r * nb + b;
      K spr, spi, smr, smi, A1, A2;
      T B1, B2;
      unpack(zs[q], spr, spi, smr, smi);
      unpack(phase[q], A1, A2, B1, B2);
      update_point<T, K, C>(v[0][r], v[1][r], v[2][r], jv[0][r], jv[1][r], MODE == MFUSED && hasJ, fam, lam, spr,
                            spi, smr, smi, A1, A2, B1, B2, dt, inv);
      if (MODE == MMAIN && src) {
        v[0][r] = cadd(v[0][r], src[q]);
        v[1][r] = cadd(v[1][r], src[sstride + q]);
        v[2][r] = cadd(v[2][r], src[2 * sstride + q]);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dft_any<RL, true>(v[a]);
#pragma unroll
      for (int r = 0; r < RL; ++r) s[a * Pc + pad16(p0 + r)] = v[a][r];
    }
  }
  __syncthreads();
}

// SOURCE: the current columns' last forward stage and the source term -dt (x_J + B1 M x_J + B2 M^2 x_J) / Nz
// per table index, to global memory
template <int RL, int NT, typename T, typename K, typename PH, typename ZS, typename C>
__device__ __forceinline__ void msource(const C* s, int Pc, int N, int fam, const PH* phase, const ZS* zs, K lam,
                                        T dt, T inv, C* src, size_t sstride) {
  const int nb = N / RL;
  for (int b = threadIdx.x; b < nb; b += NT) {
    const int p0 = b * RL;
    C j0[RL], j1[RL];
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      j0[r] = s[pad16(p0 + r)];
      j1[r] = fam == 0 ? s[Pc + pad16(p0 + r)] : cmake<C>(0, 0);
    }
    dft_any<RL, false>(j0);
    if (fam == 0) dft_any<RL, false>(j1);
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int q = r * nb + b;
      K spr, spi, smr, smi, A1, A2;
      T B1, B2;
      unpack(zs[q], spr, spi, smr, smi);
      unpack(phase[q], A1, A2, B1, B2);
      // the update of the zero state with the current: x' = -dt (x_J + B1 M x_J + B2 M^2 x_J), then / Nz
      C x0 = cmake<C>(0, 0), x1 = cmake<C>(0, 0), x2 = cmake<C>(0, 0);
      update_point<T, K, C>(x0, x1, x2, j0[r], j1[r], true, fam, lam, spr, spi, smr, smi, A1, A2, B1, B2, dt, inv);
      src[q] = x0;
      src[sstride + q] = x1;
      src[2 * sstride + q] = x2;
    }
  }
}

template <int MODE, int NT, typename T, typename K, typename PH, typename ZS, typename C>
__device__ __forceinline__ void mlast_any(int RL, C* s, int Pc, int N, bool hasJ, int fam, const PH* phase,
                                          const ZS* zs, K lam, T dt, T inv, C* src, size_t sstride) {
#define FDETD_MLAST(R)                                                                    \
  if (MODE == MSOURCE)                                                                    \
    msource<R, NT, T>(s, Pc, N, fam, phase, zs, lam, dt, inv, src, sstride);              \
  else                                                                                    \
    mfused<R, MODE, NT, T>(s, Pc, N, hasJ, fam, phase, zs, lam, dt, inv, src, sstride);
  switch (RL) {
    case 2: FDETD_MLAST(2) break;
    case 3: FDETD_MLAST(3) break;
    case 4: FDETD_MLAST(4) break;
    case 5: FDETD_MLAST(5) break;
    case 7: FDETD_MLAST(7) break;
    default: FDETD_MLAST(8) break;
  }
#undef FDETD_MLAST
}

// the adjoint of stage 0 for the three field columns, to global memory (or the bf16 split pieces)
template <int R, int NT, bool SPLIT, typename C>
__device__ __forceinline__ void mstage0_out(const C* s, int Pc, int N, const C* tw, C* const* dst,
                                            const SplitColumn* sc) {
  const int L = N / R;
#pragma unroll 1
  for (int a = 0; a < 3; ++a)
    for (int n1 = threadIdx.x; n1 < L; n1 += NT) {
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = s[a * Pc + pad16(n1 + r * L)];
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmulconj(v[r], tw[(r - 1) * L + n1]);
      dft_any<R, true>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int z = n1 + r * L;
        if (!SPLIT)
          dst[a][z] = v[r];
        else
          split_store(sc[a], z, (float)v[r].x, (float)v[r].y);
      }
    }
}

__host__ __device__ __forceinline__ constexpr int mixed_slots(int mode, bool hasJ) {
  return mode == MFUSED ? (hasJ ? 5 : 3) : (mode == MMAIN ? 3 : 2);
}
// shared-memory bytes of one launch: the mode's column slots, then the staged twiddles (whole 16-byte copies)
size_t mixed_bytes(int Nz, int precision, int mode, bool hasJ, int tw_staged) {
  const size_t elt = precision == 0 ? 16 : 8, epc = 16 / elt;
  return ((size_t)mixed_slots(mode, hasJ) * pad16(Nz) + ((size_t)tw_staged + epc - 1) / epc * epc) * elt;
}

__device__ __forceinline__ int column_of(int fam, int a) {
  if (fam == 0) return a < 2 ? a : (a == 2 ? 3 : a + 3);
  return a == 0 ? 2 : (a < 3 ? a + 3 : 8);
}

template <typename T, typename K, typename PH, typename ZS, int NT, bool SPLIT, int MODE, bool TW_SMEM>
__global__ void __launch_bounds__(NT) spectral_mixed_kernel(SpectralArgs args, MixedRadices mr) {
  typedef typename cplx<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int N = args.Nz, n = args.n, Pc = pad16(N);
  const int j = blockIdx.x, fam = blockIdx.y, md = blockIdx.z;
  const bool hasJ = MODE == MFUSED && args.hasJ != 0;
  const int ncol = MODE == MSOURCE ? (fam == 0 ? 2 : 1) : (hasJ ? (fam == 0 ? 5 : 4) : 3);
  const int slots = mixed_slots(MODE, hasJ);
  const C* coef = reinterpret_cast<const C*>(args.coef);
  const C* twg = reinterpret_cast<const C*>(args.twiddle);
  C* tws = s + (size_t)slots * Pc;
  const C* tw = TW_SMEM ? tws : twg;
  constexpr int EPC = 16 / (int)sizeof(C);
  for (int i = threadIdx.x; i < ncol * (N / EPC); i += NT) {
    const int a = i / (N / EPC), e = (i - a * (N / EPC)) * EPC;
    const int c = MODE == MSOURCE ? (fam == 0 ? 6 + a : 8) : column_of(fam, a);
    cp16(s + a * Pc + pad16(e), coef + ((size_t)(md * 9 + c) * n + j) * N + e);
  }
  if (TW_SMEM)
    for (int i = threadIdx.x; i < (args.tw_count + EPC - 1) / EPC; i += NT) cp16(tws + i * EPC, twg + i * EPC);
  cp_wait_all();
  __syncthreads();
  const PH* phase = reinterpret_cast<const PH*>(args.phase) + ((size_t)(md * 2 + fam) * n + j) * N;
  const ZS* zs = reinterpret_cast<const ZS*>(args.zsym);
  const K lam = reinterpret_cast<const K*>(args.lam)[(md * 2 + fam) * n + j];
  C* src = reinterpret_cast<C*>(args.src) + ((size_t)(md * 2 + fam) * 3 * n + j) * N;   // [md][fam][3][n][N]
  const size_t sstride = (size_t)n * N;
  // forward stages but the last
  int L = N, off = 0;
  for (int st = 0; st + 1 < mr.nst; ++st) {
    const int R = mr.rad[st];
    L /= R;
    mstage_any<false, NT>(R, s, Pc, ncol, N, L, tw + off);
    off += (R - 1) * L;
  }
  mlast_any<MODE, NT, T>(mr.rad[mr.nst - 1], s, Pc, N, hasJ, fam, phase, zs, lam, (T)args.dt, (T)1 / (T)N,
                         MODE == MMAIN && !args.src ? nullptr : src, sstride);
  if (MODE == MSOURCE) return;
  // inverse stages in reverse order, stage 0's to global memory
  for (int st = mr.nst - 2; st >= 1; --st) {
    const int R = mr.rad[st];
    off -= (R - 1) * L;
    mstage_any<true, NT>(R, s, Pc, 3, N, L, tw + off);
    L *= R;
  }
  C* out = reinterpret_cast<C*>(args.coef);
  C* dst[3];
  SplitColumn sc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dst[a] = out + ((size_t)(md * 9 + column_of(fam, a)) * n + j) * N;
    if (SPLIT) sc[a] = split_column(args.split_out, args.npieces, md, column_of(fam, a), j, args.split_kstages, N);
  }
  switch (mr.rad[0]) {
    case 2: mstage0_out<2, NT, SPLIT>(s, Pc, N, tw, dst, sc); break;
    case 3: mstage0_out<3, NT, SPLIT>(s, Pc, N, tw, dst, sc); break;
    case 4: mstage0_out<4, NT, SPLIT>(s, Pc, N, tw, dst, sc); break;
    case 5: mstage0_out<5, NT, SPLIT>(s, Pc, N, tw, dst, sc); break;
    case 7: mstage0_out<7, NT, SPLIT>(s, Pc, N, tw, dst, sc); break;
    default: mstage0_out<8, NT, SPLIT>(s, Pc, N, tw, dst, sc); break;
  }
}

template <typename T, typename K, typename PH, typename ZS, bool SPLIT, int MODE, bool TW_SMEM>
cudaError_t launch_mm(const SpectralArgs& a, const MixedRadices& mr, int nmodes, cudaStream_t st) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  const size_t smem = mixed_bytes(a.Nz, prec, MODE, MODE == MFUSED && a.hasJ, TW_SMEM ? a.tw_count : 0);
  auto k = spectral_mixed_kernel<T, K, PH, ZS, 256, SPLIT, MODE, TW_SMEM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<dim3(a.n, 2, nmodes), 256, smem, st>>>(a, mr);
  return cudaGetLastError();
}

// the fused kernel when the family's columns and the twiddles fit in shared memory; otherwise the current's
// source term first (SOURCE), then the field columns alone (MAIN), twiddles read through L1
template <typename T, typename K, typename PH, typename ZS, bool SPLIT>
cudaError_t launch_m(const SpectralArgs& a, const MixedRadices& mr, int nmodes, cudaStream_t st) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  if (mixed_bytes(a.Nz, prec, MFUSED, a.hasJ, a.tw_count) <= 227 * 1024)
    return launch_mm<T, K, PH, ZS, SPLIT, MFUSED, true>(a, mr, nmodes, st);
  if (a.hasJ) {
    if (!a.src) return cudaErrorInvalidValue;
    cudaError_t e = launch_mm<T, K, PH, ZS, SPLIT, MSOURCE, false>(a, mr, nmodes, st);
    if (e != cudaSuccess) return e;
    return launch_mm<T, K, PH, ZS, SPLIT, MMAIN, false>(a, mr, nmodes, st);
  }
  SpectralArgs b = a;
  b.src = nullptr;
  return launch_mm<T, K, PH, ZS, SPLIT, MMAIN, false>(b, mr, nmodes, st);
}

}  // namespace

// Smallest shared-memory footprint the mixed-radix transform needs at this length: the three field columns
// of the two-kernel path (twiddles through L1); the fused kernel is used whenever it fits.
size_t spectral_mixed_smem_bytes(int Nz, int precision, bool hasJ, int tw_count) {
  (void)hasJ;
  (void)tw_count;
  return mixed_bytes(Nz, precision, MMAIN, false, 0);
}

bool spectral_mixed_needs_source(int Nz, int precision, int tw_count) {
  return mixed_bytes(Nz, precision, MFUSED, true, tw_count) > 227 * 1024;
}

cudaError_t launch_spectral_mixed(const SpectralArgs& a, const MixedRadices& mr, int nmodes, int precision,
                                  bool split_out, cudaStream_t st) {
  if (mr.nst < 1 || mr.nst > MixedRadices::kMax) return cudaErrorInvalidValue;
  if (precision == 0) return launch_m<double, double, PhaseD, ZSymD, false>(a, mr, nmodes, st);
  if (split_out) return launch_m<float, df, PhaseF, ZSymF, true>(a, mr, nmodes, st);
  return launch_m<float, df, PhaseF, ZSymF, false>(a, mr, nmodes, st);
}

}  // namespace fdetd
