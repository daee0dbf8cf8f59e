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
// The z transform is a mixed-radix Stockham FFT in shared memory: each pass loads
// every butterfly of every array of the family into registers, twiddles and
// transforms it there (radix 8 for FP32, radix 4 for FP64, one radix-2/4 pass
// first when log2 Nz is not a multiple), and writes it back in place after one
// barrier.  The rotation runs between the forward and inverse transforms.
#include "common.cuh"
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

// bulk asynchronous copy of `bytes` (multiple of 16) from global to shared, completing on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"((uint64_t)src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (long it = 0; it < (1L << 26); ++it) {
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

template <typename C, typename Kc, typename Tb>
__device__ __forceinline__ C combine(C x, C y, C z, Kc A1, Kc A2, C xJ, C yJ, C zJ, Tb B1, Tb B2, Tb dt,
                                     bool hasJ) {
  C r = cadd(x, cadd(cscale(A1, y), cscale(A2, z)));
  if (hasJ) {
    C s = cadd(xJ, cadd(cscale(B1, yJ), cscale(B2, zJ)));
    r.x -= dt * s.x;
    r.y -= dt * s.y;
  }
  return r;
}

// multiply by -i (forward) / +i (inverse)
template <bool INV, typename C>
__device__ __forceinline__ C rot90(C a) {
  C r;
  if (INV) {
    r.x = -a.y;
    r.y = a.x;
  } else {
    r.x = a.y;
    r.y = -a.x;
  }
  return r;
}

// In-register DFT of RR points, natural order in and out (W = exp(-+2 pi i / RR)).
template <int RR, bool INV, typename C>
__device__ __forceinline__ void dft_small(C* v) {
  if (RR == 2) {
    const C t = v[1];
    v[1] = csub(v[0], t);
    v[0] = cadd(v[0], t);
  } else if (RR == 4) {
    const C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]), a2 = cadd(v[1], v[3]);
    const C a3 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
  } else {  // 8: two 4-point DFTs (even / odd samples) and one radix-2 stage
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<4, INV>(e);
    dft_small<4, INV>(o);
    typedef decltype(e[0].x) R;
    const R h = (R)0.70710678118654752440;
    C w1, w3;  // W8^1, W8^3 (forward), conjugates for the inverse
    w1.x = h;
    w1.y = INV ? h : -h;
    w3.x = -h;
    w3.y = INV ? h : -h;
    const C t0 = o[0], t1 = cmul(w1, o[1]), t2 = rot90<INV>(o[2]), t3 = cmul(w3, o[3]);
    v[0] = cadd(e[0], t0);
    v[4] = csub(e[0], t0);
    v[1] = cadd(e[1], t1);
    v[5] = csub(e[1], t1);
    v[2] = cadd(e[2], t2);
    v[6] = csub(e[2], t2);
    v[3] = cadd(e[3], t3);
    v[7] = csub(e[3], t3);
  }
}

// Shared-memory layout of one array: logical element i at physical i + i/8 (one pad slot per
// 8 elements), which keeps every Stockham pass at most 2-way bank-conflicted.
__device__ __forceinline__ int padx(int i) { return i + (i >> 3); }


// One in-place Stockham pass of radix RR over arrays a0 .. a0+na-1 of length N = 2^logN (sub-sequence
// length Ns before the pass).  Every butterfly of the group is read into registers before the
// barrier and written after it, so source and destination layouts may differ: SRC_PAD = false reads
// the unpadded arrays left by the bulk copy (array a at a*N), otherwise arrays sit at a*(N + N/8)
// in the padded layout.  tw points at this pass's twiddle table: entry k*(RR-1) + r-1 holds
// exp(-2 pi i r k / (Ns RR)) for k < Ns.  MAXB bounds the butterflies per thread.
template <int RR, bool INV, int NT, int MAXB, bool SRC_PAD, typename C>
__device__ __forceinline__ void stockham_pass(C* s, int a0, int na, int logN, int Ns, const C* tw) {
  constexpr int LR = RR == 2 ? 1 : (RR == 4 ? 2 : 3);
  const int N = 1 << logN;
  const int lnbf = logN - LR, nbf = 1 << lnbf;
  const int total = na << lnbf;
  const int P = N + (N >> 3);
  C v[MAXB][RR];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * NT;
    if (b < total) {
      const int a = a0 + (b >> lnbf), j = b & (nbf - 1);
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const int li = j + (r << lnbf);
        v[i][r] = SRC_PAD ? s[a * P + padx(li)] : s[a * N + li];
      }
      if (Ns > 1) {
        const C* t = tw + (j & (Ns - 1)) * (RR - 1);
#pragma unroll
        for (int r = 1; r < RR; ++r) v[i][r] = INV ? cmulconj(v[i][r], t[r - 1]) : cmul(v[i][r], t[r - 1]);
      }
      dft_small<RR, INV>(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * NT;
    if (b < total) {
      const int a = a0 + (b >> lnbf), j = b & (nbf - 1);
      const int k = j & (Ns - 1);
      C* x = s + a * P;
      const int base = (j - k) * RR + k;
#pragma unroll
      for (int r = 0; r < RR; ++r) x[padx(base + r * Ns)] = v[i][r];
    }
  }
  __syncthreads();
}

// Inverse transform by transposed Stockham passes in reverse order: the transpose of forward pass
// (RR, Ns) reads x[(j - k) RR + k + r Ns] (k = j mod Ns), applies the inverse RR-point DFT, multiplies
// by the conjugated twiddle of the forward table entry (k, r) and writes y[j + r N/RR].  The product
// of the transposed passes in reverse order is the transpose of the forward transform, which (the DFT
// matrix being symmetric) with conjugated twiddles is the inverse DFT; both directions share one
// twiddle table, and the first inverse pass touches exactly the elements the last forward pass wrote
// for the same butterfly, so the two can be fused with the rotation in registers.
template <int RR, int NT, int MAXB, typename C>
__device__ __forceinline__ void stockham_pass_T(C* s, int a0, int na, int logN, int Ns, const C* tw) {
  constexpr int LR = RR == 2 ? 1 : (RR == 4 ? 2 : 3);
  const int N = 1 << logN;
  const int lnbf = logN - LR, nbf = 1 << lnbf;
  const int total = na << lnbf;
  const int P = N + (N >> 3);
  C v[MAXB][RR];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * NT;
    if (b < total) {
      const int a = a0 + (b >> lnbf), j = b & (nbf - 1);
      const int k = j & (Ns - 1);
      const int base = (j - k) * RR + k;
#pragma unroll
      for (int r = 0; r < RR; ++r) v[i][r] = s[a * P + padx(base + r * Ns)];
      dft_small<RR, true>(v[i]);
      if (Ns > 1) {
        const C* t = tw + k * (RR - 1);
#pragma unroll
        for (int r = 1; r < RR; ++r) v[i][r] = cmulconj(v[i][r], t[r - 1]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * NT;
    if (b < total) {
      const int a = a0 + (b >> lnbf), j = b & (nbf - 1);
#pragma unroll
      for (int r = 0; r < RR; ++r) s[a * P + padx(j + (r << lnbf))] = v[i][r];
    }
  }
  __syncthreads();
}

template <int RR, int NT, int MAXB, int G, typename C>
__device__ __forceinline__ void pass_all_T(C* s, int narr, int logN, int Ns, const C* tw) {
  for (int a0 = 0; a0 < narr; a0 += G) stockham_pass_T<RR, NT, MAXB>(s, a0, min(G, narr - a0), logN, Ns, tw);
}

// The last transposed pass (Ns = 1, no twiddles) of the three field columns, storing straight to
// global memory: butterfly j writes z = j + r N/RR, consecutive across threads.  The column index is
// a compile-time loop index, so the column descriptors stay in registers.
template <int RR, int NT, bool SPLIT_OUT, typename C>
__device__ __forceinline__ void last_pass_T_to_global(const C* s, int logN, C* const* dst, const SplitColumn* sc) {
  constexpr int LR = RR == 2 ? 1 : (RR == 4 ? 2 : 3);
  const int N = 1 << logN;
  const int lnbf = logN - LR, nbf = 1 << lnbf;
  const int P = N + (N >> 3);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // the bf16 split stores are kept rolled: unrolled, they push the kernel out of the instruction cache
#pragma unroll 1
    for (int j = threadIdx.x; j < nbf; j += NT) {
      C v[RR];
#pragma unroll
      for (int r = 0; r < RR; ++r) v[r] = s[a * P + padx(j * RR + r)];
      dft_small<RR, true>(v);
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const int z = j + (r << lnbf);
        if (!SPLIT_OUT)
          dst[a][z] = v[r];
        else
          split_store(sc[a], z, (float)v[r].x, (float)v[r].y);
      }
    }
  }
}

// One pass over all narr arrays in groups of at most G.  A pass that reads the unpadded layout walks
// the groups last-first: group g's padded destination [g0 P, g1 P) then never overlaps the unpadded
// source [0, g0 N) of the groups still to be read (P > N).
template <int RR, bool INV, int NT, int MAXB, int G, bool SRC_PAD, typename C>
__device__ __forceinline__ void pass_all(C* s, int narr, int logN, int Ns, const C* tw) {
  const int ng = (narr + G - 1) / G;
  for (int gi = 0; gi < ng; ++gi) {
    const int g = SRC_PAD ? gi : ng - 1 - gi;
    const int a0 = g * G, na = min(G, narr - a0);
    stockham_pass<RR, INV, NT, MAXB, SRC_PAD>(s, a0, na, logN, Ns, tw);
  }
}

// Full FFT of narr arrays (forward or inverse, unnormalised), result in the padded layout:
// one small-radix pass first when log2 N is not a multiple of log2 R, then radix-R passes.
// The per-pass twiddle tables are stored back to back in pass order (first pass has none).
// Arrays go G at a time; each thread owns BPT radix-R butterflies per array per pass.
template <int R, bool INV, int NT, int G, int BPT, bool SRC_PAD, bool SKIP_LAST = false, typename C>
__device__ const C* fft_all(C* s, int narr, int logN, const C* tw) {
  const int lr = R == 8 ? 3 : 2;
  int Ns = 1;
  const int rem = logN % lr;
  bool from_pad = SRC_PAD;
  if (rem == 1) {
    if (from_pad)
      pass_all<2, INV, NT, G * BPT * (R / 2), G, true>(s, narr, logN, Ns, tw);
    else
      pass_all<2, INV, NT, G * BPT * (R / 2), G, false>(s, narr, logN, Ns, tw);
    Ns *= 2;
    from_pad = true;
  } else if (rem == 2) {
    if (from_pad)
      pass_all<4, INV, NT, G * BPT * (R / 4), G, true>(s, narr, logN, Ns, tw);
    else
      pass_all<4, INV, NT, G * BPT * (R / 4), G, false>(s, narr, logN, Ns, tw);
    Ns *= 4;
    from_pad = true;
  }
  const int npass = logN / lr - (SKIP_LAST ? 1 : 0);
  for (int p = 0; p < npass; ++p) {
    if (from_pad)
      pass_all<R, INV, NT, G * BPT, G, true>(s, narr, logN, Ns, tw);
    else
      pass_all<R, INV, NT, G * BPT, G, false>(s, narr, logN, Ns, tw);
    if (Ns > 1) tw += Ns * (R - 1);
    from_pad = true;
    Ns *= R;
  }
  return tw;
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

}  // namespace

// Kernel modes: FUSED transforms the family's field and current columns together; SOURCE
// transforms only the current columns and writes the midpoint source term (with the 1/Nz of the
// inverse transform) in kz space; MAIN transforms the field columns and adds that precomputed
// source (used when five columns do not fit in shared memory).
enum { FUSED = 0, MAIN = 1, SOURCE = 2 };

// T: data real type; K: coefficient type (double or df); PH / ZS: table records; R: FFT radix;
// NT: threads; G: arrays per pass group; BPT: radix-R butterflies per thread per array;
// TW_SMEM: twiddle tables copied to shared memory (else read through L1).
template <typename T, typename K, typename PH, typename ZS, int R, int NT, int G, int BPT, bool SPLIT_OUT, int MODE,
          bool TW_SMEM>
__global__ void __launch_bounds__(NT, (NT <= 256 ? 2 : 1)) spectral_kernel(SpectralArgs args) {
  typedef typename cplx<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t load_bar;
  C* s = reinterpret_cast<C*>(smem_raw);
  const int Nz = args.Nz, L = args.logNz, n = args.n;
  const int j = blockIdx.x, fam = blockIdx.y, md = blockIdx.z;
  const bool hasJ = MODE == FUSED ? args.hasJ : false;
  // coefficient array indices: E group (e, a, c), B group (b, d, f), J (eJ, aJ, cJ)
  int idx[5];
  int narr;
  if (MODE == SOURCE) {
    idx[0] = fam == 0 ? 6 : 8;
    idx[1] = 7;
    narr = fam == 0 ? 2 : 1;
  } else if (fam == 0) {
    idx[0] = 0; idx[1] = 1; idx[2] = 3; idx[3] = 6; idx[4] = 7;
    narr = hasJ ? 5 : 3;
  } else {
    idx[0] = 2; idx[1] = 4; idx[2] = 5; idx[3] = 8; idx[4] = 8;
    narr = hasJ ? 4 : 3;
  }
  const C* coef = reinterpret_cast<const C*>(args.coef);
  const C* twg = reinterpret_cast<const C*>(args.twiddle);
  const int P = Nz + (Nz >> 3);
  // column slots in shared memory; must match launch_one's sizing (the twiddles follow them)
  const int slots = MODE == FUSED ? (args.hasJ ? 5 : 3) : (MODE == MAIN ? 3 : 2);
  const C* tw = TW_SMEM ? s + (size_t)slots * P : twg;
  // the family's columns are contiguous in global memory: one bulk copy each into shared memory
  // (unpadded; the first FFT pass re-lays them out padded), completing on one mbarrier
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&load_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint32_t col = (uint32_t)(Nz * sizeof(C));
    const uint32_t twb = TW_SMEM ? (uint32_t)(args.tw_count * sizeof(C)) : 0u;
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
                     smem_addr(&load_bar)),
                 "r"(narr * col + twb)
                 : "memory");
    for (int a = 0; a < narr; ++a)
      bulk_g2s(s + (size_t)a * Nz, coef + ((size_t)(md * 9 + idx[a]) * n + j) * Nz, col, &load_bar);
    if (TW_SMEM) bulk_g2s(const_cast<C*>(tw), twg, twb, &load_bar);
    // the rotation reads this column's phase factors (and, in MAIN mode, the source term) straight
    // from global memory: start pulling them into L2 now, while the forward transforms run
    const PH* ph = reinterpret_cast<const PH*>(args.phase) + ((size_t)(md * 2 + fam) * n + j) * Nz;
    l2_prefetch(ph, (uint32_t)(Nz * sizeof(PH)));
    if (MODE == MAIN && args.src)
      for (int c = 0; c < 3; ++c)
        l2_prefetch(reinterpret_cast<const C*>(args.src) + (((size_t)(md * 2 + fam) * 3 + c) * n + j) * Nz, col);
  }
  __syncthreads();
  if (!bar_wait(&load_bar, 0)) {
    if (threadIdx.x == 0 && args.err) atomicCAS(args.err, 0, 8);
    return;
  }
  const PH* phase = reinterpret_cast<const PH*>(args.phase) + ((size_t)(md * 2 + fam) * n + j) * Nz;
  const ZS* zs = reinterpret_cast<const ZS*>(args.zsym);
  const K lam = reinterpret_cast<const K*>(args.lam)[(md * 2 + fam) * n + j];
  const T dt = (T)args.dt;
  const T inv = (T)1 / (T)Nz;
  C* src = reinterpret_cast<C*>(args.src) + ((size_t)(md * 2 + fam) * 3 * n + j) * Nz;  // [md][fam][3][n][Nz]
  const size_t sstride = (size_t)n * Nz;
  if (MODE == SOURCE) {
    // the current's midpoint source term -dt exp(dt M / 2) x_J / Nz in kz space, to global memory
    fft_all<R, false, NT, G, BPT, false>(s, narr, L, tw);
    for (int q = threadIdx.x; q < Nz; q += NT) {
      const int pq = padx(q);
      K spr, spi, smr, smi, A1, A2;
      T B1, B2;
      zsym_unpack(zs[q], spr, spi, smr, smi);
      phase_unpack(phase[q], A1, A2, B1, B2);
      C y0, y1, y2, z0, z1, z2;
      C j0 = s[pq], j1 = cmake<C>(0, 0), j2 = cmake<C>(0, 0);
      if (fam == 0) j1 = s[P + pq];
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
        C v = cadd(jj[c], cadd(cscale(B1, yy[c]), cscale(B2, zz[c])));
        v.x *= f;
        v.y *= f;
        src[c * sstride + q] = v;
      }
    }
    return;
  }
  // forward transforms: every pass but the last for all columns, the last pass for the current
  // columns (their kz values are read by any butterfly of the fused step below)
  constexpr int LR = R == 8 ? 3 : 2;
  const int lnbf = L - LR, nbf = 1 << lnbf;
  const C* twl = fft_all<R, false, NT, G, BPT, false, true>(s, narr, L, tw);
  if (narr > 3) stockham_pass<R, false, NT, G * BPT, true>(s, 3, narr - 3, L, nbf, twl);
  // fused, per butterfly jb of the last forward pass of the three field columns: the pass (in
  // registers), the exact rotation of its R kz values jb + r Nz/R, and the first (transposed) inverse
  // pass, which reads and writes exactly those elements - no barrier between them
  for (int jb = threadIdx.x; jb < nbf; jb += NT) {
    C v[3][R];
    const C* t = twl + jb * (R - 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[a][r] = s[a * P + padx(jb + (r << lnbf))];
#pragma unroll
      for (int r = 1; r < R; ++r) v[a][r] = cmul(v[a][r], t[r - 1]);
      dft_small<R, false>(v[a]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int q = jb + (r << lnbf);
      const int pq = padx(q);
      K spr, spi, smr, smi, A1, A2;
      T B1, B2;
      zsym_unpack(zs[q], spr, spi, smr, smi);
      phase_unpack(phase[q], A1, A2, B1, B2);
      C j0 = cmake<C>(0, 0), j1 = cmake<C>(0, 0);
      if (hasJ) {
        j0 = s[3 * P + pq];
        if (fam == 0) j1 = s[4 * P + pq];
      }
      rotate_point<T, K, C>(v[0][r], v[1][r], v[2][r], j0, j1, hasJ, fam, lam, spr, spi, smr, smi, A1, A2, B1, B2,
                            dt, inv);
      if (MODE == MAIN && args.src) {
        v[0][r] = cadd(v[0][r], src[q]);
        v[1][r] = cadd(v[1][r], src[sstride + q]);
        v[2][r] = cadd(v[2][r], src[2 * sstride + q]);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dft_small<R, true>(v[a]);
#pragma unroll
      for (int r = 1; r < R; ++r) v[a][r] = cmulconj(v[a][r], t[r - 1]);
#pragma unroll
      for (int r = 0; r < R; ++r) s[a * P + padx(jb + (r << lnbf))] = v[a][r];
    }
  }
  __syncthreads();
  // remaining inverse passes: transposes of the forward radix-R passes in reverse order (each pass
  // table sits before the next pass's in the forward layout), then the first forward pass's
  // transpose, which writes the result (or its bf16 split pieces) to global memory
  const int rem = L % LR, npass = L / LR;
  const C* tp = twl;
  for (int p = npass - 2; p >= (rem ? 0 : 1); --p) {
    const int Nsp = (1 << rem) << (LR * p);
    if (Nsp > 1) tp -= Nsp * (R - 1);
    pass_all_T<R, NT, G * BPT, G>(s, 3, L, Nsp, tp);
  }
  C* out = reinterpret_cast<C*>(args.coef);
  C* dst[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) dst[a] = out + ((size_t)(md * 9 + idx[a]) * n + j) * Nz;
  SplitColumn sc[3];
  if (SPLIT_OUT) {
#pragma unroll
    for (int a = 0; a < 3; ++a) sc[a] = split_column(args.split_out, args.npieces, md, idx[a], j, args.split_kstages, Nz);
  }
  if (rem == 1)
    last_pass_T_to_global<2, NT, SPLIT_OUT>(s, L, dst, sc);
  else if (rem == 2)
    last_pass_T_to_global<4, NT, SPLIT_OUT>(s, L, dst, sc);
  else
    last_pass_T_to_global<R, NT, SPLIT_OUT>(s, L, dst, sc);
}

template <typename T, typename K, typename PH, typename ZS, int R, int NT, int G, int BPT, bool SPLIT, int MODE,
          bool TW_SMEM>
static cudaError_t launch_one(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  typedef typename cplx<T>::type C;
  const int arrays = MODE == FUSED ? (a.hasJ ? 5 : 3) : (MODE == MAIN ? 3 : 2);  // = the kernel's `slots`
  const size_t smem = ((size_t)arrays * (a.Nz + a.Nz / 8) + (TW_SMEM ? (size_t)a.tw_count : 0)) * sizeof(C);
  auto k = spectral_kernel<T, K, PH, ZS, R, NT, G, BPT, SPLIT, MODE, TW_SMEM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.n, 2, nmodes);
  k<<<grid, NT, smem, st>>>(a);
  return cudaGetLastError();
}

// Configuration by transform length: NT = max(128, Nz / R) threads up to 512, groups of three arrays
// while one butterfly per thread per array suffices; beyond that one array at a time with two.
template <typename T, typename K, typename PH, typename ZS, int R, bool SPLIT, int MODE, bool TW_SMEM>
static cudaError_t launch_sized(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  const int need = a.Nz / R;
  if (need <= 128) return launch_one<T, K, PH, ZS, R, 128, 3, 1, SPLIT, MODE, TW_SMEM>(a, nmodes, st);
  if (need <= 256) return launch_one<T, K, PH, ZS, R, 256, 3, 1, SPLIT, MODE, TW_SMEM>(a, nmodes, st);
  if (need <= 512) return launch_one<T, K, PH, ZS, R, 512, 3, 1, SPLIT, MODE, TW_SMEM>(a, nmodes, st);
  if (need <= 1024) return launch_one<T, K, PH, ZS, R, 512, 1, 2, SPLIT, MODE, TW_SMEM>(a, nmodes, st);
  return cudaErrorNotSupported;
}

static size_t fused_bytes(int Nz, int precision, bool hasJ, int tw_count) {
  return ((size_t)(hasJ ? 5 : 3) * (Nz + Nz / 8) + (size_t)tw_count) * (precision == 0 ? 16 : 8);
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

bool spectral_needs_source(int Nz, int precision, int tw_count) {
  return fused_bytes(Nz, precision, true, tw_count) > 227 * 1024;
}

// Smallest shared-memory footprint a plan needs: the three field columns of the two-kernel path
// (padded layout, twiddles through L1).  The fused path is used whenever it fits.
size_t spectral_smem_bytes(int Nz, int precision, bool hasJ) {
  (void)hasJ;
  return (size_t)3 * (Nz + Nz / 8) * (precision == 0 ? 16 : 8);
}

// Per-pass twiddle tables in the order fft_all consumes them, for radix R (8 for FP32, 4 for FP64):
// the first (small-radix) pass needs none; pass p with sub-length Ns and radix R stores
// exp(-2 pi i r k / (Ns R)) at k*(R-1) + r-1 for k < Ns, r = 1..R-1.
int spectral_twiddles(int Nz, int precision, double* re, double* im) {
  const int R = precision == 0 ? 4 : 8, lr = precision == 0 ? 2 : 3;
  int logN = 0;
  while ((1 << logN) < Nz) ++logN;
  int Ns = 1 << (logN % lr), cnt = 0;
  const double pi = 3.14159265358979323846;
  for (int p = 0; p < logN / lr; ++p) {
    if (Ns > 1) {
      for (int k = 0; k < Ns; ++k)
        for (int r = 1; r < R; ++r) {
          // reduce the angle exactly: r k / (Ns R) of a full turn
          const long long num = ((long long)r * k) % ((long long)Ns * R);
          const double ang = -2.0 * pi * (double)num / ((double)Ns * R);
          if (re) {
            re[cnt] = cos(ang);
            im[cnt] = sin(ang);
          }
          ++cnt;
        }
    }
    Ns *= R;
  }
  return cnt;
}

}  // namespace fdetd
