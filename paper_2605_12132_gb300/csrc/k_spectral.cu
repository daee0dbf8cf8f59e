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
// The z transform is an in-shared-memory radix-2 FFT (decimation in time after a
// bit-reversed load, decimation in frequency for the inverse), all arrays of the
// family advancing through each stage together.
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
  A1 = p.A1; A2 = p.A2; B1 = p.B1; B2 = p.B2;
}
__device__ __forceinline__ void phase_unpack(const PhaseF& p, df& A1, df& A2, float& B1, float& B2) {
  A1 = p.A1; A2 = p.A2; B1 = p.B1; B2 = p.B2;
}
__device__ __forceinline__ void zsym_unpack(const ZSymD& z, double& spr, double& spi, double& smr, double& smi) {
  spr = z.spr; spi = z.spi; smr = z.smr; smi = z.smi;
}
__device__ __forceinline__ void zsym_unpack(const ZSymF& z, df& spr, df& spi, df& smr, df& smi) {
  spr = z.spr; spi = z.spi; smr = z.smr; smi = z.smi;
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

}  // namespace

// T: data real type; K: coefficient type (double or df); PH / ZS: table records.
template <typename T, typename K, typename PH, typename ZS, bool SPLIT_OUT>
__global__ void __launch_bounds__(256) spectral_kernel(SpectralArgs args) {
  typedef typename cplx<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int Nz = args.Nz, L = args.logNz, n = args.n;
  const int j = blockIdx.x, fam = blockIdx.y, md = blockIdx.z;
  const bool hasJ = args.hasJ;
  // coefficient array indices: E group (e, a, c), B group (b, d, f), J (eJ, aJ, cJ)
  int idx[5];
  int narr;
  if (fam == 0) {
    idx[0] = 0; idx[1] = 1; idx[2] = 3; idx[3] = 6; idx[4] = 7;
    narr = hasJ ? 5 : 3;
  } else {
    idx[0] = 2; idx[1] = 4; idx[2] = 5; idx[3] = 8; idx[4] = 8;
    narr = hasJ ? 4 : 3;
  }
  const C* coef = reinterpret_cast<const C*>(args.coef);
  const C* tw = reinterpret_cast<const C*>(args.twiddle);
  for (int a = 0; a < narr; ++a) {
    const C* src = coef + ((size_t)(md * 9 + idx[a]) * n + j) * Nz;
    C* dst = s + (size_t)a * Nz;
    for (int z = threadIdx.x; z < Nz; z += blockDim.x) dst[bitrev(z, L)] = src[z];
  }
  __syncthreads();
  const int half_total = Nz >> 1;
  for (int st = 0; st < L; ++st) {
    const int half = 1 << st;
    for (int b = threadIdx.x; b < narr * half_total; b += blockDim.x) {
      const int a = b / half_total, bb = b - a * half_total;
      const int grp = bb >> st, pos = bb & (half - 1);
      const int i0 = grp * 2 * half + pos, i1 = i0 + half;
      C* x = s + (size_t)a * Nz;
      const C w = tw[pos << (L - 1 - st)];
      const C t = cmul(w, x[i1]);
      const C u = x[i0];
      x[i0] = cadd(u, t);
      x[i1] = csub(u, t);
    }
    __syncthreads();
  }
  // exact rotation per kz
  const PH* phase = reinterpret_cast<const PH*>(args.phase) + ((size_t)(md * 2 + fam) * n + j) * Nz;
  const ZS* zs = reinterpret_cast<const ZS*>(args.zsym);
  const K lam = reinterpret_cast<const K*>(args.lam)[(md * 2 + fam) * n + j];
  const T dt = (T)args.dt;
  for (int q = threadIdx.x; q < Nz; q += blockDim.x) {
    K spr, spi, smr, smi, A1, A2;
    T B1, B2;
    zsym_unpack(zs[q], spr, spi, smr, smi);
    phase_unpack(phase[q], A1, A2, B1, B2);
    C x0 = s[q], x1 = s[Nz + q], x2 = s[2 * Nz + q];
    C j0 = cmake<C>(0, 0), j1 = cmake<C>(0, 0), j2 = cmake<C>(0, 0);
    if (hasJ) {
      j0 = s[3 * Nz + q];
      if (fam == 0) j1 = s[4 * Nz + q];
    }
    C y0, y1, y2, z0, z1, z2, yj0, yj1, yj2, zj0, zj1, zj2;
    if (fam == 0) {
      apply_tm(x0, x1, x2, y0, y1, y2, lam, spr, spi, smr, smi);
      apply_tm(y0, y1, y2, z0, z1, z2, lam, spr, spi, smr, smi);
      apply_tm(j0, j1, j2, yj0, yj1, yj2, lam, spr, spi, smr, smi);
      apply_tm(yj0, yj1, yj2, zj0, zj1, zj2, lam, spr, spi, smr, smi);
    } else {
      apply_te(x0, x1, x2, y0, y1, y2, lam, spr, spi, smr, smi);
      apply_te(y0, y1, y2, z0, z1, z2, lam, spr, spi, smr, smi);
      apply_te(j0, j1, j2, yj0, yj1, yj2, lam, spr, spi, smr, smi);
      apply_te(yj0, yj1, yj2, zj0, zj1, zj2, lam, spr, spi, smr, smi);
    }
    s[q] = combine(x0, y0, z0, A1, A2, j0, yj0, zj0, B1, B2, dt, hasJ);
    s[Nz + q] = combine(x1, y1, z1, A1, A2, j1, yj1, zj1, B1, B2, dt, hasJ);
    s[2 * Nz + q] = combine(x2, y2, z2, A1, A2, j2, yj2, zj2, B1, B2, dt, hasJ);
  }
  __syncthreads();
  for (int st = L - 1; st >= 0; --st) {
    const int half = 1 << st;
    for (int b = threadIdx.x; b < 3 * half_total; b += blockDim.x) {
      const int a = b / half_total, bb = b - a * half_total;
      const int grp = bb >> st, pos = bb & (half - 1);
      const int i0 = grp * 2 * half + pos, i1 = i0 + half;
      C* x = s + (size_t)a * Nz;
      const C w = tw[pos << (L - 1 - st)];
      const C u = x[i0], v = x[i1];
      x[i0] = cadd(u, v);
      x[i1] = cmulconj(csub(u, v), w);
    }
    __syncthreads();
  }
  const T inv = (T)1 / (T)Nz;
  if (!SPLIT_OUT) {
    C* out = reinterpret_cast<C*>(args.coef);
    for (int a = 0; a < 3; ++a) {
      C* dst = out + ((size_t)(md * 9 + idx[a]) * n + j) * Nz;
      const C* x = s + (size_t)a * Nz;
      for (int z = threadIdx.x; z < Nz; z += blockDim.x) {
        C v = x[bitrev(z, L)];
        v.x *= inv;
        v.y *= inv;
        dst[z] = v;
      }
    }
  } else {
    // bf16 split pieces for the tensor-core back-projection: [md][piece][6][n][Nz*2] (re, im interleaved)
    for (int a = 0; a < 3; ++a) {
      const C* x = s + (size_t)a * Nz;
      for (int z = threadIdx.x; z < Nz; z += blockDim.x) {
        C v = x[bitrev(z, L)];
        const float vr = (float)(v.x * inv), vi = (float)(v.y * inv);
        split_store(args.split_out, args.npieces, md, idx[a], j, z, args.split_rows, Nz, vr, vi);
      }
    }
  }
}

template <typename T, typename K, typename PH, typename ZS, bool SPLIT>
static cudaError_t launch_one(const SpectralArgs& a, int nmodes, cudaStream_t st) {
  typedef typename cplx<T>::type C;
  const size_t smem = (size_t)(a.hasJ ? 5 : 3) * a.Nz * sizeof(C);
  auto k = spectral_kernel<T, K, PH, ZS, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.n, 2, nmodes);
  k<<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_spectral(const SpectralArgs& a, int nmodes, int precision, bool split_out, cudaStream_t st) {
  if (precision == 0) return launch_one<double, double, PhaseD, ZSymD, false>(a, nmodes, st);
  if (split_out) return launch_one<float, df, PhaseF, ZSymF, true>(a, nmodes, st);
  return launch_one<float, df, PhaseF, ZSymF, false>(a, nmodes, st);
}

size_t spectral_smem_bytes(int Nz, int precision, bool hasJ) {
  return (size_t)(hasJ ? 5 : 3) * Nz * (precision == 0 ? 16 : 8);
}

}  // namespace fdetd
