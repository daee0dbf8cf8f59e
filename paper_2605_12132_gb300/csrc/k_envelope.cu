// One Taylor term of the envelope propagator (Sec. 4.2, Eq. spatialAM_envelope_H,
// complex form):
//   H_a (a, a~) = (a~,  (L_rho + L_z - chi) a + 2 i k0 (D_z^(C) a + a~))
//   out = (dt/n) H_a(in),  accout = accin + out.
// L_rho is a banded radial matrix (centred D^2 + rho^-1 D^(C), symmetric axis mirror
// folded in, taps past the outer edge dropped); z stencils are periodic.
#include "kernels.h"

namespace fdetd {

__global__ void __launch_bounds__(256) envelope_term_kernel(EnvArgs a) {
  const int r = blockIdx.x * 32 + (threadIdx.x & 31);
  const int z = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (r >= a.Nr || z >= a.Nz) return;
  const int Nr = a.Nr, Nz = a.Nz, N = a.N, W = 2 * N + 1;
  const size_t idx = (size_t)z * Nr + r;
  const float2 ac = a.in_a[idx], at = a.in_t[idx];
  // Stencils in difference form: sum_t w_t (a_{r+t} - a_r) + (sum_t w_t) a_r radially and
  // sum_n e_n (a_{z+n} + a_{z-n} - 2 a_z) along z, so that the large individual weights
  // (~dr^-2) act on small differences instead of cancelling in FP32.
  const float* band = a.lr + (size_t)r * (W + 1);
  const float2* row = a.in_a + (size_t)z * Nr;
  float lx = band[W] * ac.x, ly = band[W] * ac.y;  // row sum of the band
  for (int t = -N; t <= N; ++t) {
    const int c = r + t;
    if (t == 0 || c < 0 || c >= Nr) continue;
    const float w = band[t + N];
    const float2 v = row[c];
    lx = fmaf(w, v.x - ac.x, lx);
    ly = fmaf(w, v.y - ac.y, ly);
  }
  float dx = 0.f, dy = 0.f;
  for (int t = 1; t <= N; ++t) {
    int zp = z + t, zm = z - t;
    if (zp >= Nz) zp -= Nz;
    if (zm < 0) zm += Nz;
    const float2 p = a.in_a[(size_t)zp * Nr + r], m = a.in_a[(size_t)zm * Nr + r];
    lx = fmaf(a.cz2[t], (p.x - ac.x) + (m.x - ac.x), lx);
    ly = fmaf(a.cz2[t], (p.y - ac.y) + (m.y - ac.y), ly);
    dx = fmaf(a.cz1[t], p.x - m.x, dx);
    dy = fmaf(a.cz1[t], p.y - m.y, dy);
  }
  const float chi = a.chi[idx];
  // i * 2k0 * (d + a~) = (-2k0 (dy + at.y), 2k0 (dx + at.x))
  const float tx = lx - chi * ac.x - a.k2 * (dy + at.y);
  const float ty = ly - chi * ac.y + a.k2 * (dx + at.x);
  const float2 oa = make_float2(a.scale * at.x, a.scale * at.y);
  const float2 ot = make_float2(a.scale * tx, a.scale * ty);
  if (a.out_a) {
    a.out_a[idx] = oa;
    a.out_t[idx] = ot;
  }
  const float2 pa = a.accin_a[idx], pt = a.accin_t[idx];
  a.accout_a[idx] = make_float2(pa.x + oa.x, pa.y + oa.y);
  a.accout_t[idx] = make_float2(pt.x + ot.x, pt.y + ot.y);
}

cudaError_t launch_envelope_term(const EnvArgs& a, cudaStream_t st) {
  dim3 grid((a.Nr + 31) / 32, (a.Nz + 7) / 8);
  envelope_term_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// Absorbing layer (appendix, Eq. absorbingA_solution2): the split-operator step
//   exp(-sigma dt / 4) exp(H_a dt) exp(-sigma dt / 4) with chi~ = chi + sigma^2 inside H_a.
__global__ void envelope_chit_kernel(const float* chi, const float* sigma, float* chit, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) chit[i] = chi[i] + sigma[i] * sigma[i];
}

// (a, a~) *= exp(c sigma) pointwise, a and a~ the two consecutive planes of n points
__global__ void envelope_damp_kernel(float2* psi, const float* sigma, float c, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float f = expf(c * sigma[i]);
  float2 u = psi[i], v = psi[n + i];
  psi[i] = make_float2(f * u.x, f * u.y);
  psi[n + i] = make_float2(f * v.x, f * v.y);
}

cudaError_t launch_envelope_chit(const float* chi, const float* sigma, float* chit, size_t n, cudaStream_t st) {
  envelope_chit_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(chi, sigma, chit, n);
  return cudaGetLastError();
}

cudaError_t launch_envelope_damp(float2* psi, const float* sigma, float c, size_t n, cudaStream_t st) {
  envelope_damp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(psi, sigma, c, n);
  return cudaGetLastError();
}

}  // namespace fdetd

namespace fdetd {

// ---------------------------------------------------------------- all Taylor terms in one launch
// One envelope step psi <- psi + sum_{n=1}^{N_T} (dt H_a)^n / n! psi, every term computed from the previous
// one inside a tile held in shared memory (temporal blocking).  A CTA owns an output tile of ET_Z z rows x
// ET_R radii; term n is needed on the tile grown by (N_T - n) N cells on each side (the stencil reach N =
// order/2 per term), so the state is loaded on the tile grown by N_T N (z periodic; radii outside 0..Nr-1
// are never read by a real radius, whose band has its axis mirror folded in and its taps past the outer edge
// dropped).  Each thread computes its cells of the next term into registers, the block synchronises, and the
// term overwrites the previous one in place; the running sum of the output cells stays in registers.  The
// per-cell arithmetic is that of envelope_term_kernel (difference-form stencils, same order of operations),
// so the result equals the term-by-term launches bit for bit.  psi_in and psi_out must not alias (other
// tiles read psi_in's halo).
constexpr int ET_Z = 32, ET_R = 32, ET_NT = 512;

template <int N, int NTAY>
__global__ void __launch_bounds__(ET_NT, 1) envelope_fused_kernel(EnvArgs a, const float2* __restrict__ in_a,
                                                                    const float2* __restrict__ in_t,
                                                                    float2* __restrict__ out_a,
                                                                    float2* __restrict__ out_t) {
  constexpr int HALO = N * NTAY, DZ = ET_Z + 2 * HALO, DR = ET_R + 2 * HALO, W = 2 * N + 1;
  constexpr int ZSTEP = ET_NT / DR, ROWS_PER = DZ / ZSTEP;   // a thread owns rows lz0 + ZSTEP k of one column
  // the output rows HALO .. HALO + ET_Z - 1 are those of k in [K0, K0 + KO) for every lz0 < ZSTEP
  constexpr int K0 = HALO / ZSTEP, KO = ET_Z / ZSTEP;
  static_assert(ET_NT % DR == 0 && DZ % ZSTEP == 0 && HALO % ZSTEP == 0 && ET_Z % ZSTEP == 0, "tile shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sa = reinterpret_cast<float2*>(smem_raw);          // [DZ][DR] a of the current term
  float2* st = sa + DZ * DR;                                  // [DZ][DR] a~ of the current term
  float* sc = reinterpret_cast<float*>(st + DZ * DR);        // [DZ][DR] chi
  const int Nz = a.Nz, Nr = a.Nr;
  const int z0 = blockIdx.y * ET_Z - HALO, r0 = blockIdx.x * ET_R - HALO;
  // load the state and chi on the grown tile
  for (int i = threadIdx.x; i < DZ * DR; i += ET_NT) {
    const int lz = i / DR, lr = i - lz * DR;
    int z = z0 + lz;
    z = z < 0 ? z + Nz : (z >= Nz ? z - Nz : z);
    const int r = r0 + lr;
    float2 va = make_float2(0.f, 0.f), vt = va;
    float vc = 0.f;
    if (r >= 0 && r < Nr) {
      const size_t g = (size_t)z * Nr + r;
      va = in_a[g];
      vt = in_t[g];
      vc = a.chi[g];
    }
    sa[i] = va;
    st[i] = vt;
    sc[i] = vc;
  }
  // this thread's domain column and its radius' band (weights and row sum)
  const int lr = threadIdx.x % DR, lz0 = threadIdx.x / DR;
  const int r = r0 + lr;
  const bool real_r = r >= 0 && r < Nr;
  float band[W + 1];
#pragma unroll
  for (int t = 0; t <= W; ++t) band[t] = real_r ? a.lr[(size_t)r * (W + 1) + t] : 0.f;
  float2 sum_a[KO], sum_t[KO];
  __syncthreads();
  // the output cells' sums start from the state
#pragma unroll
  for (int k = 0; k < KO; ++k) {
    const int lz = lz0 + (K0 + k) * ZSTEP;
    sum_a[k] = sa[lz * DR + lr];
    sum_t[k] = st[lz * DR + lr];
  }
#pragma unroll 1
  for (int n = 1; n <= NTAY; ++n) {
    const int lo = n * N, hi_z = DZ - n * N, hi_r = DR - n * N;   // term n's domain in tile coordinates
    const bool col_in = real_r && lr >= lo && lr < hi_r;
    const float scale = a.dt_over[n];   // (float)(dt / n), as the term-by-term launches use
    float2 na[ROWS_PER], nt[ROWS_PER];
#pragma unroll
    for (int k = 0; k < ROWS_PER; ++k) {
      const int lz = lz0 + k * ZSTEP;
      na[k] = make_float2(0.f, 0.f);
      nt[k] = make_float2(0.f, 0.f);
      if (!col_in || lz < lo || lz >= hi_z) continue;
      const int idx = lz * DR + lr;
      const float2 ac = sa[idx], at = st[idx];
      const float2* row = sa + lz * DR;
      float lx = band[W] * ac.x, ly = band[W] * ac.y;
#pragma unroll
      for (int t = -N; t <= N; ++t) {
        const int c = r + t;
        if (t == 0 || c < 0 || c >= Nr) continue;
        const float w = band[t + N];
        const float2 v = row[lr + t];
        lx = fmaf(w, v.x - ac.x, lx);
        ly = fmaf(w, v.y - ac.y, ly);
      }
      float dx = 0.f, dy = 0.f;
#pragma unroll
      for (int t = 1; t <= N; ++t) {
        const float2 p = sa[idx + t * DR], m = sa[idx - t * DR];
        lx = fmaf(a.cz2[t], (p.x - ac.x) + (m.x - ac.x), lx);
        ly = fmaf(a.cz2[t], (p.y - ac.y) + (m.y - ac.y), ly);
        dx = fmaf(a.cz1[t], p.x - m.x, dx);
        dy = fmaf(a.cz1[t], p.y - m.y, dy);
      }
      const float chi = sc[idx];
      const float tx = lx - chi * ac.x - a.k2 * (dy + at.y);
      const float ty = ly - chi * ac.y + a.k2 * (dx + at.x);
      na[k] = make_float2(scale * at.x, scale * at.y);
      nt[k] = make_float2(scale * tx, scale * ty);
    }
    __syncthreads();   // every read of the previous term is done
#pragma unroll
    for (int k = 0; k < ROWS_PER; ++k) {
      const int lz = lz0 + k * ZSTEP;
      const int idx = lz * DR + lr;
      sa[idx] = na[k];
      st[idx] = nt[k];
      if (k >= K0 && k < K0 + KO) {
        sum_a[k - K0] = make_float2(sum_a[k - K0].x + na[k].x, sum_a[k - K0].y + na[k].y);
        sum_t[k - K0] = make_float2(sum_t[k - K0].x + nt[k].x, sum_t[k - K0].y + nt[k].y);
      }
    }
    __syncthreads();
  }
  // the output tile
#pragma unroll
  for (int k = 0; k < KO; ++k) {
    const int lz = lz0 + (K0 + k) * ZSTEP;
    if (lr < HALO || lr >= HALO + ET_R || !real_r) continue;
    const int z = z0 + lz;
    if (z >= Nz) continue;
    const size_t g = (size_t)z * Nr + r;
    out_a[g] = sum_a[k];
    out_t[g] = sum_t[k];
  }
}

size_t envelope_fused_smem(int order, int taylor_order) {
  const int halo = (order / 2) * taylor_order, dz = ET_Z + 2 * halo, dr = ET_R + 2 * halo;
  return (size_t)dz * dr * (8 + 8 + 4);
}

bool envelope_fused_supported(int order, int taylor_order) {
  const int halo = (order / 2) * taylor_order, dr = ET_R + 2 * halo;
  return (order == 8 && taylor_order == 4) && ET_NT % dr == 0 && envelope_fused_smem(order, taylor_order) <= 227 * 1024;
}

cudaError_t launch_envelope_fused(const EnvArgs& a, const float2* in_a, const float2* in_t, float2* out_a,
                                  float2* out_t, int taylor_order, cudaStream_t st) {
  if (a.N != 4 || taylor_order != 4) return cudaErrorNotSupported;
  if (a.Nz % ET_Z) return cudaErrorNotSupported;
  const size_t smem = envelope_fused_smem(2 * a.N, taylor_order);
  auto k = envelope_fused_kernel<4, 4>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.Nr + ET_R - 1) / ET_R, a.Nz / ET_Z);
  k<<<grid, ET_NT, smem, st>>>(a, in_a, in_t, out_a, out_t);
  return cudaGetLastError();
}

}  // namespace fdetd
