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
