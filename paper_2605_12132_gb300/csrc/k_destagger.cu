// Destagger of the Yee-grid field modes to the primary grids (Sec. 3 field interpolation, Eqs.
// shapesAM_destagger_E, _B, _Bth), with the upstaggering Lagrange interpolation S^(+) of Eq.
// spatialAM_staggerS at the order of the finite differences:
//   E_rho -> S_rho^(+, mA) E_rho,  E_z, B_rho -> S_z^(+),  B_z -> S_rho^(+, mS) B_z,
//   B_theta -> S_rho^(+, mA) S_z^(+) B_theta,  E_theta copied.
// The half-point value uses the 2 N_D nearest nodes (weights w_t, t = -N_D+1 .. N_D); z is periodic;
// radially the operand sits on rho_-,j = j dr with the axis value in slot 0, nodes j < 0 mirror to -j
// with the sign of the symmetric / antisymmetric extension, nodes past the outer edge are dropped.
// The stencils read neighbours through the read-only cache; B_theta goes through a shared row.
#include "common.cuh"
#include "kernels.h"

namespace fdetd {
namespace {

template <typename T>
struct DestagArgs {
  const typename cplx<T>::type* in;  // [nm][6][Nz][n]
  typename cplx<T>::type* out;       // [nm][6][Nz][n]
  T w[32];                           // w[t + N - 1], t = -N+1 .. N
  int Nz, n, N, nm;
  signed char signA[64], signS[64];  // +1 symmetric / -1 antisymmetric extension per mode
};

// One CTA per 8 z rows of one mode (a warp per row, lanes over the radii).  Phase 1: the z stencils
// (E_z, B_rho written; B_theta interpolated in z into shared memory).  Phase 2: the radial stencils
// (E_rho, B_z from global memory; B_theta from the shared row), E_theta copied.  B_theta's 2-D
// interpolation is separable, so it costs 2 x 2 N_D reads per point instead of (2 N_D)^2.
template <typename T>
__global__ void __launch_bounds__(256) destagger_kernel(DestagArgs<T> a) {
  typedef typename cplx<T>::type C;
  extern __shared__ __align__(16) unsigned char dsm[];
  C* btz = reinterpret_cast<C*>(dsm);  // [8][n]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z = blockIdx.x * 8 + warp, md = blockIdx.y;
  const int n = a.n, Nz = a.Nz, N = a.N;
  const size_t fs = (size_t)Nz * n;
  const C* F = a.in + (size_t)md * 6 * fs;
  C* O = a.out + (size_t)md * 6 * fs;
  const bool live = z < Nz;
  if (live) {
    for (int k = lane; k < n; k += 32) {
      C ez = cmake<C>(0, 0), br = ez, bt = ez;
      for (int t = -N + 1; t <= N; ++t) {
        const T wt = a.w[t + N - 1];
        int zz = z + t;
        if (zz < 0) zz += Nz;
        if (zz >= Nz) zz -= Nz;
        const size_t q = (size_t)zz * n + k;
        const C v2 = __ldg(&F[2 * fs + q]), v3 = __ldg(&F[3 * fs + q]), v4 = __ldg(&F[4 * fs + q]);
        ez.x += wt * v2.x;
        ez.y += wt * v2.y;
        br.x += wt * v3.x;
        br.y += wt * v3.y;
        bt.x += wt * v4.x;
        bt.y += wt * v4.y;
      }
      const size_t i0 = (size_t)z * n + k;
      O[2 * fs + i0] = ez;
      O[3 * fs + i0] = br;
      btz[warp * n + k] = bt;
    }
  }
  __syncthreads();
  if (!live) return;
  const T sA = (T)a.signA[md], sS = (T)a.signS[md];
  const size_t row = (size_t)z * n;
  for (int k = lane; k < n; k += 32) {
    C er = cmake<C>(0, 0), bz = er, bt = er;
    for (int t = -N + 1; t <= N; ++t) {
      const T wt = a.w[t + N - 1];
      int j = k + t;
      T sgA = (T)1, sgS = (T)1;
      if (j < 0) {
        j = -j;
        sgA = sA;
        sgS = sS;
      }
      if (j >= n) continue;
      const C vr = __ldg(&F[row + j]), vz = __ldg(&F[5 * fs + row + j]), vb = btz[warp * n + j];
      er.x += wt * sgA * vr.x;
      er.y += wt * sgA * vr.y;
      bz.x += wt * sgS * vz.x;
      bz.y += wt * sgS * vz.y;
      bt.x += wt * sgA * vb.x;
      bt.y += wt * sgA * vb.y;
    }
    const size_t i0 = row + k;
    O[i0] = er;
    O[fs + i0] = __ldg(&F[fs + i0]);
    O[4 * fs + i0] = bt;
    O[5 * fs + i0] = bz;
  }
}

}  // namespace

cudaError_t launch_destagger(const void* in, void* out, int Nz, int n, int order, const int* modes, int nmodes,
                             bool fp64, cudaStream_t st) {
  const int N = order / 2;
  if (N < 1 || N > 16 || nmodes < 1 || nmodes > 64) return cudaErrorInvalidValue;
  // Lagrange weights of the value at t = 1/2 from the nodes t = -N+1 .. N
  double w[32];
  for (int i = -N + 1; i <= N; ++i) {
    double num = 1.0, den = 1.0;
    for (int l = -N + 1; l <= N; ++l)
      if (l != i) {
        num *= 0.5 - l;
        den *= (double)(i - l);
      }
    w[i + N - 1] = num / den;
  }
  const dim3 grid((Nz + 7) / 8, nmodes);
  const size_t smem = (size_t)8 * n * (fp64 ? 16 : 8);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto fill = [&](auto& a) {
    a.Nz = Nz;
    a.n = n;
    a.N = N;
    a.nm = nmodes;
    for (int i = 0; i < 2 * N; ++i) a.w[i] = w[i];
    for (int i = 0; i < nmodes; ++i) {
      const int m = modes[i];
      a.signA[i] = ((m - 1 < 0 ? 1 - m : m - 1) % 2 == 0) ? 1 : -1;
      a.signS[i] = (m % 2 == 0) ? 1 : -1;
    }
  };
  if (fp64) {
    DestagArgs<double> a;
    fill(a);
    a.in = (const double2*)in;
    a.out = (double2*)out;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(destagger_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    destagger_kernel<double><<<grid, 256, smem, st>>>(a);
  } else {
    DestagArgs<float> a;
    fill(a);
    a.in = (const float2*)in;
    a.out = (float2*)out;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(destagger_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    destagger_kernel<float><<<grid, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace fdetd
