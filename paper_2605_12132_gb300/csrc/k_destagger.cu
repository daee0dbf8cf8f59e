// Destagger of the Yee-grid field modes to the primary grids (Sec. 3 field interpolation, Eqs.
// shapesAM_destagger_E, _B, _Bth), with the upstaggering Lagrange interpolation S^(+) of Eq.
// spatialAM_staggerS at the order of the finite differences:
//   E_rho -> S_rho^(+, mA) E_rho,  E_z, B_rho -> S_z^(+),  B_z -> S_rho^(+, mS) B_z,
//   B_theta -> S_rho^(+, mA) S_z^(+) B_theta,  E_theta copied.
// The half-point value uses the 2 N_D nearest nodes (weights w_t, t = -N_D+1 .. N_D); z is periodic;
// radially the operand sits on rho_-,j = j dr with the axis value in slot 0, nodes j < 0 mirror to -j
// with the sign of the symmetric / antisymmetric extension, nodes past the outer edge are dropped.
// One thread per (mode, z, radial point); the stencils read neighbours through the read-only cache.
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

template <typename T>
__global__ void __launch_bounds__(256) destagger_kernel(DestagArgs<T> a) {
  typedef typename cplx<T>::type C;
  const int k = blockIdx.x * 32 + (threadIdx.x & 31);
  const int z = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int md = blockIdx.z;
  const int n = a.n, Nz = a.Nz, N = a.N;
  if (k >= n || z >= Nz) return;
  const size_t fs = (size_t)Nz * n;
  const C* F = a.in + (size_t)md * 6 * fs;
  C* O = a.out + (size_t)md * 6 * fs;
  const T sA = (T)a.signA[md], sS = (T)a.signS[md];
  C er = cmake<C>(0, 0), ez = er, br = er, bt = er, bz = er;
  for (int t = -N + 1; t <= N; ++t) {
    const T wt = a.w[t + N - 1];
    // radial node k + t (mirror through the axis for negative indices)
    int j = k + t;
    T sgnA = (T)1, sgnS = (T)1;
    if (j < 0) {
      j = -j;
      sgnA = sA;
      sgnS = sS;
    }
    if (j < n) {
      const size_t row = (size_t)z * n + j;
      const C vr = __ldg(&F[row]), vz = __ldg(&F[5 * fs + row]);
      er.x += wt * sgnA * vr.x;
      er.y += wt * sgnA * vr.y;
      bz.x += wt * sgnS * vz.x;
      bz.y += wt * sgnS * vz.y;
      // B_theta: the z interpolation at radial node j, then the radial weight
      C btz = cmake<C>(0, 0);
      for (int s = -N + 1; s <= N; ++s) {
        int zz = z + s;
        if (zz < 0) zz += Nz;
        if (zz >= Nz) zz -= Nz;
        const C v = __ldg(&F[4 * fs + (size_t)zz * n + j]);
        const T ws = a.w[s + N - 1];
        btz.x += ws * v.x;
        btz.y += ws * v.y;
      }
      bt.x += wt * sgnA * btz.x;
      bt.y += wt * sgnA * btz.y;
    }
    // z node z + t (periodic) at radius k
    int zz = z + t;
    if (zz < 0) zz += Nz;
    if (zz >= Nz) zz -= Nz;
    const size_t q = (size_t)zz * n + k;
    const C vz2 = __ldg(&F[2 * fs + q]), vb = __ldg(&F[3 * fs + q]);
    ez.x += wt * vz2.x;
    ez.y += wt * vz2.y;
    br.x += wt * vb.x;
    br.y += wt * vb.y;
  }
  const size_t i0 = (size_t)z * n + k;
  O[i0] = er;
  O[fs + i0] = F[fs + i0];
  O[2 * fs + i0] = ez;
  O[3 * fs + i0] = br;
  O[4 * fs + i0] = bt;
  O[5 * fs + i0] = bz;
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
  const dim3 grid((n + 31) / 32, (Nz + 7) / 8, nmodes);
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
    destagger_kernel<double><<<grid, 256, 0, st>>>(a);
  } else {
    DestagArgs<float> a;
    fill(a);
    a.in = (const float2*)in;
    a.out = (float2*)out;
    destagger_kernel<float><<<grid, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace fdetd
