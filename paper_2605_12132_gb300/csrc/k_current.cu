// The current pipeline in front of the field step (Sec. 2.5, Eqs. spatialAM_filter_Jr, _Jz; the
// planar current correction of Sec. 3, Eqs. shapesAM_currentRHS2m ... shapesAM_currentJth), in the
// complex mode convention of the field step (d/dtheta -> i sigma m, sigma = -1):
//   1. J_rho deposited on the primary grid -> S_rho^(-, mA) J_rho on the staggered grid of E_rho
//      (Lagrange downstagger of Eq. spatialAM_staggerS); J_theta, J_z copied (F_z = identity);
//   2. delta = rho_xy - Div^+ J_rho - (i sigma m / rho) J_theta on the primary grid (FP64);
//   3. [L_rho^(mS) - m^2 rho^-2] phi = delta per (mode, z row): banded LU factors built on the host in
//      FP64, forward and back substitution in FP64 by one thread per row (the work array is k-major,
//      so a warp's loads at one radius are contiguous);
//   4. J_rho += D^- phi,  J_theta += (i sigma m / rho) phi.
#include "common.cuh"
#include "kernels.h"

namespace fdetd {
namespace {

template <typename T>
struct CurArgs {
  typedef typename cplx<T>::type C;
  const C* J;          // [nm][3][Nz][n] deposited (primary grids)
  const C* rho_xy;     // [nm][Nz][n]
  C* out;              // [nm][3][Nz][n] corrected, on the field step's Yee locations
  double2* work;       // [nm][n][Nz]: delta, then phi
  const double* divp;  // [nm][n][W]
  const double* dm;    // [nm][n][W]
  const double* lo;    // [nm][n][ND]
  const double* up;    // [nm][n][ND + 1]
  double w[32];        // half-point Lagrange weights, nodes t = -ND+1 .. ND
  double dr;
  int Nz, n, ND, nm;
  int m[64];
};

// (i sigma m) x with sigma = -1: (m x.y, -m x.x)
__device__ __forceinline__ double2 tau_m(double m, double2 x) { return make_double2(m * x.y, -m * x.x); }

// 1. downstagger J_rho, copy J_theta and J_z
template <typename T>
__global__ void __launch_bounds__(256) current_stagger_kernel(CurArgs<T> a) {
  typedef typename cplx<T>::type C;
  const int k = blockIdx.x * 32 + (threadIdx.x & 31), z = blockIdx.y * 8 + (threadIdx.x >> 5), md = blockIdx.z;
  const int n = a.n, Nz = a.Nz, N = a.ND;
  if (k >= n || z >= Nz) return;
  const size_t fs = (size_t)Nz * n, row = (size_t)z * n;
  const C* J = a.J + (size_t)md * 3 * fs;
  C* O = a.out + (size_t)md * 3 * fs;
  const int mm = a.m[md];
  const double sign = ((mm - 1 < 0 ? 1 - mm : mm - 1) % 2 == 0) ? 1.0 : -1.0;  // mA extension
  // rho_-,k is the half point above primary node k - 1
  double sx = 0, sy = 0;
  for (int t = -N + 1; t <= N; ++t) {
    int j = k - 1 + t;
    double s = 1.0;
    if (j < 0) {
      j = -1 - j;
      s = sign;
    }
    if (j < n) {
      const C v = J[row + j];
      sx += a.w[t + N - 1] * s * (double)v.x;
      sy += a.w[t + N - 1] * s * (double)v.y;
    }
  }
  O[row + k] = cmake<C>((T)sx, (T)sy);
  O[fs + row + k] = J[fs + row + k];
  O[2 * fs + row + k] = J[2 * fs + row + k];
}

// 2. planar divergence error (FP64), stored k-major for the row solves
template <typename T>
__global__ void __launch_bounds__(256) current_delta_kernel(CurArgs<T> a) {
  typedef typename cplx<T>::type C;
  const int k = blockIdx.x * 32 + (threadIdx.x & 31), z = blockIdx.y * 8 + (threadIdx.x >> 5), md = blockIdx.z;
  const int n = a.n, Nz = a.Nz, N = a.ND, W = 2 * N + 1;
  if (k >= n || z >= Nz) return;
  const size_t fs = (size_t)Nz * n, row = (size_t)z * n;
  const C* O = a.out + (size_t)md * 3 * fs;
  const double* b = a.divp + ((size_t)md * n + k) * W;
  double dx = 0, dy = 0;
  for (int t = 0; t < W; ++t) {
    const int j = k - N + t;
    if (j < 1 || j >= n) continue;  // column 0 carries rho_-,0 = 0
    const C v = O[row + j];
    dx += b[t] * (double)v.x;
    dy += b[t] * (double)v.y;
  }
  const C jt = O[fs + row + k];
  const double2 tj = tau_m((double)a.m[md], make_double2((double)jt.x, (double)jt.y));
  const double ri = 1.0 / ((k + 0.5) * a.dr);
  const C r = a.rho_xy[(size_t)md * fs + row + k];
  a.work[((size_t)md * n + k) * Nz + z] = make_double2((double)r.x - dx - tj.x * ri, (double)r.y - dy - tj.y * ri);
}

// 3. banded LU solve in place, one thread per (mode, z row)
__global__ void __launch_bounds__(128) current_solve_kernel(double2* work, const double* lo, const double* up, int Nz,
                                                            int n, int ND, int nm) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x, md = blockIdx.y;
  if (z >= Nz || md >= nm) return;
  double2* x = work + (size_t)md * n * Nz + z;  // element k at x[k * Nz]
  const double* L = lo + (size_t)md * n * ND;
  const double* U = up + (size_t)md * n * (ND + 1);
  for (int k = 0; k < n; ++k) {  // y = L^-1 delta (unit lower)
    double2 s = x[(size_t)k * Nz];
    for (int d = 1; d <= ND && d <= k; ++d) {
      const double l = L[(size_t)k * ND + d - 1];
      const double2 y = x[(size_t)(k - d) * Nz];
      s.x -= l * y.x;
      s.y -= l * y.y;
    }
    x[(size_t)k * Nz] = s;
  }
  for (int k = n - 1; k >= 0; --k) {  // phi = U^-1 y
    double2 s = x[(size_t)k * Nz];
    for (int d = 1; d <= ND && k + d < n; ++d) {
      const double u = U[(size_t)k * (ND + 1) + d];
      const double2 y = x[(size_t)(k + d) * Nz];
      s.x -= u * y.x;
      s.y -= u * y.y;
    }
    const double piv = U[(size_t)k * (ND + 1)];
    x[(size_t)k * Nz] = make_double2(s.x / piv, s.y / piv);
  }
}

// 4. J_rho += D^- phi, J_theta += (i sigma m / rho) phi
template <typename T>
__global__ void __launch_bounds__(256) current_correct_kernel(CurArgs<T> a) {
  typedef typename cplx<T>::type C;
  const int k = blockIdx.x * 32 + (threadIdx.x & 31), z = blockIdx.y * 8 + (threadIdx.x >> 5), md = blockIdx.z;
  const int n = a.n, Nz = a.Nz, N = a.ND, W = 2 * N + 1;
  if (k >= n || z >= Nz) return;
  const size_t fs = (size_t)Nz * n, row = (size_t)z * n;
  C* O = a.out + (size_t)md * 3 * fs;
  const double2* phi = a.work + (size_t)md * n * Nz + z;
  const double* b = a.dm + ((size_t)md * n + k) * W;
  double gx = 0, gy = 0;
  for (int t = 0; t < W; ++t) {
    const int j = k - N + t;
    if (j < 0 || j >= n) continue;
    const double2 p = phi[(size_t)j * Nz];
    gx += b[t] * p.x;
    gy += b[t] * p.y;
  }
  const C jr = O[row + k];
  O[row + k] = cmake<C>((T)((double)jr.x + gx), (T)((double)jr.y + gy));
  const double2 tp = tau_m((double)a.m[md], phi[(size_t)k * Nz]);
  const double ri = 1.0 / ((k + 0.5) * a.dr);
  const C jt = O[fs + row + k];
  O[fs + row + k] = cmake<C>((T)((double)jt.x + tp.x * ri), (T)((double)jt.y + tp.y * ri));
}

template <typename T>
cudaError_t run_current(const CurParams& p, cudaStream_t st) {
  CurArgs<T> a;
  a.J = (const typename cplx<T>::type*)p.J;
  a.rho_xy = (const typename cplx<T>::type*)p.rho_xy;
  a.out = (typename cplx<T>::type*)p.out;
  a.work = (double2*)p.work;
  a.divp = p.divp;
  a.dm = p.dm;
  a.lo = p.lo;
  a.up = p.up;
  a.dr = p.dr;
  a.Nz = p.Nz;
  a.n = p.n;
  a.ND = p.ND;
  a.nm = p.nm;
  for (int i = 0; i < 2 * p.ND; ++i) a.w[i] = p.w[i];
  for (int i = 0; i < p.nm; ++i) a.m[i] = p.m[i];
  const dim3 g1((p.n + 31) / 32, (p.Nz + 7) / 8, p.nm);
  current_stagger_kernel<T><<<g1, 256, 0, st>>>(a);
  current_delta_kernel<T><<<g1, 256, 0, st>>>(a);
  current_solve_kernel<<<dim3((p.Nz + 127) / 128, p.nm), 128, 0, st>>>(a.work, p.lo, p.up, p.Nz, p.n, p.ND, p.nm);
  current_correct_kernel<T><<<g1, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_current(const CurParams& p, bool fp64, cudaStream_t st) {
  if (p.ND < 1 || p.ND > 16 || p.nm < 1 || p.nm > 64) return cudaErrorInvalidValue;
  return fp64 ? run_current<double>(p, st) : run_current<float>(p, st);
}

}  // namespace fdetd
