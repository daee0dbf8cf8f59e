// CUDA-core (FP64 / FP32) radial projection and back-projection.
//
// Projection (per mode, per z row, per group):
//   coef[c][j][z] = sum_{field block f, r} P[c-block j][f-block r] * X_f[z][r]
// Back-projection:
//   X_f[z][r]     = sum_{c block, j} Q[f-block r][c-block j] * coef[c][j][z]
// P and Q are real, X and coef complex; the rotated field components
// (tau Etheta, tau Br, tau Bz, tau Jtheta, tau = -i) are formed on load and undone
// on store, which keeps both matrices real.  Only the nonzero 3x3 block pattern
// of P and Q is traversed:
//   forward E/J: e <- Ez; a, c <- (Er, Et)      forward B: b, d <- (Bt, Br); f <- Bz
//   backward E:  Er, Et <- (a, c); Ez <- e      backward B: Bt, Br <- (b, d); Bz <- f
#include "common.cuh"
#include "kernels.h"

namespace fdetd {

namespace {

constexpr int TILE = 64, KT = 16;

// field index / rotation of input block ib for group g (0 = E, 1 = B, 2 = J)
__device__ __forceinline__ int fwd_field(int g, int ib) {
  return g == 1 ? (ib == 0 ? 4 : (ib == 1 ? 3 : 5)) : ib;
}
__device__ __forceinline__ bool fwd_rot(int g, int ib) { return g == 1 ? (ib >= 1) : (ib == 1); }

__device__ __forceinline__ int fwd_blocks(int g, int ob, int* list) {
  const bool b = (g == 1);
  if ((!b && ob == 0) || (b && ob == 2)) {
    list[0] = 2;
    return 1;
  }
  list[0] = 0;
  list[1] = 1;
  return 2;
}
__device__ __forceinline__ int bwd_blocks(int g, int fb, int* list) {
  if (fb == 2) {
    list[0] = (g == 0) ? 0 : 2;
    return 1;
  }
  if (g == 0) {
    list[0] = 1;
    list[1] = 2;
  } else {
    list[0] = 0;
    list[1] = 1;
  }
  return 2;
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(256) project_simt(ProjArgs a) {
  typedef typename cplx<T>::type C;
  __shared__ T Ps[KT][TILE + 1];
  __shared__ C Xs[KT][TILE + 1];
  const int n = a.n, Nz = a.Nz, N3 = 3 * n;
  const int z0 = blockIdx.x * TILE, j0 = blockIdx.y * TILE;
  const int ngroups = a.J ? 3 : 2;
  const int md = blockIdx.z / (3 * ngroups), rem = blockIdx.z % (3 * ngroups);
  const int g = rem / 3, ob = rem % 3;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const T* Pm = reinterpret_cast<const T*>(a.P) + ((size_t)(md * 2 + (g == 1 ? 1 : 0)) * N3 + ob * n) * N3;
  const C* X = g == 2 ? reinterpret_cast<const C*>(a.J) + (size_t)md * 3 * Nz * n
                      : reinterpret_cast<const C*>(a.fields) + (size_t)md * 6 * Nz * n;
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[i][k] = cmake<C>(0, 0);
  int blist[2];
  const int nb = fwd_blocks(g, ob, blist);
  for (int bi = 0; bi < nb; ++bi) {
    const int ib = blist[bi];
    const C* Xf = X + (size_t)fwd_field(g, ib) * Nz * n;
    const bool rot = fwd_rot(g, ib);
    for (int r0 = 0; r0 < n; r0 += KT) {
      for (int t = threadIdx.x; t < TILE * KT; t += blockDim.x) {
        const int jj = t / KT, kk = t % KT;
        const int j = j0 + jj, r = r0 + kk;
        Ps[kk][jj] = (j < n && r < n) ? Pm[(size_t)j * N3 + ib * n + r] : (T)0;
        const int zz = jj;
        C v = cmake<C>(0, 0);
        if (r < n) v = Xf[(size_t)(z0 + zz) * n + r];
        Xs[kk][zz] = rot ? mul_tau(v) : v;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < KT; ++kk) {
        T p[4];
        C x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) p[k] = Ps[kk][ty + 16 * k];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = Xs[kk][tx + 16 * i];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc[i][k].x += p[k] * x[i].x;
            acc[i][k].y += p[k] * x[i].y;
          }
      }
      __syncthreads();
    }
  }
  const int cidx = g * 3 + ob;
  C* out = reinterpret_cast<C*>(a.coef) + (size_t)(md * 9 + cidx) * n * Nz;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = j0 + ty + 16 * k;
    if (j >= n) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) out[(size_t)j * Nz + z0 + tx + 16 * i] = acc[i][k];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) backproject_simt(BackArgs a) {
  typedef typename cplx<T>::type C;
  __shared__ T Qs[KT][TILE + 1];
  __shared__ C Cs[KT][TILE + 1];
  const int n = a.n, Nz = a.Nz, N3 = 3 * n;
  const int z0 = blockIdx.x * TILE, r0 = blockIdx.y * TILE;
  const int md = blockIdx.z / 6, rem = blockIdx.z % 6;
  const int g = rem / 3, fb = rem % 3;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const T* Qm = reinterpret_cast<const T*>(a.Q) + ((size_t)(md * 2 + g) * N3 + fb * n) * N3;
  const C* coef = reinterpret_cast<const C*>(a.coef) + (size_t)md * 9 * n * Nz;
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[i][k] = cmake<C>(0, 0);
  int blist[2];
  const int nb = bwd_blocks(g, fb, blist);
  for (int bi = 0; bi < nb; ++bi) {
    const int cb = blist[bi];
    const C* Cb = coef + (size_t)(g * 3 + cb) * n * Nz;
    for (int jb = 0; jb < n; jb += KT) {
      for (int t = threadIdx.x; t < TILE * KT; t += blockDim.x) {
        const int rr = t / KT, kk = t % KT;
        const int r = r0 + rr, j = jb + kk;
        Qs[kk][rr] = (r < n && j < n) ? Qm[(size_t)r * N3 + cb * n + j] : (T)0;
        const int kk2 = t / TILE, zz = t % TILE;
        const int j2 = jb + kk2;
        Cs[kk2][zz] = (j2 < n) ? Cb[(size_t)j2 * Nz + z0 + zz] : cmake<C>(0, 0);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < KT; ++kk) {
        T q[4];
        C c[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = Qs[kk][tx + 16 * i];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = Cs[kk][ty + 16 * k];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc[i][k].x += q[i] * c[k].x;
            acc[i][k].y += q[i] * c[k].y;
          }
      }
      __syncthreads();
    }
  }
  const int field = g == 0 ? fb : (fb == 0 ? 4 : (fb == 1 ? 3 : 5));
  const bool rot = (g == 0) ? (fb == 1) : (fb >= 1);
  C* out = reinterpret_cast<C*>(a.fields) + ((size_t)md * 6 + field) * Nz * n;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int z = z0 + ty + 16 * k;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + tx + 16 * i;
      if (r < n) out[(size_t)z * n + r] = rot ? mul_itau(acc[i][k]) : acc[i][k];
    }
  }
}

cudaError_t launch_project_simt(const ProjArgs& a, int nmodes, int precision, cudaStream_t st) {
  const int ngroups = a.J ? 3 : 2;
  dim3 grid(a.Nz / TILE, (a.n + TILE - 1) / TILE, nmodes * ngroups * 3);
  if (precision == 0)
    project_simt<double><<<grid, 256, 0, st>>>(a);
  else
    project_simt<float><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_backproject_simt(const BackArgs& a, int nmodes, int precision, cudaStream_t st) {
  dim3 grid(a.Nz / TILE, (a.n + TILE - 1) / TILE, nmodes * 6);
  if (precision == 0)
    backproject_simt<double><<<grid, 256, 0, st>>>(a);
  else
    backproject_simt<float><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fdetd
