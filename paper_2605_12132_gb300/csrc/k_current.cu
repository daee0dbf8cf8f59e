// The current pipeline in front of the field step (Sec. 2.5, Eqs. spatialAM_filter_Jr, _Jz; the
// planar current correction of Sec. 3, Eqs. shapesAM_currentRHS2m ... shapesAM_currentJth), in the
// complex mode convention of the field step (d/dtheta -> i sigma m, sigma = -1):
//   1. J_rho deposited on the primary grid -> S_rho^(-, mA) J_rho on the staggered grid of E_rho
//      (Lagrange downstagger of Eq. spatialAM_staggerS); J_theta, J_z copied (F_z = identity);
//   2. delta = rho_xy - Div^+ J_rho - (i sigma m / rho) J_theta on the primary grid;
//   3. [L_rho^(mS) - m^2 rho^-2] phi = delta per (mode, z row) by the banded LU factors built on the host;
//   4. J_rho += D^- phi,  J_theta += (i sigma m / rho) phi.
// Every step is radial, so one CTA carries R z rows of one mode through all four with delta / phi
// in shared memory.  Steps 2-4 need more than FP32: a rounding error of the divergence is amplified
// by the inverse Laplacian (by about sqrt(Nr) for noise, by Nr for a smooth error), and the gradient
// of a smooth phi cancels.  FP64 is slow on this part, so FP32 data use double-float arithmetic
// (value = h + l, two floats, ~46-bit significand; coefficients stored as float pairs by the host),
// and FP64 data use FP64.  The downstagger is an interpolation whose rounding the correction projects
// out rather than amplifies; it runs in the data type.
//
// The solve runs on one warp per 16 rows: lane (row, re/im component) carries a real banded
// substitution, specialised by the band width, with the band rows prefetched across the warp.  The stencil phases run one thread per radius over the CTA's rows,
// from rows staged in shared memory.
#include "common.cuh"
#include "kernels.h"

namespace fdetd {
namespace {

// ---------------------------------------------------------------- double-float arithmetic
struct dfl {
  float h, l;
};

// a += p + e, with p + a.h summed exactly (two-sum) and the error folded into a.l
__device__ __forceinline__ void acc_add(dfl& a, float p, float e) {
  const float s = a.h + p, v = s - a.h;
  a.l += ((a.h - (s - v)) + (p - v)) + e;
  a.h = s;
}
// a += c x for an exact float x: p = c.h x rounded, its error by FMA, plus c.l x
__device__ __forceinline__ void mac(dfl& a, float2 c, float x) {
  const float p = c.x * x;
  acc_add(a, p, fmaf(c.y, x, fmaf(c.x, x, -p)));
}
__device__ __forceinline__ void mac(dfl& a, float2 c, dfl x) {
  const float p = c.x * x.h;
  acc_add(a, p, fmaf(c.y, x.h, fmaf(c.x, x.l, fmaf(c.x, x.h, -p))));
}
__device__ __forceinline__ dfl norm(dfl a) {
  const float s = a.h + a.l;
  dfl r;
  r.h = s;
  r.l = a.l - (s - a.h);
  return r;
}
__device__ __forceinline__ dfl mul(dfl a, float2 c) {
  const float p = a.h * c.x;
  dfl r;
  r.h = p;
  r.l = fmaf(a.l, c.x, fmaf(a.h, c.y, fmaf(a.h, c.x, -p)));
  return norm(r);
}
__device__ __forceinline__ float2 neg(float2 c) { return make_float2(-c.x, -c.y); }
__device__ __forceinline__ void lift(dfl& a, float x) {
  a.h = x;
  a.l = 0.f;
}
__device__ __forceinline__ float lower(dfl a) { return a.h + a.l; }

__device__ __forceinline__ void mac(double& a, double c, double x) { a = fma(c, x, a); }
__device__ __forceinline__ double norm(double a) { return a; }
__device__ __forceinline__ double mul(double a, double c) { return a * c; }
__device__ __forceinline__ double neg(double c) { return -c; }
__device__ __forceinline__ void lift(double& a, double x) { a = x; }
__device__ __forceinline__ double lower(double a) { return a; }

template <typename T> struct CurNum;
template <> struct CurNum<float> {
  typedef dfl A;     // accumulator / shared-memory value
  typedef float2 K;  // coefficient (h, l)
};
template <> struct CurNum<double> {
  typedef double A;
  typedef double K;
};

constexpr int MAX_ND = 16;  // half the largest finite-difference order

template <typename T>
struct CurArgs {
  typedef typename cplx<T>::type C;
  typedef typename CurNum<T>::K K;
  const C* J;       // [nm][3][Nz][n] deposited (primary grids)
  const C* rho_xy;  // [nm][Nz][n]
  C* out;           // [nm][3][Nz][n] corrected, on the field step's Yee locations
  const K* divp;    // [nm][W][n]: -Div^+ band, tap t of row k at t * n + k
  const K* dm;      // [nm][W][n]: D^- band
  const K* lo;      // [nm][n][ND]: -L(k, k - d) at k * ND + d - 1 (unit lower factor)
  const K* up;      // [nm][n][ND]: -U(k, k + d) at k * ND + d - 1
  const K* ipiv;    // [nm][n]: 1 / U(k, k)
  const K* mri;     // [nm][n]: m / rho_k
  T w[32];          // half-point Lagrange weights, nodes t = -ND+1 .. ND
  int Nz, n, ND, R;
  int stagger_only;      // 1: step 1 alone (J_rho downstaggered, J_theta and J_z copied), no correction
  signed char sign[64];  // mA extension sign per mode
};

__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ float2 shfl(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ void kzero(float2& c) { c = make_float2(0.f, 0.f); }
__device__ __forceinline__ void kzero(double& c) { c = 0.0; }

// Banded forward and back substitution of one real system of length n at x[0], x[2], ... (shared
// memory), ND sub- and super-diagonals, run by a whole warp (lanes with live == false follow along
// without touching x).  The last ND values sit in registers and the terms are added farthest first, so
// only the last one waits for the value just computed.  The band rows are uniform across the warp:
// lane l loads element l % ND of row k0 + l / ND for a group of G = 32 / ND rows, two groups ahead,
// and each step takes its coefficients from the lanes by shuffles, so no step waits on memory.
template <int ND, typename A, typename K>
__device__ __forceinline__ void solve_rows(A* x, bool live, int n, const K* L, const K* U, const K* ip) {
  constexpr int G = 32 / ND;
  const int lane = threadIdx.x & 31, gr = lane / ND, gd = lane - gr * ND;
  auto fetch = [&](const K* B, int row) {  // this lane's element of row `row` (zero outside)
    K c;
    kzero(c);
    if (gr < G && row >= 0 && row < n) c = B[(size_t)row * ND + gd];
    return c;
  };
  A win[ND];  // win[d - 1] = the value d places back
#pragma unroll
  for (int d = 0; d < ND; ++d) lift(win[d], 0.f);
  K cur = fetch(L, gr), nxt = fetch(L, G + gr);
  for (int k0 = 0; k0 < n; k0 += G) {
    const K nn = fetch(L, k0 + 2 * G + gr);
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int k = k0 + i;
      if (k < n) {  // uniform
        A s;
        lift(s, 0.f);
        if (live) s = x[2 * k];
#pragma unroll
        for (int d = ND; d >= 1; --d) mac(s, shfl(cur, i * ND + d - 1), win[d - 1]);
        s = norm(s);
        if (live) x[2 * k] = s;
#pragma unroll
        for (int d = ND - 1; d >= 1; --d) win[d] = win[d - 1];
        win[0] = s;
      }
    }
    cur = nxt;
    nxt = nn;
  }
  // back substitution from row n - 1 down: group g holds rows n - 1 - (g G + i)
#pragma unroll
  for (int d = 0; d < ND; ++d) lift(win[d], 0.f);
  auto fetchU = [&](int g) {
    K c;
    kzero(c);
    const int row = n - 1 - (g * G + gr);
    if (gr < G && row >= 0) c = U[(size_t)row * ND + gd];
    return c;
  };
  auto fetchP = [&](int g) {  // 1 / U(k, k) for the group's rows, on lanes 0 .. G-1
    K c;
    kzero(c);
    const int row = n - 1 - (g * G + lane);
    if (lane < G && row >= 0) c = ip[row];
    return c;
  };
  cur = fetchU(0);
  nxt = fetchU(1);
  K pc = fetchP(0), pnx = fetchP(1);
  for (int g = 0; g * G < n; ++g) {
    const K nn = fetchU(g + 2), pnn = fetchP(g + 2);
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int k = n - 1 - (g * G + i);
      if (k >= 0) {  // uniform
        A s;
        lift(s, 0.f);
        if (live) s = x[2 * k];
#pragma unroll
        for (int d = ND; d >= 1; --d) mac(s, shfl(cur, i * ND + d - 1), win[d - 1]);
        s = mul(s, shfl(pc, i));
        if (live) x[2 * k] = s;
#pragma unroll
        for (int d = ND - 1; d >= 1; --d) win[d] = win[d - 1];
        win[0] = s;
      }
    }
    cur = nxt;
    nxt = nn;
    pc = pnx;
    pnx = pnn;
  }
}

// One CTA per (R z rows, mode), 256 threads.  Shared memory: js[R][n] holds the staggered J_rho rows
// (data type); ph[R][n + 1][2] holds first the deposited J_rho rows (staged for the stencil), then
// delta, then phi.  In the stencil phases a thread owns one radius k and walks the R rows, so each
// band coefficient of row k is read once per CTA.
template <typename T>
__global__ void __launch_bounds__(256) current_kernel(CurArgs<T> a) {
  typedef typename cplx<T>::type C;
  typedef typename CurNum<T>::A A;
  typedef typename CurNum<T>::K K;
  constexpr int RM = 16;  // rows per CTA at most (one solving warp: row x component)
  extern __shared__ __align__(16) unsigned char csm[];
  const int n = a.n, Nz = a.Nz, N = a.ND, W = 2 * N + 1, P = n + 1;
  const int z0 = blockIdx.x * a.R, md = blockIdx.y;
  const int rows = min(a.R, Nz - z0);
  C* js = reinterpret_cast<C*>(csm);
  A* ph = reinterpret_cast<A*>(csm + (size_t)a.R * n * sizeof(C));
  C* raw = reinterpret_cast<C*>(ph);
  const size_t fs = (size_t)Nz * n, zq = (size_t)z0 * n;
  const C* J = a.J + (size_t)md * 3 * fs;
  const C* rho = a.stagger_only ? nullptr : a.rho_xy + (size_t)md * fs;
  C* O = a.out + (size_t)md * 3 * fs;
  const T sgn = (T)a.sign[md];
  const K* mr = a.mri + (size_t)md * n;

  // 0. stage the deposited J_rho rows; copy J_theta, J_z
  for (int i = threadIdx.x; i < rows * n; i += blockDim.x) {
    raw[i] = J[zq + i];
    O[fs + zq + i] = J[fs + zq + i];
    O[2 * fs + zq + i] = J[2 * fs + zq + i];
  }
  __syncthreads();

  // 1. downstagger J_rho (rho_-,k is the half point above primary node k - 1)
  for (int i = threadIdx.x; i < rows * n; i += blockDim.x) {
    const int r = i / n, k = i - r * n;
    const C* row = raw + r * n;
    T sx = 0, sy = 0;
    for (int t = -N + 1; t <= N; ++t) {
      int j = k - 1 + t;
      T ws = a.w[t + N - 1];
      if (j < 0) {
        j = -1 - j;
        ws *= sgn;
      }
      if (j < n) {
        const C v = row[j];
        sx = fmad(ws, v.x, sx);
        sy = fmad(ws, v.y, sy);
      }
    }
    const C v = cmake<C>(sx, sy);
    js[i] = v;
    O[zq + i] = v;
  }
  if (a.stagger_only) return;  // uniform over the block: nothing below runs
  __syncthreads();

  // 2. delta = rho_xy - Div^+ J_rho - (i sigma m / rho) J_theta, thread per radius over the rows
  const K* bp = a.divp + (size_t)md * W * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    A dx[RM], dy[RM];
#pragma unroll
    for (int r = 0; r < RM; ++r)
      if (r < rows) {
        const C rv = rho[zq + (size_t)r * n + k];
        lift(dx[r], rv.x);
        lift(dy[r], rv.y);
      }
    for (int t = 0; t < W; ++t) {
      const int j = k - N + t;
      if (j < 0 || j >= n) continue;
      const K b = bp[(size_t)t * n + k];
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < rows) {
          const C v = js[r * n + j];
          mac(dx[r], b, v.x);
          mac(dy[r], b, v.y);
        }
    }
    const K c = mr[k];  // (i sigma m) x / rho = (m x.y, -m x.x) / rho
#pragma unroll
    for (int r = 0; r < RM; ++r)
      if (r < rows) {
        const C jt = O[fs + zq + (size_t)r * n + k];
        mac(dx[r], neg(c), jt.y);
        mac(dy[r], c, jt.x);
        A* x = ph + ((size_t)r * P + k) * 2;
        x[0] = norm(dx[r]);
        x[1] = norm(dy[r]);
      }
  }
  __syncthreads();

  // 3. forward (unit lower) and back (upper) substitution, one real system per lane of warp 0
  if (threadIdx.x < 32) {
    const bool live = (int)threadIdx.x < 2 * rows;
    A* x = ph + (size_t)(live ? threadIdx.x >> 1 : 0) * P * 2 + (threadIdx.x & 1);  // element k at x[2 k]
    const K* L = a.lo + (size_t)md * n * N;
    const K* U = a.up + (size_t)md * n * N;
    const K* ip = a.ipiv + (size_t)md * n;
    switch (N) {
#define FDETD_SOLVE_CASE(ND) \
  case ND:                   \
    solve_rows<ND>(x, live, n, L, U, ip); \
    break;
      FDETD_SOLVE_CASE(1) FDETD_SOLVE_CASE(2) FDETD_SOLVE_CASE(3) FDETD_SOLVE_CASE(4)
      FDETD_SOLVE_CASE(5) FDETD_SOLVE_CASE(6) FDETD_SOLVE_CASE(7) FDETD_SOLVE_CASE(8)
      FDETD_SOLVE_CASE(9) FDETD_SOLVE_CASE(10) FDETD_SOLVE_CASE(11) FDETD_SOLVE_CASE(12)
      FDETD_SOLVE_CASE(13) FDETD_SOLVE_CASE(14) FDETD_SOLVE_CASE(15) FDETD_SOLVE_CASE(16)
#undef FDETD_SOLVE_CASE
      default:
        break;
    }
  }
  __syncthreads();

  // 4. J_rho += D^- phi, J_theta += (i sigma m / rho) phi, thread per radius over the rows
  const K* gm = a.dm + (size_t)md * W * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    A gx[RM], gy[RM];
#pragma unroll
    for (int r = 0; r < RM; ++r)
      if (r < rows) {
        const C v = js[r * n + k];
        lift(gx[r], v.x);
        lift(gy[r], v.y);
      }
    for (int t = 0; t < W; ++t) {
      const int j = k - N + t;
      if (j < 0 || j >= n) continue;
      const K b = gm[(size_t)t * n + k];
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < rows) {
          const A* xr = ph + ((size_t)r * P + j) * 2;
          mac(gx[r], b, xr[0]);
          mac(gy[r], b, xr[1]);
        }
    }
    const K c = mr[k];
#pragma unroll
    for (int r = 0; r < RM; ++r)
      if (r < rows) {
        const size_t q = zq + (size_t)r * n + k;
        const A* xr = ph + ((size_t)r * P + k) * 2;
        const C jt = O[fs + q];
        A tx, ty;
        lift(tx, jt.x);
        lift(ty, jt.y);
        mac(tx, c, xr[1]);
        mac(ty, neg(c), xr[0]);
        O[q] = cmake<C>(lower(gx[r]), lower(gy[r]));
        O[fs + q] = cmake<C>(lower(tx), lower(ty));
      }
  }
}

template <typename T>
cudaError_t run_current(const CurParams& p, cudaStream_t st) {
  typedef typename CurNum<T>::K K;
  CurArgs<T> a;
  a.J = (const typename cplx<T>::type*)p.J;
  a.rho_xy = (const typename cplx<T>::type*)p.rho_xy;
  a.out = (typename cplx<T>::type*)p.out;
  const K* base = (const K*)p.bands;
  const size_t nm = p.nm, n = p.n, W = 2 * p.ND + 1;
  a.stagger_only = p.stagger_only;
  a.divp = a.dm = a.lo = a.up = a.ipiv = a.mri = nullptr;
  if (base) {  // the correction's tables (absent in the stagger-only form)
    a.divp = base;
    a.dm = a.divp + nm * W * n;
    a.lo = a.dm + nm * W * n;
    a.up = a.lo + nm * n * p.ND;
    a.ipiv = a.up + nm * n * p.ND;
    a.mri = a.ipiv + nm * n;
  }
  a.Nz = p.Nz;
  a.n = p.n;
  a.ND = p.ND;
  for (int i = 0; i < 2 * p.ND; ++i) a.w[i] = (T)p.w[i];
  for (int i = 0; i < p.nm; ++i) {
    const int m = p.m[i];
    a.sign[i] = ((m - 1 < 0 ? 1 - m : m - 1) % 2 == 0) ? 1 : -1;
  }
  // 16 rows fill the solving warp; fewer when the rows would not leave room for two CTAs per SM
  int R = 16;
  const size_t row_bytes =
      (size_t)(p.n + 1) * 2 * sizeof(typename CurNum<T>::A) + (size_t)p.n * sizeof(typename cplx<T>::type);
  while (R > 1 && (size_t)R * row_bytes > 110 * 1024) R >>= 1;
  if ((size_t)R * row_bytes > 227 * 1024) return cudaErrorInvalidValue;
  a.R = R;
  const size_t smem = (size_t)R * row_bytes;
  auto k = current_kernel<T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<dim3((p.Nz + R - 1) / R, p.nm), 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_current(const CurParams& p, bool fp64, cudaStream_t st) {
  if (p.ND < 1 || p.ND > MAX_ND || p.nm < 1 || p.nm > 64) return cudaErrorInvalidValue;
  if (!p.stagger_only && (!p.bands || !p.rho_xy)) return cudaErrorInvalidValue;
  return fp64 ? run_current<double>(p, st) : run_current<float>(p, st);
}

}  // namespace fdetd
