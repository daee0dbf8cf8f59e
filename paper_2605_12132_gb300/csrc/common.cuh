// Shared device helpers and plan layout for the FDETD kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdetd {

// ---------------------------------------------------------------- complex helpers
template <typename T> struct cplx;
template <> struct cplx<double> { typedef double2 type; };
template <> struct cplx<float> { typedef float2 type; };

template <typename C> __device__ __forceinline__ C cmake(double r, double i) { C c; c.x = r; c.y = i; return c; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C c; c.x = a.x + b.x; c.y = a.y + b.y; return c; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C c; c.x = a.x - b.x; c.y = a.y - b.y; return c; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C> __device__ __forceinline__ C cmulconj(C a, C b) {  // a * conj(b)
  C c; c.x = a.x * b.x + a.y * b.y; c.y = a.y * b.x - a.x * b.y; return c;
}
// multiply by tau = -i (rotated variables) and by 1/tau = +i
template <typename C> __device__ __forceinline__ C mul_tau(C a) { C c; c.x = a.y; c.y = -a.x; return c; }
template <typename C> __device__ __forceinline__ C mul_itau(C a) { C c; c.x = -a.y; c.y = a.x; return c; }

// ---------------------------------------------------------------- coefficient arithmetic
// FP64 path: coefficients are doubles.  FP32 paths: coefficients are unevaluated
// sums hi + lo of two floats, so that a coefficient rounded once to FP32 does not
// bias every step the same way (a coherent phase error would grow linearly with
// the number of steps); data stay FP32.
struct df { float h, l; };

__device__ __forceinline__ double rmul(double c, double x) { return c * x; }
__device__ __forceinline__ float rmul(df c, float x) { return fmaf(c.h, x, c.l * x); }

template <typename K, typename C> __device__ __forceinline__ C cscale(K c, C x) {
  C r; r.x = rmul(c, x.x); r.y = rmul(c, x.y); return r;
}
// complex coefficient (re, im) times complex data
template <typename K, typename C> __device__ __forceinline__ C ccoef(K re, K im, C x) {
  C r; r.x = rmul(re, x.x) - rmul(im, x.y); r.y = rmul(re, x.y) + rmul(im, x.x); return r;
}

// Phase record per (family, j, q): exp(t M) = I + A1 M + A2 M^2 at t = dt (A) and dt/2 (B).
struct PhaseD { double A1, A2, B1, B2; };
struct PhaseF { df A1, A2; };  // B1, B2 follow from A1, A2 (half-angle identities) in the kernel

// z symbol per q: s+ = i kappa e^{+i th/2} (complex); s- = i kappa e^{-i th/2} = (-Re s+, Im s+)
struct ZSymD { double spr, spi; };
struct ZSymF { df spr, spi; };
// z symbol with kappa^2 = |s+|^2 (FP32-data kernel specialised on Nz), 32 bytes
struct ZSymK { df spr, spi, k2, pad; };

__device__ __forceinline__ unsigned bitrev(unsigned x, int bits) { return __brev(x) >> (32 - bits); }

// 4 x 4 transpose over the four lanes 4g .. 4g+3 of a group (q = lane & 3; every lane of the warp takes part):
// on entry x[c] is element (q, c) of the group's block, on exit element (c, q).  Two butterfly exchanges:
// across lanes q ^ 1 the elements whose column's low bit differs from q's, then across q ^ 2 those whose
// column's high bit differs.
__device__ __forceinline__ void transpose4(float* x, int q) {
  const bool lo = q & 1, hi = q & 2;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = lo ? x[2 * k] : x[2 * k + 1];
    const float r = __shfl_xor_sync(0xffffffffu, send, 1);
    if (lo) x[2 * k] = r;
    else x[2 * k + 1] = r;
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = hi ? x[k] : x[k + 2];
    const float r = __shfl_xor_sync(0xffffffffu, send, 2);
    if (hi) x[k] = r;
    else x[k + 2] = r;
  }
}

}  // namespace fdetd
