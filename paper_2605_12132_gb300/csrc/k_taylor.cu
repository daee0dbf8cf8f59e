// The paper's own time stepper on the GPU: the midpoint step of Eq. maxwellAM_solution2 with both
// exponentials replaced by N-term Taylor polynomials of the real-space operator H (Sec. 2.5
// summary), applied by banded stencils - no radial transform:
//   x <- T_N(h H)^S x - dt T_N(h' H)^S' J_state,  h = dt / S,  h' = (dt / 2) / S',  S' = max(1, S / 2),
// T_N(A) = sum_{n <= N} A^n / n!.  One kernel launch per Taylor term evaluates
//   out = (h / n) H(in),  acc_out = acc_in + out  [- dt src on the last term of a step],
// with H of Eqs. spatialAM_maxwell_Er ... _Bz: periodic staggered z differences and banded radial
// operators (parity folds and the B_z axis value of Sec. 2.4 included, see taylor_bands).
// FP32 state (complex64) and arithmetic.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fdetd.h"
#include "kernels.h"
#include "plan_host.h"

namespace fdetd {
namespace {

constexpr int kMaxModes = 64;

struct TaylorArgs {
  const float2* in;     // [nm][6][Nz][n]: the previous term (or the state for the first term)
  float2* out;          // the new term (null on the last term)
  const float2* accin;  // running sum in
  float2* accout;       // running sum out (may equal accin)
  const float2* sub;    // optional: accout -= sub_scale * sub
  float sub_scale;
  const float* bands;   // [nm][4][n][W]
  const float* rho_inv;   // [n] 1 / rho_k
  const float* rhom_inv;  // [n] 1 / rho_-,k (k >= 1; 0 at the axis)
  float cz[17];         // staggered z coefficients c_t / dz at [t], t = 1..ND
  float scale;          // h / n
  int Nz, n, ND, nm;
  int m[kMaxModes];
};

__device__ __forceinline__ float2 ld(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 fma2(float w, float2 v, float2 acc) {
  return make_float2(fmaf(w, v.x, acc.x), fmaf(w, v.y, acc.y));
}
// tau m x with tau = -i (mode sign sigma = -1): (m x.y, -m x.x)
__device__ __forceinline__ float2 taum(float m, float2 x) { return make_float2(m * x.y, -m * x.x); }

__global__ void __launch_bounds__(256) taylor_term_kernel(TaylorArgs a) {
  const int k = blockIdx.x * 32 + (threadIdx.x & 31);
  const int z = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int md = blockIdx.z;
  const int n = a.n, Nz = a.Nz, ND = a.ND, W = 2 * ND + 1;
  if (k >= n || z >= Nz) return;
  const size_t fs = (size_t)Nz * n;  // field stride
  const float2* F = a.in + (size_t)md * 6 * fs;
  const float2 *Er = F, *Et = F + fs, *Ez = F + 2 * fs, *Br = F + 3 * fs, *Bt = F + 4 * fs, *Bz = F + 5 * fs;
  const float m = (float)a.m[md];
  // z differences at (z, k): D^+ g_i = sum c_t (g_{i+t} - g_{i-t+1}), D^- f_i = sum c_t (f_{i+t-1} - f_{i-t})
  float2 dpBt = make_float2(0.f, 0.f), dpBr = dpBt, dmEt = dpBt, dmEr = dpBt;
  for (int t = 1; t <= ND; ++t) {
    int zp = z + t, zq = z - t + 1, zr = z + t - 1, zs = z - t;
    if (zp >= Nz) zp -= Nz;
    if (zq < 0) zq += Nz;
    if (zr >= Nz) zr -= Nz;
    if (zs < 0) zs += Nz;
    const float c = a.cz[t];
    const size_t ip = (size_t)zp * n + k, iq = (size_t)zq * n + k, ir = (size_t)zr * n + k, is = (size_t)zs * n + k;
    float2 u = ld(Bt + ip), v = ld(Bt + iq);
    dpBt = fma2(c, make_float2(u.x - v.x, u.y - v.y), dpBt);
    u = ld(Br + ip), v = ld(Br + iq);
    dpBr = fma2(c, make_float2(u.x - v.x, u.y - v.y), dpBr);
    u = ld(Et + ir), v = ld(Et + is);
    dmEt = fma2(c, make_float2(u.x - v.x, u.y - v.y), dmEt);
    u = ld(Er + ir), v = ld(Er + is);
    dmEr = fma2(c, make_float2(u.x - v.x, u.y - v.y), dmEr);
  }
  // radial bands at row k over columns k - ND .. k + ND; staggered-grid operands skip the axis slot
  const float* b0 = a.bands + (((size_t)md * 4 + 0) * n + k) * W;
  const float* b1 = b0 + (size_t)n * W;
  const float* b2 = b1 + (size_t)n * W;
  const float* b3 = b2 + (size_t)n * W;
  float2 r0 = make_float2(0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
  const size_t row = (size_t)z * n;
  for (int t = 0; t < W; ++t) {
    const int j = k - ND + t;
    if (j < 0 || j >= n) continue;
    if (j >= 1) {
      r0 = fma2(__ldg(b0 + t), ld(Bz + row + j), r0);
      r1 = fma2(__ldg(b1 + t), ld(Bt + row + j), r1);
    }
    if (k >= 1) {
      r2 = fma2(__ldg(b2 + t), ld(Ez + row + j), r2);
      r3 = fma2(__ldg(b3 + t), ld(Et + row + j), r3);
    }
  }
  const size_t i0 = row + k;
  const float ri = a.rho_inv[k], rmi = a.rhom_inv[k];
  float2 h[6];
  if (k >= 1) {
    const float2 tb = taum(m, ld(Bz + i0));
    h[0] = make_float2(-dpBt.x + tb.x * rmi, -dpBt.y + tb.y * rmi);
    h[4] = make_float2(-dmEr.x + r2.x, -dmEr.y + r2.y);
    const float2 te = taum(m, ld(Er + i0));
    h[5] = make_float2(te.x * rmi - r3.x, te.y * rmi - r3.y);
  } else {
    h[0] = h[4] = h[5] = make_float2(0.f, 0.f);
  }
  h[1] = make_float2(dpBr.x - r0.x, dpBr.y - r0.y);
  const float2 tbr = taum(m, ld(Br + i0));
  h[2] = make_float2(-tbr.x * ri + r1.x, -tbr.y * ri + r1.y);
  const float2 tez = taum(m, ld(Ez + i0));
  h[3] = make_float2(dmEt.x - tez.x * ri, dmEt.y - tez.y * ri);
  const size_t base = (size_t)md * 6 * fs + i0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const size_t o = base + (size_t)f * fs;
    const float2 v = make_float2(a.scale * h[f].x, a.scale * h[f].y);
    if (a.out) a.out[o] = v;
    float2 s = a.accin[o];
    s.x += v.x;
    s.y += v.y;
    if (a.sub) {
      const float2 q = a.sub[o];
      s.x -= a.sub_scale * q.x;
      s.y -= a.sub_scale * q.y;
    }
    a.accout[o] = s;
  }
}

// J_state = (J_rho, J_theta, J_z, 0, 0, 0) per mode
__global__ void taylor_jstate_kernel(const float2* J, float2* X, size_t fs, int nm) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)nm * 6 * fs;
  if (i >= total) return;
  const size_t md = i / (6 * fs), rest = i % (6 * fs), f = rest / fs, c = rest % fs;
  X[i] = f < 3 ? J[(md * 3 + f) * fs + c] : make_float2(0.f, 0.f);
}

// axis slot of E_rho, B_theta (polar weights) and B_z (scalar weights) from slots 1..ND
__global__ void taylor_axis_kernel(float2* F, const float* axis, int Nz, int n, int ND, int nm) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  const int md = blockIdx.y;
  if (z >= Nz || md >= nm) return;
  const size_t fs = (size_t)Nz * n;
  const float* wp = axis + (size_t)md * 2 * ND;
  const float* ws = wp + ND;
  const int fields[3] = {0, 4, 5};
  for (int q = 0; q < 3; ++q) {
    float2* row = F + ((size_t)md * 6 + fields[q]) * fs + (size_t)z * n;
    const float* w = q < 2 ? wp : ws;
    float2 s = make_float2(0.f, 0.f);
    for (int t = 0; t < ND && t + 1 < n; ++t) s = fma2(w[t], row[t + 1], s);
    row[0] = s;
  }
}

}  // namespace
}  // namespace fdetd

using namespace fdetd;

struct fdetd_taylor_s {
  int Nz = 0, Nr = 0, nm = 0, order = 0, NT = 0, S = 0;
  double dz = 0, dr = 0, dt = 0;
  float* d_bands = nullptr;
  float* d_rho = nullptr;   // rho_inv [n], rhom_inv [n]
  float* d_axis = nullptr;  // [nm][2][ND]
  float2* d_buf = nullptr;  // T0, T1, ACC, SRC, XJ: [nm][6][Nz][n] each
  TaylorArgs base;
};

static int taylor_fail(int code, const std::string& msg) { return fdetd::set_error(code, msg); }

extern "C" int fdetd_taylor_destroy(fdetd_taylor_t p) {
  if (!p) return FDETD_OK;
  if (p->d_bands) cudaFree(p->d_bands);
  if (p->d_rho) cudaFree(p->d_rho);
  if (p->d_axis) cudaFree(p->d_axis);
  if (p->d_buf) cudaFree(p->d_buf);
  delete p;
  return FDETD_OK;
}

extern "C" int fdetd_taylor_plan(fdetd_taylor_t* out, int Nz, int Nr, const int* modes, int nmodes, int order,
                                 double dz, double dr, double dt, int taylor_order, int substeps) {
  if (!out) return taylor_fail(FDETD_ERR_ARG, "out is null");
  *out = nullptr;
  if (!modes || nmodes < 1 || nmodes > kMaxModes) return taylor_fail(FDETD_ERR_ARG, "need 1..64 modes");
  if (Nz < 2 || order < 2 || order > 32 || (order & 1) || Nr < order / 2 + 2)
    return taylor_fail(FDETD_ERR_ARG, "bad Nz, order or Nr (Nr >= order/2 + 2)");
  if (taylor_order < 2 || taylor_order > 32 || substeps < 1 || substeps > 1024)
    return taylor_fail(FDETD_ERR_ARG, "taylor_order must be 2..32 and substeps 1..1024");
  if (!(dz > 0) || !(dr > 0) || !(dt > 0)) return taylor_fail(FDETD_ERR_ARG, "dz, dr, dt must be positive");
  const int ND = order / 2, W = 2 * ND + 1, n = Nr;
  std::vector<float> bands((size_t)nmodes * 4 * n * W), axis((size_t)nmodes * 2 * ND);
  for (int i = 0; i < nmodes; ++i) {
    if (modes[i] < 0 || modes[i] > 64) return taylor_fail(FDETD_ERR_ARG, "mode numbers must be 0..64");
    std::vector<double> b, ax;
    if (taylor_bands(n, order, dr, modes[i], b, ax)) return taylor_fail(FDETD_ERR_ARG, "radial band construction failed");
    for (size_t q = 0; q < b.size(); ++q) bands[(size_t)i * 4 * n * W + q] = (float)b[q];
    for (size_t q = 0; q < ax.size(); ++q) axis[(size_t)i * 2 * ND + q] = (float)ax[q];
  }
  std::vector<float> rho(2 * (size_t)n);
  for (int k = 0; k < n; ++k) {
    rho[k] = (float)(1.0 / ((k + 0.5) * dr));
    rho[n + k] = k ? (float)(1.0 / (k * dr)) : 0.f;
  }
  const std::vector<double> c = staggered_coeffs(order);
  fdetd_taylor_s* p = new fdetd_taylor_s();
  p->Nz = Nz;
  p->Nr = Nr;
  p->nm = nmodes;
  p->order = order;
  p->NT = taylor_order;
  p->S = substeps;
  p->dz = dz;
  p->dr = dr;
  p->dt = dt;
  const size_t fs = (size_t)nmodes * 6 * Nz * n;
  cudaError_t e = cudaMalloc(&p->d_bands, bands.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_rho, rho.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_axis, std::max<size_t>(1, axis.size()) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_buf, 5 * fs * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemcpy(p->d_bands, bands.data(), bands.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_rho, rho.data(), rho.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_axis, axis.data(), axis.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    fdetd_taylor_destroy(p);
    return taylor_fail(e == cudaErrorMemoryAllocation ? FDETD_ERR_OOM : FDETD_ERR_CUDA,
                       std::string("taylor plan: ") + cudaGetErrorString(e));
  }
  TaylorArgs& a = p->base;
  memset(&a, 0, sizeof(a));
  a.bands = p->d_bands;
  a.rho_inv = p->d_rho;
  a.rhom_inv = p->d_rho + n;
  for (int t = 1; t <= ND; ++t) a.cz[t] = (float)(c[t - 1] / dz);
  a.Nz = Nz;
  a.n = n;
  a.ND = ND;
  a.nm = nmodes;
  for (int i = 0; i < nmodes; ++i) a.m[i] = modes[i];
  *out = p;
  return FDETD_OK;
}

// One substep T_N(h H) applied to x_in, written to x_out (x_out may equal x_in: it is read only by
// the first term and written only by the last), the last term optionally subtracting sub_scale*sub.
static cudaError_t taylor_series(fdetd_taylor_s* p, const float2* x_in, float2* x_out, double h, const float2* sub,
                                 float sub_scale, cudaStream_t st) {
  const size_t fs = (size_t)p->nm * 6 * p->Nz * p->Nr;
  float2* T[2] = {p->d_buf, p->d_buf + fs};
  float2* ACC = p->d_buf + 2 * fs;
  const dim3 grid((p->Nr + 31) / 32, (p->Nz + 7) / 8, p->nm);
  for (int t = 1; t <= p->NT; ++t) {
    TaylorArgs a = p->base;
    a.scale = (float)(h / t);
    a.in = t == 1 ? x_in : T[(t - 2) & 1];
    const bool last = t == p->NT;
    a.out = last ? nullptr : T[(t - 1) & 1];
    a.accin = t == 1 ? x_in : ACC;
    a.accout = last ? x_out : ACC;
    a.sub = last ? sub : nullptr;
    a.sub_scale = sub_scale;
    taylor_term_kernel<<<grid, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

extern "C" int fdetd_taylor_step(fdetd_taylor_t p, void* fields, const void* J, int nsteps, void* stream) {
  if (!p) return taylor_fail(FDETD_ERR_ARG, "plan is null");
  if (!fields) return taylor_fail(FDETD_ERR_ARG, "fields is null");
  if (nsteps < 0) return taylor_fail(FDETD_ERR_ARG, "nsteps < 0");
  if (((uintptr_t)fields & 7) || ((uintptr_t)J & 7)) return taylor_fail(FDETD_ERR_ARG, "pointers must be 8-byte aligned");
  if (nsteps == 0) return FDETD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  float2* x = (float2*)fields;
  const size_t fsz = (size_t)p->Nz * p->Nr;
  const size_t fs = (size_t)p->nm * 6 * fsz;
  float2* SRC = p->d_buf + 3 * fs;
  float2* XJ = p->d_buf + 4 * fs;
  cudaError_t e = cudaSuccess;
  if (J) {
    // the current's source term T_N(h' H)^S' J_state, h' = (dt / 2) / S' (J constant over the call)
    const int S2 = std::max(1, p->S / 2);
    const int threads = 256;
    const unsigned blocks = (unsigned)((fs + threads - 1) / threads);
    taylor_jstate_kernel<<<blocks, threads, 0, st>>>((const float2*)J, XJ, fsz, p->nm);
    e = cudaGetLastError();
    for (int s = 0; e == cudaSuccess && s < S2; ++s)
      e = taylor_series(p, s == 0 ? XJ : SRC, SRC, 0.5 * p->dt / S2, nullptr, 0.f, st);
  }
  for (int step = 0; e == cudaSuccess && step < nsteps; ++step)
    for (int s = 0; e == cudaSuccess && s < p->S; ++s) {
      const bool last = s == p->S - 1;
      e = taylor_series(p, x, x, p->dt / p->S, (J && last) ? SRC : nullptr, (float)p->dt, st);
    }
  if (e == cudaSuccess) {
    const dim3 grid((p->Nz + 127) / 128, p->nm);
    taylor_axis_kernel<<<grid, 128, 0, st>>>(x, p->d_axis, p->Nz, p->Nr, p->order / 2, p->nm);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return taylor_fail(FDETD_ERR_CUDA, std::string("taylor step: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

extern "C" int fdetd_taylor_launches_per_step(fdetd_taylor_t p) { return p ? p->S * p->NT : 0; }

// Host-only export of the banded radial operators and axis weights of one mode (CPU tests).
extern "C" int fdetd_taylor_host_bands(int Nr, int order, double dr, int m, double* bands, double* axis) {
  std::vector<double> b, ax;
  if (taylor_bands(Nr, order, dr, m, b, ax)) return FDETD_ERR_ARG;
  if (bands) std::copy(b.begin(), b.end(), bands);
  if (axis) std::copy(ax.begin(), ax.end(), axis);
  return FDETD_OK;
}
