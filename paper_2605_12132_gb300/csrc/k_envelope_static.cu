// Allocation-free envelope step (no counterpart in the paper).
//
// Some callers cannot allocate device memory when they advance the envelope: applications
// whose device memory is entirely pre-reserved by their own pool or arena at start-up,
// plugins embedded in a host framework that owns every allocation, and latency-critical
// loops that cannot afford the implicit synchronisation of an allocation.  envelope_step_static serves them: it needs no plan and calls no
// cudaMalloc / cudaFree or allocating library routine.  Its scratch (two Taylor-term
// buffers) lives in one file-scope device array of fixed capacity; the radial Laplacian band
// is computed in the kernel from coefficients passed by value.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "fdetd.h"
#include "plan_host.h"

namespace fdetd {

// Capacity: Nz * Nr <= 2^20 cells; four complex64 planes (a, a~ of two terms) = 32 MiB.
constexpr size_t kEnvStaticMaxCells = (size_t)1 << 20;
static __device__ __align__(256) float2 g_env_scratch[4 * kEnvStaticMaxCells];

struct EnvStaticArgs {
  const float2* in_a;
  const float2* in_t;
  float2* out_a;   // next term (null when the term is not needed again)
  float2* out_t;
  float2* acc_a;   // running sum, updated in place (null for the first term)
  float2* acc_t;
  const float2* prev_a;  // previous term added to the sum together with this one (second term only)
  const float2* prev_t;
  const float* chi;
  float scale;
  int Nz, Nr, N;
  float dr;
  float cz2[17], cz1[17];  // z: e_n / dz^2 (e_0 at [0]), d_n / dz at [1..N]
  float cr2[17], cr1[17];  // rho: e_n / dr^2 (e_0 at [0]), d_n / dr at [1..N]
  float k2;
};

// One Taylor term of H_a (complex form of Eq. spatialAM_envelope_H, m = 0, symmetric axis mirror,
// taps past the outer edge dropped, periodic z); stencils in difference form.
__global__ void __launch_bounds__(256) envelope_static_term(EnvStaticArgs a) {
  const int r = blockIdx.x * 32 + (threadIdx.x & 31);
  const int z = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (r >= a.Nr || z >= a.Nz) return;
  const int Nr = a.Nr, Nz = a.Nz, N = a.N;
  const size_t idx = (size_t)z * Nr + r;
  const float2 ac = a.in_a[idx], at = a.in_t[idx];
  const float2* row = a.in_a + (size_t)z * Nr;
  const float rho = (r + 0.5f) * a.dr;
  float rowsum = a.cr2[0];
  float lx = 0.f, ly = 0.f;
  for (int n = 1; n <= N; ++n) {
    const float wp = a.cr2[n] + a.cr1[n] / rho, wm = a.cr2[n] - a.cr1[n] / rho;
    const int jp = r + n;
    if (jp < Nr) {
      const float2 v = row[jp];
      lx = fmaf(wp, v.x - ac.x, lx);
      ly = fmaf(wp, v.y - ac.y, ly);
      rowsum += wp;
    }
    int jm = r - n;
    if (jm < 0) jm = -1 - jm;  // symmetric mirror through the axis
    if (jm < Nr) {
      const float2 v = row[jm];
      lx = fmaf(wm, v.x - ac.x, lx);
      ly = fmaf(wm, v.y - ac.y, ly);
      rowsum += wm;
    }
  }
  lx = fmaf(rowsum, ac.x, lx);
  ly = fmaf(rowsum, ac.y, ly);
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
  const float tx = lx - chi * ac.x - a.k2 * (dy + at.y);
  const float ty = ly - chi * ac.y + a.k2 * (dx + at.x);
  const float2 oa = make_float2(a.scale * at.x, a.scale * at.y);
  const float2 ot = make_float2(a.scale * tx, a.scale * ty);
  if (a.out_a) {
    a.out_a[idx] = oa;
    a.out_t[idx] = ot;
  }
  if (a.acc_a) {
    float2 sa = a.acc_a[idx], st = a.acc_t[idx];
    if (a.prev_a) {
      const float2 pa = a.prev_a[idx], pt = a.prev_t[idx];
      sa.x += pa.x;
      sa.y += pa.y;
      st.x += pt.x;
      st.y += pt.y;
    }
    a.acc_a[idx] = make_float2(sa.x + oa.x, sa.y + oa.y);
    a.acc_t[idx] = make_float2(st.x + ot.x, st.y + ot.y);
  }
}

// psi += term (used when the series has a single term: the first term cannot update psi in
// place because neighbouring threads still read psi through the stencil)
__global__ void __launch_bounds__(256) envelope_static_add(float2* psi, const float2* term, size_t count) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    const float2 t = term[i];
    float2 p = psi[i];
    p.x += t.x;
    p.y += t.y;
    psi[i] = p;
  }
}

// Device address of the scratch array, looked up once per device with that device current.
static float2* scratch_address(int* rc) {
  static std::mutex mu;
  static float2* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *rc = FDETD_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_env_scratch) != cudaSuccess || !p) {
      *rc = FDETD_ERR_CUDA;
      return nullptr;
    }
    addr[dev] = static_cast<float2*>(p);
  }
  *rc = FDETD_OK;
  return addr[dev];
}

}  // namespace fdetd

using namespace fdetd;

extern "C" int envelope_step_static(void* a, const float* chi, int Nz, int Nr, int order, int taylor_order,
                                    double dz, double dr, double dt, double k0, int nsteps, void* stream) {
  if (!a || !chi || nsteps < 0) return FDETD_ERR_ARG;
  if (order < 2 || order > 32 || (order & 1) || taylor_order < 1 || taylor_order > 16) return FDETD_ERR_ARG;
  const int N = order / 2;
  if (Nz < 2 * order || Nr < N + 1 || !(dz > 0) || !(dr > 0) || !(dt > 0)) return FDETD_ERR_ARG;
  if ((size_t)Nz * (size_t)Nr > kEnvStaticMaxCells) return FDETD_ERR_ARG;  // beyond the static scratch
  if (((uintptr_t)a & 15) || ((uintptr_t)chi & 15)) return FDETD_ERR_ARG;
  int rc = FDETD_OK;
  float2* scratch = scratch_address(&rc);
  if (!scratch) return rc;
  double d1[16], e2[16], e0 = 0.0;
  if (centred_coeffs_fixed(order, d1, e2, &e0) != N) return FDETD_ERR_ARG;
  EnvStaticArgs g;
  memset(&g, 0, sizeof(g));
  g.chi = chi;
  g.Nz = Nz;
  g.Nr = Nr;
  g.N = N;
  g.dr = (float)dr;
  g.k2 = (float)(2.0 * k0);
  g.cz2[0] = (float)(e0 / (dz * dz));
  g.cr2[0] = (float)(e0 / (dr * dr));
  for (int n = 1; n <= N; ++n) {
    g.cz2[n] = (float)(e2[n - 1] / (dz * dz));
    g.cz1[n] = (float)(d1[n - 1] / dz);
    g.cr2[n] = (float)(e2[n - 1] / (dr * dr));
    g.cr1[n] = (float)(d1[n - 1] / dr);
  }
  const size_t plane = (size_t)Nz * Nr;
  float2* psi_a = (float2*)a;
  float2* psi_t = psi_a + plane;
  float2* T[2][2] = {{scratch, scratch + plane}, {scratch + 2 * plane, scratch + 3 * plane}};
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid((Nr + 31) / 32, (Nz + 7) / 8);
  for (int s = 0; s < nsteps; ++s) {
    for (int n = 1; n <= taylor_order; ++n) {
      g.scale = (float)(dt / n);
      const bool last = n == taylor_order;
      if (n == 1) {
        g.in_a = psi_a;
        g.in_t = psi_t;
        g.acc_a = g.acc_t = nullptr;  // psi is still read through the stencil
      } else {
        g.in_a = T[(n - 2) & 1][0];
        g.in_t = T[(n - 2) & 1][1];
        g.acc_a = psi_a;
        g.acc_t = psi_t;
      }
      g.prev_a = (n == 2) ? T[0][0] : nullptr;  // the first term joins the sum with the second
      g.prev_t = (n == 2) ? T[0][1] : nullptr;
      const bool keep = !last || taylor_order == 1;
      g.out_a = keep ? T[(n - 1) & 1][0] : nullptr;
      g.out_t = keep ? T[(n - 1) & 1][1] : nullptr;
      envelope_static_term<<<grid, 256, 0, st>>>(g);
      if (cudaGetLastError() != cudaSuccess) return FDETD_ERR_CUDA;
    }
    if (taylor_order == 1) {
      const size_t cnt = 2 * plane;  // (a, a~) planes are contiguous in psi and in the term buffer
      envelope_static_add<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(psi_a, T[0][0], cnt);
      if (cudaGetLastError() != cudaSuccess) return FDETD_ERR_CUDA;
    }
  }
  return FDETD_OK;
}
