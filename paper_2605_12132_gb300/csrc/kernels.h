// Kernel argument records and launchers of the FDETD step (internal).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace fdetd {

// Records an error message for fdetd_last_error and returns code (defined in fdetd_api.cu).
int set_error(int code, const std::string& msg);

// ---------------------------------------------------------------- spectral kernel
struct SpectralArgs {
  void* coef;            // [nmodes][9][n][Nz] complex<T>; first 6 arrays updated in place
  const void* phase;     // [nmodes][2][n][Nz] PhaseD / PhaseF, Nz in position order (spectral_positions)
  const void* zsym;      // [Nz] ZSymD / ZSymF, position order
  const void* lam;       // [nmodes][2][n] double / df (lambda for TM, mu for TE)
  const void* twiddle;   // per-stage twiddle tables (spectral_twiddles), complex<T>
  int tw_count;          // entries in `twiddle`
  __nv_bfloat16* split_out;  // tensor-core path: pre-tiled pieces, see split_store
  int npieces;
  int split_kstages;         // 64-wide j stages of the back-projection (ceil(n / 64))
  int Nz, logNz, n;
  double dt;
  int hasJ;
  int* err;              // the plan's device failure flag (the spectral kernel has no waits that could set it)
  void* src;             // [nmodes][2][3][n][Nz] complex<T>: kz-space source term (two-kernel path)
  const void* zsymk;     // [Nz] ZSymK, position order (FP32 data: the kernel specialised on Nz)
  unsigned long long* phases;  // cycle counters of the Nz-specialised kernel's phases (8 words) or null
};

cudaError_t launch_spectral(const SpectralArgs& a, int nmodes, int precision, bool split_out, cudaStream_t st);
// column-split form (three kernels, one column in shared memory at a time): power-of-two Nz whose single
// padded column fits in shared memory; bitwise the results of the fused form
cudaError_t launch_spectral_columns(const SpectralArgs& a, int nmodes, int precision, bool split_out,
                                    cudaStream_t st);
bool spectral_columns_supported(int Nz, int precision);
size_t spectral_smem_bytes(int Nz, int precision, bool hasJ);
int spectral_twiddles(int Nz, int precision, double* re, double* im);
// kz index held at each position of the forward transform's output (the order of the phase and z tables)
void spectral_positions(int Nz, int precision, int* kz);
bool spectral_needs_source(int Nz, int precision, int tw_count);
// Stage radices of the z transform (first to last); spectral_radices fills them for any Nz = 2^a 3^b 5^c 7^d
struct MixedRadices {
  static constexpr int kMax = 16;
  int nst;
  int rad[kMax];
};
int spectral_radices(int Nz, int precision, int* rad);   // returns the number of stages (0: not 7-smooth)
// Nz not a power of two (7-smooth): one kernel with runtime stage radices (k_spectral_mixed.cu)
size_t spectral_mixed_smem_bytes(int Nz, int precision, bool hasJ, int tw_count);
bool spectral_mixed_needs_source(int Nz, int precision, int tw_count);
cudaError_t launch_spectral_mixed(const SpectralArgs& a, const MixedRadices& mr, int nmodes, int precision,
                                  bool split_out, cudaStream_t st);
// FP32 data, Nz = 2^k in 64..4096: the kernel specialised on Nz (k_spectral32.cu); cudaErrorNotSupported
// for other lengths
bool spectral32_supported(int Nz);
size_t spectral32_smem_bytes(int Nz, bool hasJ);
cudaError_t launch_spectral32(const SpectralArgs& a, int nmodes, bool split_out, cudaStream_t st);

// bf16 split of FP32 values into npieces (2 or 3) terms whose sum reproduces them to 16 / 24
// significant bits, stored in the pre-tiled operand layout of the back-projection: 16 KB blocks
// (md, piece, c, ks = j / 64, zb = z / 64), each [2 halves][64 j rows][128 B] holding (z, re/im)
// pairs of 64 z along N, the 16-byte chunks of a row swizzled by (j & 7) (the 128-byte swizzle the
// MMA descriptor expects).  SplitColumn holds what is fixed for one coefficient column (md, c, j).
struct SplitColumn {
  unsigned char* base;  // block (md, piece 0, c, j / 64, zb = 0) + row (j & 63)
  size_t piece_stride;  // bytes between pieces: 6 kst (Nz / 64) 16 KB
  int npieces, jr7;     // pieces; j & 7
};

__device__ __forceinline__ SplitColumn split_column(__nv_bfloat16* out, int npieces, int md, int c, int j, int kst,
                                                    int Nz) {
  SplitColumn d;
  const size_t nzb = (size_t)(Nz >> 6);
  d.base = reinterpret_cast<unsigned char*>(out) +
           (((((size_t)md * npieces) * 6 + c) * kst + (j >> 6)) * nzb) * 16384 + (size_t)(j & 63) * 128;
  d.piece_stride = (size_t)6 * kst * nzb * 16384;
  d.npieces = npieces;
  d.jr7 = j & 7;
  return d;
}

__device__ __forceinline__ void split_store(const SplitColumn& d, int z, float vr, float vi) {
  const int zl = z & 63;
  const size_t off = (size_t)(z >> 6) * 16384 + (size_t)(zl >> 5) * 8192 +
                     ((uint32_t)(((zl & 31) >> 2) ^ d.jr7) << 4) + (uint32_t)(zl & 3) * 4u;
  unsigned char* q = d.base + off;
  float r0 = vr, r1 = vi;
  for (int p = 0; p < d.npieces; ++p) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(r0), h1 = __float2bfloat16_rn(r1);
    __nv_bfloat162 pr;
    pr.x = h0;
    pr.y = h1;
    *reinterpret_cast<__nv_bfloat162*>(q) = pr;
    q += d.piece_stride;
    r0 -= __bfloat162float(h0);
    r1 -= __bfloat162float(h1);
  }
}

// split_store of four consecutive z (z0 a multiple of 4): their (re, im) pairs share one 16-byte chunk of the
// swizzled row, so each piece is one 16-byte store
__device__ __forceinline__ void split_store4(const SplitColumn& d, int z0, const float* vr, const float* vi) {
  const int zl = z0 & 63;
  const size_t off = (size_t)(z0 >> 6) * 16384 + (size_t)(zl >> 5) * 8192 + ((uint32_t)(((zl & 31) >> 2) ^ d.jr7) << 4);
  unsigned char* q = d.base + off;
  float r0[4], r1[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    r0[k] = vr[k];
    r1[k] = vi[k];
  }
  for (int p = 0; p < d.npieces; ++p) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(r0[k]), h1 = __float2bfloat16_rn(r1[k]);
      __nv_bfloat162 pr;
      pr.x = h0;
      pr.y = h1;
      w[k] = *reinterpret_cast<const uint32_t*>(&pr);
      r0[k] -= __bfloat162float(h0);
      r1[k] -= __bfloat162float(h1);
    }
    *reinterpret_cast<uint4*>(q) = make_uint4(w[0], w[1], w[2], w[3]);
    q += d.piece_stride;
  }
}

// ---------------------------------------------------------------- CUDA-core projections
struct ProjArgs {
  const void* fields;  // [nmodes][6][Nz][Nr] complex<T>
  const void* J;       // [nmodes][3][Nz][Nr] complex<T> or null
  const void* P;       // [nmodes][2][3n][3n] T   (PE, PB)
  void* coef;          // [nmodes][9][n][Nz] complex<T>
  int Nz, n;
};
struct BackArgs {
  void* fields;        // [nmodes][6][Nz][Nr] complex<T>
  const void* Q;       // [nmodes][2][3n][3n] T   (QE, QB)
  const void* coef;    // [nmodes][9][n][Nz] complex<T>
  int Nz, n;
};

cudaError_t launch_project_simt(const ProjArgs& a, int nmodes, int precision, cudaStream_t st);
cudaError_t launch_backproject_simt(const BackArgs& a, int nmodes, int precision, cudaStream_t st);

// ---------------------------------------------------------------- tensor-core projections
// One instance of a grouped launch (kernel parameter; pointers are device pointers).
constexpr int kMaxGroupInstances = 64;
struct GInst {
  float2* fields;      // [nmodes][6][Nz][n] complex64, read by the projection, written by the back-projection
  const float2* J;     // [nmodes][3][Nz][n] or null
  float* coef;         // [nmodes][9][n][2 Nz] FP32 coefficient scratch
  const uint8_t* P;    // pre-tiled projection pieces
  const uint8_t* Q;    // pre-tiled back-projection pieces
  const uint8_t* S;    // pre-tiled split coefficients (written by the spectral kernel)
  int* err;            // device failure flag of the instance's plan
  int Nz, n, njb, pad;
};
struct GroupParams {
  GInst inst[kMaxGroupInstances];
  CUtensorMap fmap[kMaxGroupInstances];  // FP32 views of the fields (rows of 2 n floats), 64 x 64 boxes
  CUtensorMap jmap[kMaxGroupInstances];  // the same for J (unused entries zero)
  int count;
  long long spin;                         // polls before a pipeline wait gives up (kSpinLimit unless set)
  unsigned long long* waits;              // pipeline cycle counters, 8 per kernel (null: not counted)
};
// Tile shapes and schedules of the persistent kernels (chosen by the autotuner):
// tn_p / tn_b = N tile of the projection / back-projection (128 or 256); sched = tile order
// (0: longest first, round-robin over CTAs; 1: longest first, snake order).
struct TcConfig {
  int tn_p, tn_b, sched_p, sched_b;
};

struct TcPlan;   // defined in k_tc.cu
struct TcGroup;  // a tile table over one or more instances
cudaError_t tc_create(TcPlan** out, int Nz, int n, int nmodes, int npieces, const double* P, const double* Q,
                      int* err, char* msg, size_t msglen);
void tc_destroy(TcPlan* p);
size_t tc_device_bytes(const TcPlan* p);
__nv_bfloat16* tc_split_buffer(TcPlan* p);
int tc_split_kstages(const TcPlan* p);
int tc_pieces(const TcPlan* p);
TcConfig tc_default_config(int npieces);
TcConfig tc_plan_config(const TcPlan* p);
cudaError_t tc_plan_set_config(TcPlan* p, const TcConfig& c);
bool tc_config_valid(const TcPlan* const* plans, int count, const TcConfig& c);
// single-instance launches through a one-instance group kept by the plan (built on first use,
// which must not happen during a stream capture: tc_prepare builds it ahead)
cudaError_t tc_prepare(TcPlan* p, const void* fields, const void* J, void* coef);
cudaError_t tc_project(TcPlan* p, const void* fields, const void* J, void* coef, cudaStream_t st);
cudaError_t tc_backproject(TcPlan* p, void* fields, cudaStream_t st);
int tc_launches_per_step(const TcPlan* p);
// polls before a pipeline wait of this plan's single-instance launches gives up (< 0: the default limit;
// 0: every wait gives up at once, which drives the timeout path on a healthy pipeline)
void tc_set_wait_limit(TcPlan* p, long long polls);
// pipeline cycle counters (16 device words: 8 of the projection, 8 of the back-projection; null stops counting)
void tc_set_waits(TcPlan* p, unsigned long long* counters);
void tc_group_set_waits(TcGroup* g, unsigned long long* counters);
// grouped launches over up to kMaxGroupInstances instances of one precision
cudaError_t tc_group_create(TcGroup** out, TcPlan* const* plans, const void* const* fields, const void* const* J,
                            int count, const TcConfig& cfg);
void tc_group_set_coef(TcGroup* g, int k, void* coef);
void tc_group_set_fields(TcGroup* g, int k, void* fields);
void tc_group_destroy(TcGroup* g);
cudaError_t tc_group_project(TcGroup* g, cudaStream_t st);
cudaError_t tc_group_backproject(TcGroup* g, cudaStream_t st);
int tc_group_tiles(const TcGroup* g, int which);

// ---------------------------------------------------------------- current pipeline
struct CurParams {
  const void* J;       // [nm][3][Nz][n] complex<T> deposited on the primary grids
  const void* rho_xy;  // [nm][Nz][n] complex<T>
  void* out;           // [nm][3][Nz][n] complex<T>
  // -Div^+ [nm][W][n], D^- [nm][W][n], -L [nm][n][ND], -U off-diagonals [nm][n][ND], 1/U(k,k) [nm][n],
  // m/rho [nm][n], back to back; 8-byte elements: doubles (FP64 data) or (hi, lo) float pairs (FP32 data)
  const void* bands;
  double w[32];        // half-point Lagrange weights
  double dr;
  int Nz, n, ND, nm;
  int m[64];
  int stagger_only;    // 1: the downstagger of J_rho alone (rho_xy and bands unused, may be null)
};
cudaError_t launch_current(const CurParams& p, bool fp64, cudaStream_t st);

// ---------------------------------------------------------------- destagger to the primary grids
cudaError_t launch_destagger(const void* in, void* out, int Nz, int n, int order, const int* modes, int nmodes,
                             bool fp64, cudaStream_t st);

// ---------------------------------------------------------------- envelope
struct EnvArgs {
  // One Taylor term: out = scale * H_a(in); accout = accin + out.
  const float2* in_a;   // [Nz][Nr] previous term, a part
  const float2* in_t;   // [Nz][Nr] previous term, a~ part
  float2* out_a;        // next term (may be null when not needed again)
  float2* out_t;
  const float2* accin_a;
  const float2* accin_t;
  float2* accout_a;     // running Taylor sum
  float2* accout_t;
  const float* chi;     // [Nz][Nr]
  const float* lr;      // [Nr][2N+2] radial Laplacian band, axis mirror folded (column r + t at index t + N),
                        // last entry of each row = the row sum (FP64-accumulated)
  float scale;          // dt / n
  int Nz, Nr, N;        // N = order / 2
  float cz2[17];        // centred second derivative in z divided by dz^2: e0, e1..eN
  float cz1[17];        // centred first derivative in z divided by dz: d1..dN at [1..N]
  float k2;             // 2 k0
  float dt_over[17];    // (float)(dt / n), n = 1..16 (the fused launch)
};
cudaError_t launch_envelope_term(const EnvArgs& a, cudaStream_t st);
// all N_T Taylor terms of one step in one launch (temporal blocking); order 8 and N_T = 4, Nz a multiple of 32
size_t envelope_fused_smem(int order, int taylor_order);
bool envelope_fused_supported(int order, int taylor_order);
cudaError_t launch_envelope_fused(const EnvArgs& a, const float2* in_a, const float2* in_t, float2* out_a,
                                  float2* out_t, int taylor_order, cudaStream_t st);
cudaError_t launch_envelope_chit(const float* chi, const float* sigma, float* chit, size_t n, cudaStream_t st);
cudaError_t launch_envelope_damp(float2* psi, const float* sigma, float c, size_t n, cudaStream_t st);

}  // namespace fdetd
