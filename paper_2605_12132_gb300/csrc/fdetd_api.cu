// C-ABI of the FDETD solver: plan construction (host FP64 tables -> device),
// the per-step launch sequence, the host-only table export, and the envelope
// propagator.  See include/fdetd.h for the contract of every entry point.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "common.cuh"
#include "fdetd.h"
#include "kernels.h"
#include "plan_host.h"

using namespace fdetd;

static thread_local std::string g_err;
static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int fdetd::set_error(int code, const std::string& msg) { return fail(code, msg); }

static df to_df(double x) {
  df r;
  r.h = (float)x;
  r.l = (float)(x - (double)r.h);
  return r;
}

struct fdetd_plan_s {
  int Nz = 0, Nr = 0, nmodes = 0, order = 0, precision = 0, logNz = 0, tw_count = 0;
  bool columns = false;       // z transform in its column-split form (three launches)
  bool j_primary = false;     // J_rho handed to fdetd_step on the primary grid (FDETD_FLAG_J_ON_PRIMARY)
  void* d_jstag = nullptr;    // its downstaggered copy, the J the step uses
  double dz = 0, dr = 0, dt = 0;
  std::vector<int> modes;
  void* d_P = nullptr;
  void* d_Q = nullptr;
  void* d_phase = nullptr;
  void* d_zsym = nullptr;
  void* d_zsymk = nullptr;   // z symbols with kappa^2 (FP32 data, Nz up to 4096)
  void* d_lam = nullptr;
  void* d_tw = nullptr;
  void* d_coef = nullptr;
  void* d_src = nullptr;     // kz-space source term of the two-kernel spectral path (long Nz)
  int* d_err = nullptr;      // device-side failure code (bounded waits that expired)
  void* d_hostio = nullptr;  // staging for fdetd_step_host (lazy)
  size_t hostio_bytes = 0;
  TcPlan* tc = nullptr;
  size_t bytes = 0;
  void* d_cur = nullptr;     // current correction: band tables per mode (built on first use)
  // optional per-kernel timing: events recorded around each launch on the launch stream
  bool profiling = false;
  unsigned long long* d_waits = nullptr;  // pipeline cycle counters of the tensor-core kernels (profiling)
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  double kern_ms[3] = {0, 0, 0};
  long kern_calls[3] = {0, 0, 0};
};

static void prof_mark(fdetd_plan_s* p, int kind, bool begin, cudaStream_t st) {
  if (!p->profiling) return;
  if (begin) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    p->ev.push_back({kind, {a, b}});
    cudaEventRecord(a, st);
  } else {
    cudaEventRecord(p->ev.back().second.second, st);
  }
}

static void prof_collect(fdetd_plan_s* p) {
  for (auto& e : p->ev) {
    float ms = 0.f;
    cudaEventSynchronize(e.second.second);
    cudaEventElapsedTime(&ms, e.second.first, e.second.second);
    p->kern_ms[e.first] += ms;
    p->kern_calls[e.first] += 1;
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  p->ev.clear();
}

static void plan_free(fdetd_plan_s* p) {
  if (!p) return;
  prof_collect(p);
  void* ptrs[] = {p->d_P,    p->d_Q,   p->d_phase,  p->d_zsym, p->d_zsymk, p->d_lam,
                  p->d_tw,   p->d_coef, p->d_src,   p->d_hostio, p->d_err,  p->d_cur, p->d_waits, p->d_jstag};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->tc) tc_destroy(p->tc);
  delete p;
}

static cudaError_t upload(void** dst, const void* src, size_t bytes, size_t& total) {
  cudaError_t e = cudaMalloc(dst, bytes);
  if (e != cudaSuccess) return e;
  total += bytes;
  return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
}

static bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

extern "C" int fdetd_plan_modes(fdetd_plan_t* out, int Nz, int Nr, const int* modes, int nmodes, int order,
                                double dz, double dr, double dt, int precision, uint64_t flags) {
  if (!out) return fail(FDETD_ERR_ARG, "out is null");
  *out = nullptr;
  if (!modes || nmodes < 1 || nmodes > 64) return fail(FDETD_ERR_ARG, "need 1..64 modes");
  if (precision < FDETD_PREC_FP64 || precision > FDETD_PREC_BF16X6) return fail(FDETD_ERR_ARG, "unknown precision");
  int radices[MixedRadices::kMax];
  if (Nz < 64 || Nz > 8192 || Nz % 64 || !spectral_radices(Nz, precision == FDETD_PREC_FP64 ? 0 : 1, radices))
    return fail(FDETD_ERR_UNSUPPORTED, "the z transform needs Nz = 64 k in 64..8192 with no prime factor above 7");
  const bool hasJ_max = true;
  const int prec01 = precision == FDETD_PREC_FP64 ? 0 : 1;
  const bool fits = is_pow2(Nz) ? spectral_smem_bytes(Nz, precision, hasJ_max) <= 227 * 1024
                                : spectral_mixed_smem_bytes(Nz, prec01, hasJ_max,
                                                            spectral_twiddles(Nz, prec01, nullptr, nullptr)) <=
                                      227 * 1024;
  const bool force_cols = (flags & FDETD_FLAG_SPECTRAL_COLUMNS) != 0;
  if (force_cols && !is_pow2(Nz))
    return fail(FDETD_ERR_UNSUPPORTED, "the column-split z transform takes power-of-two lengths");
  const bool columns = is_pow2(Nz) && (force_cols || !fits) && spectral_columns_supported(Nz, prec01);
  if (!fits && !columns)
    return fail(FDETD_ERR_UNSUPPORTED, "Nz too long for the z transform at this precision");
  HostPlan hp;
  std::string msg;
  int rc = build_host_plan(hp, Nz, Nr, modes, nmodes, order, dz, dr, dt, msg);
  if (rc) return fail(rc == 4 ? FDETD_ERR_EIG : FDETD_ERR_ARG, msg);

  fdetd_plan_s* p = new fdetd_plan_s();
  p->Nz = Nz;
  p->Nr = Nr;
  p->columns = columns;
  p->j_primary = (flags & FDETD_FLAG_J_ON_PRIMARY) != 0;
  p->nmodes = nmodes;
  p->order = order;
  p->precision = precision;
  p->dz = dz;
  p->dr = dr;
  p->dt = dt;
  p->modes.assign(modes, modes + nmodes);
  while ((1 << p->logNz) < Nz) ++p->logNz;   // log2 Nz (power-of-two lengths only)
  const int n = Nr, N3 = 3 * Nr;
  const bool fp64 = precision == FDETD_PREC_FP64;
  const bool tc = precision == FDETD_PREC_BF16X3 || precision == FDETD_PREC_BF16X6;
  cudaError_t e = cudaMalloc((void**)&p->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    plan_free(p);
    return fail(FDETD_ERR_CUDA, std::string("plan: ") + cudaGetErrorString(e));
  }

  // projection matrices: [nmodes][2][3n][3n]
  std::vector<double> P((size_t)nmodes * 2 * N3 * N3), Q(P.size());
  for (int i = 0; i < nmodes; ++i) {
    const size_t blk = (size_t)N3 * N3;
    std::copy(hp.mp[i].PE.begin(), hp.mp[i].PE.end(), P.begin() + (2 * i) * blk);
    std::copy(hp.mp[i].PB.begin(), hp.mp[i].PB.end(), P.begin() + (2 * i + 1) * blk);
    std::copy(hp.mp[i].QE.begin(), hp.mp[i].QE.end(), Q.begin() + (2 * i) * blk);
    std::copy(hp.mp[i].QB.begin(), hp.mp[i].QB.end(), Q.begin() + (2 * i + 1) * blk);
  }
  if (tc) {
    char m2[256] = {0};
    e = tc_create(&p->tc, Nz, n, nmodes, precision == FDETD_PREC_BF16X3 ? 2 : 3, P.data(), Q.data(), p->d_err, m2,
                  sizeof(m2));
    if (e != cudaSuccess) {
      plan_free(p);
      return fail(e == cudaErrorNotSupported ? FDETD_ERR_UNSUPPORTED : FDETD_ERR_CUDA,
                  std::string("tensor-core plan: ") + m2 + " (" + cudaGetErrorString(e) + ")");
    }
    p->bytes += tc_device_bytes(p->tc);
  } else if (fp64) {
    if ((e = upload(&p->d_P, P.data(), P.size() * 8, p->bytes)) != cudaSuccess) goto cuda_fail;
    if ((e = upload(&p->d_Q, Q.data(), Q.size() * 8, p->bytes)) != cudaSuccess) goto cuda_fail;
  } else {
    std::vector<float> Pf(P.begin(), P.end()), Qf(Q.begin(), Q.end());
    if ((e = upload(&p->d_P, Pf.data(), Pf.size() * 4, p->bytes)) != cudaSuccess) goto cuda_fail;
    if ((e = upload(&p->d_Q, Qf.data(), Qf.size() * 4, p->bytes)) != cudaSuccess) goto cuda_fail;
  }
  {
    // phase tables [nmodes][2][n][Nz], eigenvalue tables [nmodes][2][n], z symbols [Nz], twiddles;
    // the per-kz tables are stored in the order the spectral kernel's forward transform leaves kz in
    const size_t nph = (size_t)nmodes * 2 * n * Nz;
    std::vector<int> kz_at(Nz);
    spectral_positions(Nz, fp64 ? 0 : 1, kz_at.data());
    std::vector<PhaseD> phd;
    std::vector<PhaseF> phf;
    if (fp64) phd.resize(nph); else phf.resize(nph);
    std::vector<double> lamd((size_t)nmodes * 2 * n);
    std::vector<df> lamf(lamd.size());
    for (int i = 0; i < nmodes; ++i)
      for (int fam = 0; fam < 2; ++fam)
        for (int j = 0; j < n; ++j) {
          const ModePlan& mp = hp.mp[i];
          const double lv = fam == 0 ? mp.lam[j] : mp.mu[j];
          const bool live = fam == 0 ? mp.tm_live[j] : mp.te_live[j];
          lamd[(size_t)(i * 2 + fam) * n + j] = lv;
          lamf[(size_t)(i * 2 + fam) * n + j] = to_df(lv);
          for (int q = 0; q < Nz; ++q) {  // q: position
            double A1 = 0, A2 = 0, B1 = 0, B2 = 0;
            if (live) {
              const double w = std::sqrt(hp.kappa2[kz_at[q]] + lv);
              phase_coeffs(w, dt, &A1, &A2);
              phase_coeffs(w, 0.5 * dt, &B1, &B2);
            }
            const size_t k = ((size_t)(i * 2 + fam) * n + j) * Nz + q;
            if (fp64) {
              phd[k] = PhaseD{A1, A2, B1, B2};
            } else {
              PhaseF f;
              f.A1 = to_df(A1);
              f.A2 = to_df(A2);
              phf[k] = f;
            }
          }
        }
    if (fp64) {
      if ((e = upload(&p->d_phase, phd.data(), nph * sizeof(PhaseD), p->bytes)) != cudaSuccess) goto cuda_fail;
      if ((e = upload(&p->d_lam, lamd.data(), lamd.size() * 8, p->bytes)) != cudaSuccess) goto cuda_fail;
    } else {
      if ((e = upload(&p->d_phase, phf.data(), nph * sizeof(PhaseF), p->bytes)) != cudaSuccess) goto cuda_fail;
      if ((e = upload(&p->d_lam, lamf.data(), lamf.size() * sizeof(df), p->bytes)) != cudaSuccess) goto cuda_fail;
    }
    std::vector<ZSymD> zd(Nz);
    std::vector<ZSymF> zf(Nz);
    for (int q = 0; q < Nz; ++q) {
      const int k = kz_at[q];
      zd[q] = ZSymD{hp.sp_re[k], hp.sp_im[k]};
      ZSymF f;
      f.spr = to_df(hp.sp_re[k]);
      f.spi = to_df(hp.sp_im[k]);
      zf[q] = f;
    }
    if (fp64) {
      if ((e = upload(&p->d_zsym, zd.data(), Nz * sizeof(ZSymD), p->bytes)) != cudaSuccess) goto cuda_fail;
    } else {
      if ((e = upload(&p->d_zsym, zf.data(), Nz * sizeof(ZSymF), p->bytes)) != cudaSuccess) goto cuda_fail;
      if (spectral32_supported(Nz)) {
        std::vector<ZSymK> zk(Nz);
        for (int q = 0; q < Nz; ++q) {
          const int k = kz_at[q];
          zk[q].spr = to_df(hp.sp_re[k]);
          zk[q].spi = to_df(hp.sp_im[k]);
          zk[q].k2 = to_df(hp.kappa2[k]);
          zk[q].pad = to_df(0.0);
        }
        if ((e = upload(&p->d_zsymk, zk.data(), Nz * sizeof(ZSymK), p->bytes)) != cudaSuccess) goto cuda_fail;
      }
    }
    const int prec_k = fp64 ? 0 : 1;
    p->tw_count = spectral_twiddles(Nz, prec_k, nullptr, nullptr);
    std::vector<double> tre(p->tw_count + 1), tim(p->tw_count + 1);
    spectral_twiddles(Nz, prec_k, tre.data(), tim.data());
    std::vector<double> twd(2 * (p->tw_count + 1));
    std::vector<float> twf(2 * (p->tw_count + 1));
    for (int k = 0; k < p->tw_count; ++k) {
      twd[2 * k] = tre[k];
      twd[2 * k + 1] = tim[k];
      twf[2 * k] = (float)tre[k];
      twf[2 * k + 1] = (float)tim[k];
    }
    if (fp64) {
      if ((e = upload(&p->d_tw, twd.data(), twd.size() * 8, p->bytes)) != cudaSuccess) goto cuda_fail;
    } else {
      if ((e = upload(&p->d_tw, twf.data(), twf.size() * 4, p->bytes)) != cudaSuccess) goto cuda_fail;
    }
    const size_t cbytes = (size_t)nmodes * 9 * n * Nz * (fp64 ? 16 : 8);
    if ((e = cudaMalloc(&p->d_coef, cbytes)) != cudaSuccess) goto cuda_fail;
    p->bytes += cbytes;
    if (p->j_primary) {
      const size_t jbytes = (size_t)nmodes * 3 * n * Nz * (fp64 ? 16 : 8);
      if ((e = cudaMalloc(&p->d_jstag, jbytes)) != cudaSuccess) goto cuda_fail;
      p->bytes += jbytes;
    }
    if (!p->columns && (is_pow2(Nz) ? spectral_needs_source(Nz, prec_k, p->tw_count)
                                     : spectral_mixed_needs_source(Nz, prec_k, p->tw_count))) {
      const size_t sbytes = (size_t)nmodes * 2 * 3 * n * Nz * (fp64 ? 16 : 8);
      if ((e = cudaMalloc(&p->d_src, sbytes)) != cudaSuccess) goto cuda_fail;
      p->bytes += sbytes;
    }
  }
  *out = p;
  return FDETD_OK;
cuda_fail:
  plan_free(p);
  return fail(e == cudaErrorMemoryAllocation ? FDETD_ERR_OOM : FDETD_ERR_CUDA,
              std::string("plan upload: ") + cudaGetErrorString(e));
}

extern "C" int fdetd_plan(fdetd_plan_t* out, int Nz, int Nr, int M, int order, double dz, double dr, double dt,
                          int precision, uint64_t flags) {
  if (M < 0 || M > 63) return fail(FDETD_ERR_ARG, "M must be 0..63");
  std::vector<int> modes(M + 1);
  for (int m = 0; m <= M; ++m) modes[m] = m;
  return fdetd_plan_modes(out, Nz, Nr, modes.data(), M + 1, order, dz, dr, dt, precision, flags);
}

static SpectralArgs spectral_args(fdetd_plan_s* p, bool hasJ) {
  SpectralArgs sa;
  sa.coef = p->d_coef;
  sa.phase = p->d_phase;
  sa.zsym = p->d_zsym;
  sa.zsymk = p->d_zsymk;
  sa.lam = p->d_lam;
  sa.twiddle = p->d_tw;
  sa.tw_count = p->tw_count;
  sa.split_out = p->tc ? tc_split_buffer(p->tc) : nullptr;
  sa.npieces = p->precision == FDETD_PREC_BF16X3 ? 2 : 3;
  sa.split_kstages = p->tc ? tc_split_kstages(p->tc) : 0;
  sa.err = p->d_err;
  sa.src = p->d_src;
  sa.Nz = p->Nz;
  sa.logNz = p->logNz;
  sa.n = p->Nr;
  sa.dt = p->dt;
  sa.hasJ = hasJ;
  sa.phases = p->profiling && p->d_waits ? p->d_waits + 16 : nullptr;
  return sa;
}

// The three stages of one step (projection, z transforms with the exact rotation, back-projection).
static int stage_project(fdetd_plan_s* p, void* fields, const void* J, cudaStream_t st) {
  const int prec = p->precision == FDETD_PREC_FP64 ? 0 : 1;
  cudaError_t e;
  prof_mark(p, 0, true, st);
  if (p->tc) {
    e = tc_project(p->tc, fields, J, p->d_coef, st);
  } else {
    ProjArgs pa{fields, J, p->d_P, p->d_coef, p->Nz, p->Nr};
    e = launch_project_simt(pa, p->nmodes, prec, st);
  }
  prof_mark(p, 0, false, st);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("projection: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

static int stage_spectral(fdetd_plan_s* p, bool hasJ, cudaStream_t st) {
  const int prec = p->precision == FDETD_PREC_FP64 ? 0 : 1;
  const SpectralArgs sa = spectral_args(p, hasJ);
  prof_mark(p, 1, true, st);
  // FP32 data, Nz a power of two up to 4096: the kernel specialised on Nz; other powers of two: the general
  // power-of-two kernel; other 7-smooth lengths: the mixed-radix kernel
  cudaError_t e;
  if (p->columns) {
    e = launch_spectral_columns(sa, p->nmodes, prec, p->tc != nullptr, st);
  } else if (!is_pow2(p->Nz)) {
    MixedRadices mr;
    mr.nst = spectral_radices(p->Nz, prec, mr.rad);
    e = launch_spectral_mixed(sa, mr, p->nmodes, prec, p->tc != nullptr, st);
  } else if (prec == 1 && sa.zsymk) {
    e = launch_spectral32(sa, p->nmodes, p->tc != nullptr, st);
  } else {
    e = launch_spectral(sa, p->nmodes, prec, p->tc != nullptr, st);
  }
  prof_mark(p, 1, false, st);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("spectral: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

static int stage_backproject(fdetd_plan_s* p, void* fields, cudaStream_t st) {
  const int prec = p->precision == FDETD_PREC_FP64 ? 0 : 1;
  cudaError_t e;
  prof_mark(p, 2, true, st);
  if (p->tc) {
    e = tc_backproject(p->tc, fields, st);
  } else {
    BackArgs ba{fields, p->d_Q, p->d_coef, p->Nz, p->Nr};
    e = launch_backproject_simt(ba, p->nmodes, prec, st);
  }
  prof_mark(p, 2, false, st);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("back-projection: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

static int stagger_current(fdetd_plan_s* p, const void* J, cudaStream_t st);

extern "C" int fdetd_step(fdetd_plan_t p, void* fields, const void* J, int nsteps, void* stream) {
  if (!p) return fail(FDETD_ERR_ARG, "plan is null");
  if (!fields) return fail(FDETD_ERR_ARG, "fields is null");
  if (nsteps < 0) return fail(FDETD_ERR_ARG, "nsteps < 0");
  if (((uintptr_t)fields & 15) || ((uintptr_t)J & 15)) return fail(FDETD_ERR_ARG, "pointers must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  if (p->j_primary && J && nsteps > 0) {
    // J_rho deposited on the primary grid: S_rho^(-, mA) into the plan's copy, which the steps then use
    const int rc = stagger_current(p, J, st);
    if (rc) return rc;
    J = p->d_jstag;
  }
  for (int s = 0; s < nsteps; ++s) {
    int rc = stage_project(p, fields, J, st);
    if (!rc) rc = stage_spectral(p, J != nullptr, st);
    if (!rc) rc = stage_backproject(p, fields, st);
    if (rc) return rc;
  }
  return FDETD_OK;
}

// ---- autotuning of the tensor-core tile shapes and schedules

static float time_launches(const std::function<cudaError_t()>& f, cudaStream_t st, int reps, cudaError_t* err) {
  cudaEvent_t a = nullptr, b = nullptr;
  float ms = -1.f;
  *err = cudaEventCreate(&a);
  if (*err == cudaSuccess) *err = cudaEventCreate(&b);
  if (*err == cudaSuccess) *err = f();  // warm-up
  if (*err == cudaSuccess) *err = cudaEventRecord(a, st);
  for (int r = 0; *err == cudaSuccess && r < reps; ++r) *err = f();
  if (*err == cudaSuccess) *err = cudaEventRecord(b, st);
  if (*err == cudaSuccess) *err = cudaEventSynchronize(b);
  if (*err == cudaSuccess) *err = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return ms / reps;
}

// Times every candidate (N tile and tile order of each kernel) on the instances' own data and
// returns the fastest.  The projection candidates read the fields and overwrite only the plans'
// coefficient scratch; the back-projection candidates write into one scratch array (sized for the
// largest instance and shared by all of them), so the caller's fields are never modified.
static int tune_group(std::vector<fdetd_plan_s*>& plans, const std::vector<void*>& fields,
                      const std::vector<const void*>& J, cudaStream_t st, TcConfig* best, float* best_ms) {
  const int count = (int)plans.size();
  std::vector<TcPlan*> tp(count);
  std::vector<const void*> fp(count);
  size_t maxb = 0;
  for (int k = 0; k < count; ++k) {
    tp[k] = plans[k]->tc;
    fp[k] = fields[k];
    maxb = std::max(maxb, (size_t)plans[k]->nmodes * 6 * plans[k]->Nz * plans[k]->Nr * 8);
  }
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, maxb) != cudaSuccess) return fail(FDETD_ERR_OOM, "autotune scratch allocation failed");
  TcConfig cur = tc_default_config(tc_pieces(tp[0]));
  float bp = 1e30f, bb = 1e30f;
  int rc = FDETD_OK;
  for (int which = 0; which < 2 && rc == FDETD_OK; ++which)
    for (int tn : {128, 256})
      for (int sched : {0, 1}) {
        if (rc != FDETD_OK) break;
        TcConfig c = cur;
        if (which == 0) {
          c.tn_p = tn;
          c.sched_p = sched;
        } else {
          c.tn_b = tn;
          c.sched_b = sched;
        }
        if (!tc_config_valid(tp.data(), count, c)) continue;
        TcGroup* G = nullptr;
        cudaError_t e = tc_group_create(&G, tp.data(), fp.data(), J.data(), count, c);
        if (e != cudaSuccess) {
          rc = fail(FDETD_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
          break;
        }
        for (int k = 0; k < count; ++k) {
          tc_group_set_coef(G, k, plans[k]->d_coef);
          if (which == 1) tc_group_set_fields(G, k, scratch);
        }
        const float ms = time_launches(
            [&]() { return which == 0 ? tc_group_project(G, st) : tc_group_backproject(G, st); }, st, 3, &e);
        tc_group_destroy(G);
        if (e != cudaSuccess) {
          rc = fail(FDETD_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
          break;
        }
        if (which == 0 && ms < bp) {
          bp = ms;
          cur.tn_p = tn;
          cur.sched_p = sched;
        }
        if (which == 1 && ms < bb) {
          bb = ms;
          cur.tn_b = tn;
          cur.sched_b = sched;
        }
      }
  cudaFree(scratch);
  if (rc) return rc;
  *best = cur;
  if (best_ms) {
    best_ms[0] = bp;
    best_ms[1] = bb;
  }
  return FDETD_OK;
}

extern "C" int fdetd_plan_autotune(fdetd_plan_t p, const void* fields, const void* J, void* stream, double* ms) {
  if (!p || !fields) return fail(FDETD_ERR_ARG, "null argument");
  if (((uintptr_t)fields & 15) || ((uintptr_t)J & 15)) return fail(FDETD_ERR_ARG, "pointers must be 16-byte aligned");
  if (!p->tc) return FDETD_OK;
  std::vector<fdetd_plan_s*> pl{p};
  std::vector<void*> f{const_cast<void*>(fields)};
  std::vector<const void*> j{J};
  TcConfig best;
  float bms[2] = {0, 0};
  int rc = tune_group(pl, f, j, (cudaStream_t)stream, &best, bms);
  if (rc) return rc;
  if (tc_plan_set_config(p->tc, best) != cudaSuccess) return fail(FDETD_ERR_CUDA, "autotune: invalid configuration");
  if (ms) {
    ms[0] = bms[0];
    ms[1] = bms[1];
  }
  return FDETD_OK;
}

extern "C" int fdetd_plan_tile_config(fdetd_plan_t p, int* cfg) {
  if (!p || !cfg) return fail(FDETD_ERR_ARG, "null argument");
  if (!p->tc) return fail(FDETD_ERR_ARG, "not a tensor-core plan");
  const TcConfig c = tc_plan_config(p->tc);
  cfg[0] = c.tn_p;
  cfg[1] = c.tn_b;
  cfg[2] = c.sched_p;
  cfg[3] = c.sched_b;
  return FDETD_OK;
}

extern "C" int fdetd_plan_set_tile_config(fdetd_plan_t p, const int* cfg) {
  if (!p || !cfg) return fail(FDETD_ERR_ARG, "null argument");
  if (!p->tc) return fail(FDETD_ERR_ARG, "not a tensor-core plan");
  const TcConfig c{cfg[0], cfg[1], cfg[2], cfg[3]};
  if (tc_plan_set_config(p->tc, c) != cudaSuccess) return fail(FDETD_ERR_ARG, "invalid tile configuration");
  return FDETD_OK;
}

extern "C" int fdetd_destagger(fdetd_plan_t p, const void* fields, void* out, void* stream) {
  if (!p || !fields || !out) return fail(FDETD_ERR_ARG, "null argument");
  if (fields == out) return fail(FDETD_ERR_ARG, "out must not alias fields");
  const size_t elt = p->precision == FDETD_PREC_FP64 ? 16 : 8;
  const size_t bytes = (size_t)p->nmodes * 6 * p->Nz * p->Nr * elt;
  const char *a = (const char*)fields, *b = (const char*)out;
  if (a < b + bytes && b < a + bytes) return fail(FDETD_ERR_ARG, "out must not overlap fields");
  cudaError_t e = launch_destagger(fields, out, p->Nz, p->Nr, p->order, p->modes.data(), p->nmodes,
                                   p->precision == FDETD_PREC_FP64, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("destagger: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

// Lagrange weights of the half point rho_k + dr / 2 on the 2 ND primary nodes k - ND + 1 .. k + ND (the
// downstagger S_rho^(-, mA) of Eq. spatialAM_staggerS)
static void half_point_weights(int ND, double* w) {
  for (int i = -ND + 1; i <= ND; ++i) {
    double num = 1.0, den = 1.0;
    for (int l = -ND + 1; l <= ND; ++l)
      if (l != i) {
        num *= 0.5 - l;
        den *= (double)(i - l);
      }
    w[i + ND - 1] = num / den;
  }
}

// J with J_rho on the primary grid -> the plan's scratch with J_rho downstaggered (FDETD_FLAG_J_ON_PRIMARY)
static int stagger_current(fdetd_plan_s* p, const void* J, cudaStream_t st) {
  CurParams cp;
  memset(&cp, 0, sizeof(cp));
  cp.J = J;
  cp.out = p->d_jstag;
  cp.stagger_only = 1;
  cp.dr = p->dr;
  cp.Nz = p->Nz;
  cp.n = p->Nr;
  cp.ND = p->order / 2;
  cp.nm = p->nmodes;
  for (int i = 0; i < p->nmodes; ++i) cp.m[i] = p->modes[i];
  half_point_weights(cp.ND, cp.w);
  cudaError_t e = launch_current(cp, p->precision == FDETD_PREC_FP64, st);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("J_rho downstagger: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

extern "C" int fdetd_current_correct(fdetd_plan_t p, const void* J, const void* rho_xy, void* J_out, void* stream) {
  if (!p || !J || !rho_xy || !J_out) return fail(FDETD_ERR_ARG, "null argument");
  const size_t elt = p->precision == FDETD_PREC_FP64 ? 16 : 8;
  const size_t jb = (size_t)p->nmodes * 3 * p->Nz * p->Nr * elt, rb = (size_t)p->nmodes * p->Nz * p->Nr * elt;
  auto overlap = [](const void* a, size_t na, const void* b, size_t nb) {
    const char *x = (const char*)a, *y = (const char*)b;
    return x < y + nb && y < x + na;
  };
  if (overlap(J_out, jb, J, jb) || overlap(J_out, jb, rho_xy, rb)) return fail(FDETD_ERR_ARG, "J_out must not overlap the inputs");
  const int n = p->Nr, ND = p->order / 2, W = 2 * ND + 1;
  const size_t nm = (size_t)p->nmodes;
  if (!p->d_cur) {
    // tables in the order the kernel reads them (array-major, [mode] within each); FP32 plans get each
    // value as a float pair hi + lo so the device can work in double-float arithmetic
    const size_t o_dm = nm * W * n, o_lo = 2 * o_dm, o_up = o_lo + nm * n * ND, o_ip = o_up + nm * n * ND,
                 o_mr = o_ip + nm * n, total = o_mr + nm * n;
    std::vector<double> all(total, 0.0);
    for (int i = 0; i < p->nmodes; ++i) {
      std::vector<double> divp, dm, lo, up;
      const int rc = current_bands(n, p->order, p->dr, p->modes[i], divp, dm, lo, up);
      if (rc) return fail(FDETD_ERR_EIG, "current correction: vanishing pivot of the radial Laplacian");
      for (int k = 0; k < n; ++k) {
        for (int t = 0; t < W; ++t) {
          all[(size_t)i * W * n + (size_t)t * n + k] = -divp[(size_t)k * W + t];
          all[o_dm + (size_t)i * W * n + (size_t)t * n + k] = dm[(size_t)k * W + t];
        }
        for (int d = 1; d <= ND; ++d) {
          all[o_lo + ((size_t)i * n + k) * ND + d - 1] = -lo[(size_t)k * ND + d - 1];
          all[o_up + ((size_t)i * n + k) * ND + d - 1] = -up[(size_t)k * (ND + 1) + d];
        }
        all[o_ip + (size_t)i * n + k] = 1.0 / up[(size_t)k * (ND + 1)];
        all[o_mr + (size_t)i * n + k] = (double)p->modes[i] / ((k + 0.5) * p->dr);
      }
    }
    if (p->precision != FDETD_PREC_FP64)
      for (double& v : all) {
        const float h = (float)v, l = (float)(v - (double)h);
        float pair[2] = {h, l};
        memcpy(&v, pair, 8);
      }
    size_t dummy = 0;
    cudaError_t e = upload(&p->d_cur, all.data(), all.size() * 8, dummy);
    if (e != cudaSuccess) {
      if (p->d_cur) cudaFree(p->d_cur);
      p->d_cur = nullptr;
      return fail(FDETD_ERR_OOM, std::string("current correction: ") + cudaGetErrorString(e));
    }
    p->bytes += all.size() * 8;
  }
  CurParams cp;
  memset(&cp, 0, sizeof(cp));
  cp.J = J;
  cp.rho_xy = rho_xy;
  cp.out = J_out;
  cp.bands = p->d_cur;
  cp.dr = p->dr;
  cp.Nz = p->Nz;
  cp.n = n;
  cp.ND = ND;
  cp.nm = p->nmodes;
  for (int i = 0; i < p->nmodes; ++i) cp.m[i] = p->modes[i];
  half_point_weights(ND, cp.w);
  cudaError_t e = launch_current(cp, p->precision == FDETD_PREC_FP64, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("current correction: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

extern "C" int fdetd_current_host_bands(int Nr, int order, double dr, int m, double* divp, double* dm, double* lo,
                                        double* up) {
  std::vector<double> a, b, c, d;
  const int rc = current_bands(Nr, order, dr, m, a, b, c, d);
  if (rc == 1) return fail(FDETD_ERR_ARG, "bad order or Nr");
  if (rc == 2) return fail(FDETD_ERR_EIG, "vanishing pivot");
  if (divp) std::copy(a.begin(), a.end(), divp);
  if (dm) std::copy(b.begin(), b.end(), dm);
  if (lo) std::copy(c.begin(), c.end(), lo);
  if (up) std::copy(d.begin(), d.end(), up);
  return FDETD_OK;
}

extern "C" int fdetd_step_host(fdetd_plan_t p, void* host_fields, const void* host_J, int nsteps, void* stream) {
  if (!p || !host_fields) return fail(FDETD_ERR_ARG, "null argument");
  const size_t elt = p->precision == FDETD_PREC_FP64 ? 16 : 8;
  const size_t fb = (size_t)p->nmodes * 6 * p->Nz * p->Nr * elt, jb = (size_t)p->nmodes * 3 * p->Nz * p->Nr * elt;
  const size_t need = fb + (host_J ? jb : 0);
  cudaStream_t st = (cudaStream_t)stream;
  if (p->hostio_bytes < need) {
    if (p->d_hostio) cudaFree(p->d_hostio);
    p->d_hostio = nullptr;
    p->hostio_bytes = 0;
    if (cudaMalloc(&p->d_hostio, need) != cudaSuccess) return fail(FDETD_ERR_OOM, "staging allocation failed");
    p->hostio_bytes = need;
  }
  char* dF = (char*)p->d_hostio;
  char* dJ = host_J ? dF + fb : nullptr;
  cudaError_t e = cudaMemcpyAsync(dF, host_fields, fb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && host_J) e = cudaMemcpyAsync(dJ, host_J, jb, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("h2d: ") + cudaGetErrorString(e));
  int rc = fdetd_step(p, dF, dJ, nsteps, stream);
  if (rc) return rc;
  e = cudaMemcpyAsync(host_fields, dF, fb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("d2h: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

extern "C" size_t fdetd_plan_device_bytes(fdetd_plan_t p) { return p ? p->bytes : 0; }

extern "C" int fdetd_plan_launches_per_step(fdetd_plan_t p) {
  if (!p) return 0;
  // + the source kernel of the two-kernel form, or the three launches of the column-split form
  return (p->tc ? tc_launches_per_step(p->tc) : 2) + (p->columns ? 3 : (p->d_src ? 2 : 1));
}

extern "C" int fdetd_plan_status(fdetd_plan_t p, void* stream) {
  if (!p) return fail(FDETD_ERR_ARG, "plan is null");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  int flag = 0;
  e = cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, cudaGetErrorString(e));
  if (flag) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return fail(FDETD_ERR_TIMEOUT, "a kernel's bounded wait expired (stage code " + std::to_string(flag) + ")");
  }
  return FDETD_OK;
}

extern "C" int fdetd_stream_status(fdetd_plan_t p, void* stream) { return fdetd_plan_status(p, stream); }

extern "C" int fdetd_plan_set_wait_limit(fdetd_plan_t p, long long polls) {
  if (!p) return fail(FDETD_ERR_ARG, "plan is null");
  if (!p->tc) return fail(FDETD_ERR_UNSUPPORTED, "only the tensor-core pipelines have bounded waits");
  tc_set_wait_limit(p->tc, polls);
  return FDETD_OK;
}

// pipeline counters: 8 words of the projection, 8 of the back-projection, 8 of the spectral kernel
constexpr int kWaitWords = 24;

extern "C" int fdetd_plan_set_profiling(fdetd_plan_t p, int on) {
  if (!p) return fail(FDETD_ERR_ARG, "plan is null");
  prof_collect(p);
  p->profiling = on != 0;
  for (int k = 0; k < 3; ++k) {
    p->kern_ms[k] = 0;
    p->kern_calls[k] = 0;
  }
  if (on) {
    cudaError_t e = p->d_waits ? cudaSuccess : cudaMalloc(&p->d_waits, kWaitWords * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(p->d_waits, 0, kWaitWords * sizeof(unsigned long long));
    if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("pipeline counters: ") + cudaGetErrorString(e));
  }
  if (p->tc) tc_set_waits(p->tc, on ? p->d_waits : nullptr);
  return FDETD_OK;
}

static int read_waits(const unsigned long long* d, unsigned long long* out) {
  if (!d) {
    std::fill(out, out + kWaitWords, 0ull);
    return FDETD_OK;
  }
  cudaError_t e = cudaMemcpy(out, d, kWaitWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("pipeline counters: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

extern "C" int fdetd_plan_pipeline_waits(fdetd_plan_t p, unsigned long long* out) {
  if (!p || !out) return fail(FDETD_ERR_ARG, "null argument");
  return read_waits(p->d_waits, out);
}

extern "C" int fdetd_plan_kernel_times(fdetd_plan_t p, double* ms, long* calls) {
  if (!p || !ms || !calls) return fail(FDETD_ERR_ARG, "null argument");
  prof_collect(p);
  for (int k = 0; k < 3; ++k) {
    ms[k] = p->kern_ms[k];
    calls[k] = p->kern_calls[k];
  }
  return FDETD_OK;
}

extern "C" int fdetd_plan_destroy(fdetd_plan_t p) {
  plan_free(p);
  return FDETD_OK;
}

extern "C" int fdetd_host_tables(int Nz, int Nr, int m, int order, double dz, double dr, double dt, double* PE,
                                 double* PB, double* QE, double* QB, double* lam, double* mu, uint8_t* tm_live,
                                 uint8_t* te_live, double* kappa2, double* sp, double* sm) {
  HostPlan hp;
  std::string msg;
  int rc = build_host_plan(hp, Nz, Nr, &m, 1, order, dz, dr, dt, msg);
  if (rc) return fail(rc == 4 ? FDETD_ERR_EIG : FDETD_ERR_ARG, msg);
  const ModePlan& mp = hp.mp[0];
  auto cp = [](double* dst, const std::vector<double>& v) {
    if (dst) std::copy(v.begin(), v.end(), dst);
  };
  cp(PE, mp.PE);
  cp(PB, mp.PB);
  cp(QE, mp.QE);
  cp(QB, mp.QB);
  cp(lam, mp.lam);
  cp(mu, mp.mu);
  cp(kappa2, hp.kappa2);
  if (tm_live) std::copy(mp.tm_live.begin(), mp.tm_live.end(), tm_live);
  if (te_live) std::copy(mp.te_live.begin(), mp.te_live.end(), te_live);
  for (int q = 0; q < Nz; ++q) {
    if (sp) { sp[2 * q] = hp.sp_re[q]; sp[2 * q + 1] = hp.sp_im[q]; }
    if (sm) { sm[2 * q] = hp.sm_re[q]; sm[2 * q + 1] = hp.sm_im[q]; }
  }
  return FDETD_OK;
}

extern "C" int fdetd_host_spectral_order(int Nz, int precision, int* kz) {
  int rad[MixedRadices::kMax];
  if (!kz || Nz < 2 || !spectral_radices(Nz, precision == FDETD_PREC_FP64 ? 0 : 1, rad))
    return fail(FDETD_ERR_ARG, "Nz must be >= 2 with no prime factor above 7");
  spectral_positions(Nz, precision == FDETD_PREC_FP64 ? 0 : 1, kz);
  return FDETD_OK;
}

extern "C" int fdetd_host_spectral_radices(int Nz, int precision, int* rad) {
  if (!rad || Nz < 2) return -FDETD_ERR_ARG;
  return spectral_radices(Nz, precision == FDETD_PREC_FP64 ? 0 : 1, rad);
}

extern "C" int fdetd_plan_cache_set_limit(size_t bytes) {
  mode_cache_set_limit(bytes);
  return FDETD_OK;
}

extern "C" int fdetd_plan_cache_warm(int Nr, int order, double dr, const int* modes, int nmodes) {
  if (order < 2 || order > 32 || (order & 1) || Nr < order / 2 + 2 || !(dr > 0) || nmodes < 1 || !modes)
    return fail(FDETD_ERR_ARG, "invalid order, Nr, dr or modes");
  for (int i = 0; i < nmodes; ++i) {
    if (modes[i] < 0 || modes[i] > 64) return fail(FDETD_ERR_ARG, "mode numbers must be 0..64");
    std::string msg;
    const int rc = mode_cache_warm(Nr, order, dr, modes[i], msg);
    if (rc) return fail(rc == 4 ? FDETD_ERR_EIG : FDETD_ERR_ARG, msg);
  }
  return FDETD_OK;
}

extern "C" int fdetd_plan_cache_stats(size_t* bytes, size_t* limit, int* entries, uint64_t* hits,
                                      uint64_t* misses) {
  mode_cache_stats(bytes, limit, entries, hits, misses);
  return FDETD_OK;
}

extern "C" int fdetd_host_plan_digest(int Nz, int Nr, const int* modes, int nmodes, int order, double dz, double dr,
                                      double dt, double* digest) {
  if (!modes || nmodes < 1 || !digest) return fail(FDETD_ERR_ARG, "null modes or digest");
  HostPlan hp;
  std::string msg;
  const int rc = build_host_plan(hp, Nz, Nr, modes, nmodes, order, dz, dr, dt, msg);
  if (rc) return fail(rc == 4 ? FDETD_ERR_EIG : FDETD_ERR_ARG, msg);
  auto sum = [](const std::vector<double>& v) {
    double a = 0.0;
    for (double x : v) a += x;  // left to right
    return a;
  };
  for (int i = 0; i < nmodes; ++i) {
    const ModePlan& mp = hp.mp[i];
    double* d = digest + 6 * i;
    d[0] = sum(mp.PE);
    d[1] = sum(mp.PB);
    d[2] = sum(mp.QE);
    d[3] = sum(mp.QB);
    d[4] = sum(mp.lam);
    d[5] = sum(mp.mu);
  }
  return FDETD_OK;
}

extern "C" int fdetd_host_coeffs(int kind, int order, double* out) {
  if (order < 2 || order > 32 || (order & 1) || !out) return fail(FDETD_ERR_ARG, "bad order or null out");
  std::vector<double> v;
  if (kind == 0) v = staggered_coeffs(order);
  else if (kind == 1) v = centred_d1_coeffs(order);
  else if (kind == 2) {
    double e0 = 0;
    std::vector<double> e = centred_d2_coeffs(order, &e0);
    v.push_back(e0);
    v.insert(v.end(), e.begin(), e.end());
  } else if (kind == 3) v = axis_coeffs(order / 2);
  else return fail(FDETD_ERR_ARG, "unknown kind");
  std::copy(v.begin(), v.end(), out);
  return (int)v.size();
}

// ------------------------------------------------------------------ batches of instances

struct fdetd_batch_s {
  struct Inst {
    fdetd_plan_s* plan;
    void* fields;
    const void* J;
  };
  std::vector<Inst> inst;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int steps = 0;
  int autotune = 1;
  // tensor-core instances of one precision share grouped projection / back-projection launches
  struct Group {
    TcGroup* g = nullptr;
    std::vector<int> members;
    TcConfig cfg;
    float tuned_ms[2] = {0, 0};
  };
  std::vector<Group> groups;
  // stage timing: per captured step, events before the grouped projections, after them, after the
  // spectral branches have joined, after the grouped back-projections (recorded as graph nodes)
  int profiling = 0;
  unsigned long long* d_waits = nullptr;  // pipeline cycle counters of the grouped kernels (profiling)
  // host-buffer step: the instances split into parts with a one-step graph each, so that the copies of one part
  // overlap the compute of another (built at the first fdetd_batch_step_host, dropped with the main graph)
  struct Part {
    std::vector<int> members;
    std::vector<Group> groups;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t in = nullptr, done = nullptr;
  };
  std::vector<Part> parts;
  int host_parts = 16;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  std::vector<cudaEvent_t> stage_ev;
  double stage_ms[3] = {0, 0, 0};
  long stage_calls = 0;
};

static void batch_release_events(fdetd_batch_s* b) {
  for (auto e : b->stage_ev) cudaEventDestroy(e);
  b->stage_ev.clear();
}

static void batch_release_parts(fdetd_batch_s* b) {
  for (auto& P : b->parts) {
    if (P.exec) cudaGraphExecDestroy(P.exec);
    if (P.graph) cudaGraphDestroy(P.graph);
    for (auto& g : P.groups)
      if (g.g) tc_group_destroy(g.g);
    if (P.in) cudaEventDestroy(P.in);
    if (P.done) cudaEventDestroy(P.done);
  }
  b->parts.clear();
}

static void batch_release_graph(fdetd_batch_s* b) {
  batch_release_parts(b);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  for (auto& g : b->groups)
    if (g.g) tc_group_destroy(g.g);
  b->groups.clear();
}

extern "C" int fdetd_batch_create(fdetd_batch_t* out) {
  if (!out) return fail(FDETD_ERR_ARG, "out is null");
  fdetd_batch_s* b = new fdetd_batch_s();
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return fail(FDETD_ERR_CUDA, "event creation failed");
  }
  *out = b;
  return FDETD_OK;
}

extern "C" int fdetd_batch_add(fdetd_batch_t b, fdetd_plan_t plan, void* fields, const void* J, int* index) {
  if (!b || !plan || !fields) return fail(FDETD_ERR_ARG, "null argument");
  if (((uintptr_t)fields & 15) || ((uintptr_t)J & 15)) return fail(FDETD_ERR_ARG, "pointers must be 16-byte aligned");
  for (auto& i : b->inst)
    if (i.plan == plan) return fail(FDETD_ERR_ARG, "a plan may appear once per batch (its scratch is not shared)");
  if (plan->j_primary && J)
    return fail(FDETD_ERR_ARG, "a J_ON_PRIMARY plan steps with fdetd_step (a batch takes J on the Yee locations)");
  cudaStream_t s;
  cudaEvent_t e;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(FDETD_ERR_CUDA, "stream");
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaStreamDestroy(s);
    return fail(FDETD_ERR_CUDA, "event");
  }
  b->inst.push_back({plan, fields, J});
  b->side.push_back(s);
  b->join.push_back(e);
  batch_release_graph(b);
  if (index) *index = (int)b->inst.size() - 1;
  return FDETD_OK;
}

// Groups the tensor-core instances by precision (at most kMaxGroupInstances per group), picks each
// group's tile shapes and schedules (autotuned on the instances' data unless disabled), and
// captures `nsteps` steps: per step, one grouped projection launch per group, every instance's
// spectral kernel on its own branch, one grouped back-projection launch per group.  Instances on
// the CUDA-core paths run their own step sequence on concurrent branches.
// Tensor-core groups over the instances `ids`: by precision, at most kMaxGroupInstances per group; tile shapes
// autotuned on the instances' data, or taken from `like` (a group list of the same batch) when given.
static int build_groups(fdetd_batch_s* b, const std::vector<int>& ids_all, cudaStream_t s0,
                        const std::vector<fdetd_batch_s::Group>* like, std::vector<fdetd_batch_s::Group>& out) {
  for (int np : {2, 3}) {
    std::vector<int> ids;
    for (int k : ids_all)
      if (b->inst[k].plan->tc && tc_pieces(b->inst[k].plan->tc) == np) ids.push_back(k);
    for (size_t c0 = 0; c0 < ids.size(); c0 += kMaxGroupInstances) {
      fdetd_batch_s::Group G;
      G.members.assign(ids.begin() + c0, ids.begin() + std::min(ids.size(), c0 + (size_t)kMaxGroupInstances));
      std::vector<fdetd_plan_s*> pl;
      std::vector<TcPlan*> tp;
      std::vector<void*> f;
      std::vector<const void*> fc, j;
      for (int k : G.members) {
        pl.push_back(b->inst[k].plan);
        tp.push_back(b->inst[k].plan->tc);
        f.push_back(b->inst[k].fields);
        fc.push_back(b->inst[k].fields);
        j.push_back(b->inst[k].J);
      }
      G.cfg = tc_default_config(np);
      bool found = false;
      if (like)
        for (const auto& L : *like)
          if (!found && L.g && tc_pieces(b->inst[L.members[0]].plan->tc) == np) {
            G.cfg = L.cfg;
            found = true;
          }
      if (!found && b->autotune) {
        int rc = tune_group(pl, f, j, s0, &G.cfg, G.tuned_ms);
        if (rc) return rc;
      }
      cudaError_t e = tc_group_create(&G.g, tp.data(), fc.data(), j.data(), (int)G.members.size(), G.cfg);
      if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("batch group: ") + cudaGetErrorString(e));
      for (size_t k = 0; k < G.members.size(); ++k) tc_group_set_coef(G.g, (int)k, pl[k]->d_coef);
      out.push_back(G);
    }
  }
  return FDETD_OK;
}

// Captures `nsteps` steps of the instances `ids` (their groups already built) into a graph: per step, one grouped
// projection launch per group, every instance's spectral kernel on its own branch, one grouped back-projection
// launch per group; CUDA-core instances run their own step sequence on a branch.  With `marks`, event nodes
// stamp each step's stage boundaries (marks[4 step + 0..3]).
static int capture_steps(fdetd_batch_s* b, const std::vector<int>& ids, std::vector<fdetd_batch_s::Group>& groups,
                         int nsteps, cudaStream_t s0, const std::vector<cudaEvent_t>* marks, cudaGraph_t* graph_out,
                         cudaGraphExec_t* exec_out) {
  *graph_out = nullptr;
  *exec_out = nullptr;
  cudaStream_t cap = s0;
  cudaStream_t own = nullptr;
  if (!cap) {  // the legacy default stream cannot be captured
    if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) return fail(FDETD_ERR_CUDA, "stream");
    cap = own;
  }
  // recorded as event nodes of the graph (external), so that each replay stamps them
  auto mark = [&](int step, int k) -> cudaError_t {
    return marks ? cudaEventRecordWithFlags((*marks)[(size_t)4 * step + k], cap, cudaEventRecordExternal)
                 : cudaSuccess;
  };
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int rc = FDETD_OK;
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, cap);
  std::vector<int> simt;
  for (int k : ids) {
    if (e != cudaSuccess || rc != FDETD_OK) break;
    if (b->inst[k].plan->tc) continue;
    simt.push_back(k);
    e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
    if (e == cudaSuccess) rc = fdetd_step(b->inst[k].plan, b->inst[k].fields, b->inst[k].J, nsteps, b->side[k]);
  }
  for (int s = 0; s < nsteps && e == cudaSuccess && rc == FDETD_OK; ++s) {
    e = mark(s, 0);
    for (auto& G : groups) {
      if (e != cudaSuccess) break;
      e = tc_group_project(G.g, cap);
    }
    if (e == cudaSuccess) e = mark(s, 1);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, cap);
    for (auto& G : groups)
      for (int k : G.members) {
        if (e != cudaSuccess || rc != FDETD_OK) break;
        e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
        if (e == cudaSuccess) rc = stage_spectral(b->inst[k].plan, b->inst[k].J != nullptr, b->side[k]);
        if (e == cudaSuccess && rc == FDETD_OK) e = cudaEventRecord(b->join[k], b->side[k]);
        if (e == cudaSuccess && rc == FDETD_OK) e = cudaStreamWaitEvent(cap, b->join[k], 0);
      }
    if (e == cudaSuccess && rc == FDETD_OK) e = mark(s, 2);
    for (auto& G : groups) {
      if (e != cudaSuccess || rc != FDETD_OK) break;
      e = tc_group_backproject(G.g, cap);
    }
    if (e == cudaSuccess && rc == FDETD_OK) e = mark(s, 3);
  }
  for (int k : simt) {
    if (e != cudaSuccess || rc != FDETD_OK) break;
    e = cudaEventRecord(b->join[k], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, b->join[k], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  if (own) cudaStreamDestroy(own);
  if (rc != FDETD_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e == cudaSuccess) e = e2;
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(FDETD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  *graph_out = g;
  *exec_out = ex;
  return FDETD_OK;
}

extern "C" int fdetd_batch_capture(fdetd_batch_t b, int nsteps, void* stream) {
  if (!b || nsteps < 1) return fail(FDETD_ERR_ARG, "bad batch or nsteps");
  if (b->inst.empty()) return fail(FDETD_ERR_ARG, "empty batch");
  for (auto& i : b->inst)
    if (i.plan->profiling) return fail(FDETD_ERR_ARG, "turn profiling off before capturing");
  batch_release_graph(b);
  cudaStream_t s0 = (cudaStream_t)stream;
  std::vector<int> all(b->inst.size());
  for (size_t k = 0; k < all.size(); ++k) all[k] = (int)k;
  // groups are built and tuned before the capture: tile tables are uploaded synchronously
  int rc = build_groups(b, all, s0, nullptr, b->groups);
  if (rc == FDETD_OK && b->profiling) {
    cudaError_t e2 = b->d_waits ? cudaSuccess : cudaMalloc(&b->d_waits, kWaitWords * sizeof(unsigned long long));
    if (e2 == cudaSuccess) e2 = cudaMemset(b->d_waits, 0, kWaitWords * sizeof(unsigned long long));
    if (e2 != cudaSuccess) rc = fail(FDETD_ERR_CUDA, std::string("pipeline counters: ") + cudaGetErrorString(e2));
    for (auto& G : b->groups) tc_group_set_waits(G.g, b->d_waits);
  }
  if (rc != FDETD_OK) {
    batch_release_graph(b);
    return rc;
  }
  if (cudaStreamSynchronize(s0) != cudaSuccess) return fail(FDETD_ERR_CUDA, "batch: stream error before capture");
  batch_release_events(b);
  if (b->profiling) {
    b->stage_ev.resize((size_t)4 * nsteps, nullptr);
    for (auto& ev : b->stage_ev)
      if (cudaEventCreate(&ev) != cudaSuccess) {
        batch_release_events(b);
        return fail(FDETD_ERR_CUDA, "batch: timing event creation failed");
      }
  }
  rc = capture_steps(b, all, b->groups, nsteps, s0, b->profiling ? &b->stage_ev : nullptr, &b->graph, &b->exec);
  if (rc != FDETD_OK) return rc;
  b->steps = nsteps;
  return FDETD_OK;
}

extern "C" int fdetd_batch_set_autotune(fdetd_batch_t b, int on) {
  if (!b) return fail(FDETD_ERR_ARG, "batch is null");
  b->autotune = on != 0;
  batch_release_graph(b);
  return FDETD_OK;
}

extern "C" int fdetd_batch_group_info(fdetd_batch_t b, int gi, int* info, double* ms) {
  if (!b || !info) return -FDETD_ERR_ARG;
  if (gi < 0 || gi >= (int)b->groups.size()) return (int)b->groups.size();
  const auto& G = b->groups[gi];
  info[0] = G.cfg.tn_p;
  info[1] = G.cfg.tn_b;
  info[2] = G.cfg.sched_p;
  info[3] = G.cfg.sched_b;
  info[4] = (int)G.members.size();
  info[5] = tc_group_tiles(G.g, 0);
  info[6] = tc_group_tiles(G.g, 1);
  if (ms) {
    ms[0] = G.tuned_ms[0];
    ms[1] = G.tuned_ms[1];
  }
  return (int)b->groups.size();
}

extern "C" int fdetd_batch_launch(fdetd_batch_t b, void* stream) {
  if (!b || !b->exec) return fail(FDETD_ERR_ARG, "batch has no captured graph");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

extern "C" int fdetd_batch_set_profiling(fdetd_batch_t b, int on) {
  if (!b) return fail(FDETD_ERR_ARG, "batch is null");
  b->profiling = on != 0;
  b->stage_ms[0] = b->stage_ms[1] = b->stage_ms[2] = 0;
  b->stage_calls = 0;
  batch_release_graph(b);
  batch_release_events(b);
  return FDETD_OK;
}

extern "C" int fdetd_batch_collect_stage_times(fdetd_batch_t b) {
  if (!b || !b->exec || !b->profiling) return fail(FDETD_ERR_ARG, "batch not captured with profiling on");
  for (size_t s = 0; s + 3 < b->stage_ev.size(); s += 4) {
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      cudaError_t e = cudaEventElapsedTime(&ms, b->stage_ev[s + k], b->stage_ev[s + k + 1]);
      if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("batch stage timing: ") + cudaGetErrorString(e));
      b->stage_ms[k] += ms;
    }
    ++b->stage_calls;
  }
  return FDETD_OK;
}

extern "C" int fdetd_batch_pipeline_waits(fdetd_batch_t b, unsigned long long* out) {
  if (!b || !out) return fail(FDETD_ERR_ARG, "null argument");
  return read_waits(b->d_waits, out);
}

extern "C" int fdetd_batch_stage_times(fdetd_batch_t b, double* ms, long* steps) {
  if (!b || !ms) return fail(FDETD_ERR_ARG, "null argument");
  for (int k = 0; k < 3; ++k) ms[k] = b->stage_ms[k];
  if (steps) *steps = b->stage_calls;
  return FDETD_OK;
}

static size_t inst_field_bytes(const fdetd_plan_s* p) {
  return 6 * (size_t)p->nmodes * p->Nz * p->Nr * (p->precision == FDETD_PREC_FP64 ? 16 : 8);
}

// Splits the instances into at most host_parts contiguous parts of about equal bytes and captures a one-step
// graph for each (groups with the tile shapes the main capture chose).
// Contiguous split of n items of the given sizes into at most `parts` parts: part p closes at the first item
// where the running size reaches (p + 1) / P of the total (P = min(parts, n)), the last part takes the rest.
// part_of[k] = the part of item k; returns the number of parts.
static int split_parts(const size_t* bytes, int n, int parts, int* part_of) {
  const int P = std::max(1, std::min(parts, n));
  size_t total = 0;
  for (int k = 0; k < n; ++k) total += bytes[k];
  size_t acc = 0;
  int p = 0;
  for (int k = 0; k < n; ++k) {
    part_of[k] = p;
    acc += bytes[k];
    if (k < n - 1 && p < P - 1 && acc * P >= total * (size_t)(p + 1)) ++p;
  }
  return n ? p + 1 : 0;
}

extern "C" int fdetd_host_split_parts(const size_t* bytes, int n, int parts, int* part_of) {
  if (n < 0 || parts < 1 || (n && (!bytes || !part_of))) return -FDETD_ERR_ARG;
  return split_parts(bytes, n, parts, part_of);
}

static int build_parts(fdetd_batch_s* b, cudaStream_t st) {
  batch_release_parts(b);
  const int n = (int)b->inst.size();
  std::vector<size_t> sizes(n);
  std::vector<int> part_of(n);
  for (int k = 0; k < n; ++k) sizes[k] = inst_field_bytes(b->inst[k].plan);
  const int np = split_parts(sizes.data(), n, b->host_parts, part_of.data());
  b->parts.resize(np);
  for (int k = 0; k < n; ++k) b->parts[part_of[k]].members.push_back(k);
  if (!b->s_in && cudaStreamCreateWithFlags(&b->s_in, cudaStreamNonBlocking) != cudaSuccess)
    return fail(FDETD_ERR_CUDA, "stream");
  if (!b->s_out && cudaStreamCreateWithFlags(&b->s_out, cudaStreamNonBlocking) != cudaSuccess)
    return fail(FDETD_ERR_CUDA, "stream");
  if (!b->ev_start && cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming) != cudaSuccess)
    return fail(FDETD_ERR_CUDA, "event");
  if (!b->ev_end && cudaEventCreateWithFlags(&b->ev_end, cudaEventDisableTiming) != cudaSuccess)
    return fail(FDETD_ERR_CUDA, "event");
  for (auto& part : b->parts) {
    int rc = build_groups(b, part.members, st, &b->groups, part.groups);
    if (rc == FDETD_OK && (cudaEventCreateWithFlags(&part.in, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&part.done, cudaEventDisableTiming) != cudaSuccess))
      rc = fail(FDETD_ERR_CUDA, "event");
    if (rc == FDETD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(FDETD_ERR_CUDA, "stream error");
    if (rc == FDETD_OK) rc = capture_steps(b, part.members, part.groups, 1, st, nullptr, &part.graph, &part.exec);
    if (rc != FDETD_OK) {
      batch_release_parts(b);
      return rc;
    }
  }
  return FDETD_OK;
}

extern "C" int fdetd_batch_set_host_pipeline(fdetd_batch_t b, int parts) {
  if (!b || parts < 1) return fail(FDETD_ERR_ARG, "bad batch or parts < 1");
  if (parts != b->host_parts) batch_release_parts(b);
  b->host_parts = parts;
  return FDETD_OK;
}

extern "C" int fdetd_batch_step_host(fdetd_batch_t b, void* const* host_fields, const void* const* host_J,
                                     int nlaunch, void* stream) {
  if (!b || !b->exec || !host_fields) return fail(FDETD_ERR_ARG, "batch has no captured graph or null fields");
  if (nlaunch < 0) return fail(FDETD_ERR_ARG, "nlaunch < 0");
  for (size_t k = 0; k < b->inst.size(); ++k) {
    if (!host_fields[k]) return fail(FDETD_ERR_ARG, "null host fields");
    if (b->inst[k].J && (!host_J || !host_J[k]))
      return fail(FDETD_ERR_ARG, "instance was added with a current: host J needed");
  }
  cudaStream_t st = (cudaStream_t)stream;
  auto h2d = [&](int k, cudaStream_t s) {
    const fdetd_plan_s* p = b->inst[k].plan;
    const size_t fb = inst_field_bytes(p);
    cudaError_t e = cudaMemcpyAsync(b->inst[k].fields, host_fields[k], fb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && b->inst[k].J)
      e = cudaMemcpyAsync((void*)b->inst[k].J, host_J[k], fb / 2, cudaMemcpyHostToDevice, s);
    return e;
  };
  auto d2h = [&](int k, cudaStream_t s) {
    return cudaMemcpyAsync(host_fields[k], b->inst[k].fields, inst_field_bytes(b->inst[k].plan),
                           cudaMemcpyDeviceToHost, s);
  };
  cudaError_t e = cudaSuccess;
  if (b->host_parts <= 1 || b->inst.size() < 2 || nlaunch == 0) {
    // serial form: every copy in, the main graph, every copy out, on the caller's stream
    for (size_t k = 0; k < b->inst.size() && e == cudaSuccess; ++k) e = h2d((int)k, st);
    for (int s = 0; s < nlaunch && e == cudaSuccess; ++s) e = cudaGraphLaunch(b->exec, st);
    for (size_t k = 0; k < b->inst.size() && e == cudaSuccess; ++k) e = d2h((int)k, st);
  } else {
    if (b->parts.empty()) {
      const int rc = build_parts(b, st);
      if (rc) return rc;
    }
    // copies in on s_in, the parts' graphs on the caller's stream, copies out on s_out: part p's copies
    // overlap the compute of the parts around it; the copy engines of the two directions run concurrently
    e = cudaEventRecord(b->ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s_in, b->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s_out, b->ev_start, 0);
    for (auto& part : b->parts) {
      for (int k : part.members)
        if (e == cudaSuccess) e = h2d(k, b->s_in);
      if (e == cudaSuccess) e = cudaEventRecord(part.in, b->s_in);
    }
    for (auto& part : b->parts) {
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, part.in, 0);
      // a part's graph holds one step; the main graph holds b->steps
      for (int s = 0; s < nlaunch * b->steps && e == cudaSuccess; ++s) e = cudaGraphLaunch(part.exec, st);
      if (e == cudaSuccess) e = cudaEventRecord(part.done, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s_out, part.done, 0);
      for (int k : part.members)
        if (e == cudaSuccess) e = d2h(k, b->s_out);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_end, b->s_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_end, 0);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("batch host step: ") + cudaGetErrorString(e));
  return FDETD_OK;
}

extern "C" int fdetd_batch_destroy(fdetd_batch_t b) {
  if (!b) return FDETD_OK;
  batch_release_graph(b);
  batch_release_events(b);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_waits) cudaFree(b->d_waits);
  if (b->s_in) cudaStreamDestroy(b->s_in);
  if (b->s_out) cudaStreamDestroy(b->s_out);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  if (b->ev_end) cudaEventDestroy(b->ev_end);
  delete b;
  return FDETD_OK;
}

// ------------------------------------------------------------------ envelope

struct envelope_plan_s {
  int Nz = 0, Nr = 0, order = 0, NT = 0;
  double dz = 0, dr = 0, dt = 0, k0 = 0;
  float* d_lr = nullptr;
  float2* d_buf = nullptr;  // T0 (a, a~), T1 (a, a~), ACC (a, a~)
  float* d_chit = nullptr;  // chi + sigma^2 of the absorbing-layer step
  size_t bytes = 0;         // device bytes held
  EnvArgs base;
};

extern "C" int envelope_plan(envelope_plan_t* out, int Nz, int Nr, int order, int taylor_order, double dz,
                             double dr, double dt, double k0) {
  if (!out) return fail(FDETD_ERR_ARG, "out is null");
  *out = nullptr;
  if (order < 2 || order > 32 || (order & 1)) return fail(FDETD_ERR_ARG, "order must be even, 2..32");
  const int N = order / 2;
  if (taylor_order < 1 || taylor_order > 16) return fail(FDETD_ERR_ARG, "taylor_order must be 1..16");
  if (Nz < 2 * order || Nr < N + 1 || !(dz > 0) || !(dr > 0) || !(dt > 0))
    return fail(FDETD_ERR_ARG, "invalid sizes or spacings");
  envelope_plan_s* p = new envelope_plan_s();
  p->Nz = Nz; p->Nr = Nr; p->order = order; p->NT = taylor_order;
  p->dz = dz; p->dr = dr; p->dt = dt; p->k0 = k0;
  double e0 = 0;
  const std::vector<double> e2 = centred_d2_coeffs(order, &e0), d1 = centred_d1_coeffs(order);
  // radial Laplacian band (Eq. spatialAM_laplaceR), symmetric mirror j<0 -> -1-j (m = 0)
  const int W = 2 * N + 1;
  std::vector<double> band((size_t)Nr * W, 0.0);
  for (int k = 0; k < Nr; ++k) {
    const double rho = (k + 0.5) * dr;
    band[(size_t)k * W + N] += e0 / (dr * dr);
    for (int t = 1; t <= N; ++t) {
      const int js[2] = {k + t, k - t};
      const double ws[2] = {e2[t - 1] / (dr * dr) + d1[t - 1] / (dr * rho), e2[t - 1] / (dr * dr) - d1[t - 1] / (dr * rho)};
      for (int s = 0; s < 2; ++s) {
        int j = js[s];
        if (j < 0) j = -1 - j;
        if (j < Nr) band[(size_t)k * W + (j - k) + N] += ws[s];
      }
    }
  }
  std::vector<float> bandf((size_t)Nr * (W + 1));
  for (int k = 0; k < Nr; ++k) {
    double rs = 0.0;
    for (int t = 0; t < W; ++t) {
      bandf[(size_t)k * (W + 1) + t] = (float)band[(size_t)k * W + t];
      rs += band[(size_t)k * W + t];
    }
    bandf[(size_t)k * (W + 1) + W] = (float)rs;
  }
  size_t tot = 0;
  cudaError_t e = upload((void**)&p->d_lr, bandf.data(), bandf.size() * 4, tot);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_buf, (size_t)6 * Nz * Nr * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_chit, (size_t)Nz * Nr * sizeof(float));
  p->bytes = tot + (size_t)6 * Nz * Nr * sizeof(float2) + (size_t)Nz * Nr * sizeof(float);
  if (e != cudaSuccess) {
    if (p->d_lr) cudaFree(p->d_lr);
    if (p->d_buf) cudaFree(p->d_buf);
    delete p;
    return fail(e == cudaErrorMemoryAllocation ? FDETD_ERR_OOM : FDETD_ERR_CUDA, cudaGetErrorString(e));
  }
  EnvArgs& b = p->base;
  memset(&b, 0, sizeof(b));
  b.lr = p->d_lr;
  b.Nz = Nz;
  b.Nr = Nr;
  b.N = N;
  b.cz2[0] = (float)(e0 / (dz * dz));
  for (int t = 1; t <= N; ++t) {
    b.cz2[t] = (float)(e2[t - 1] / (dz * dz));
    b.cz1[t] = (float)(d1[t - 1] / dz);
  }
  b.k2 = (float)(2.0 * k0);
  for (int n = 1; n <= 16; ++n) b.dt_over[n] = (float)(dt / n);
  *out = p;
  return FDETD_OK;
}

// One Taylor-N_T step of (a, a~) in place with susceptibility chi.
static int envelope_taylor(envelope_plan_t p, float2* psi_a, float2* psi_t, const float* chi, cudaStream_t st) {
  const size_t plane = (size_t)p->Nz * p->Nr;
  float2* T[2][2] = {{p->d_buf, p->d_buf + plane}, {p->d_buf + 2 * plane, p->d_buf + 3 * plane}};
  float2* ACC[2] = {p->d_buf + 4 * plane, p->d_buf + 5 * plane};
  EnvArgs g = p->base;
  g.chi = chi;
  for (int n = 1; n <= p->NT; ++n) {
    g.scale = (float)(p->dt / n);
    if (n == 1) {
      g.in_a = psi_a; g.in_t = psi_t;
      g.accin_a = psi_a; g.accin_t = psi_t;
    } else {
      g.in_a = T[(n - 2) & 1][0]; g.in_t = T[(n - 2) & 1][1];
      g.accin_a = ACC[0]; g.accin_t = ACC[1];
    }
    const bool last = n == p->NT;
    g.out_a = last ? nullptr : T[(n - 1) & 1][0];
    g.out_t = last ? nullptr : T[(n - 1) & 1][1];
    const bool to_psi = last && n > 1;
    g.accout_a = to_psi ? psi_a : ACC[0];
    g.accout_t = to_psi ? psi_t : ACC[1];
    cudaError_t e = launch_envelope_term(g, st);
    if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("envelope: ") + cudaGetErrorString(e));
  }
  if (p->NT == 1) {
    cudaError_t e = cudaMemcpyAsync(psi_a, ACC[0], 2 * plane * sizeof(float2), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, cudaGetErrorString(e));
  }
  return FDETD_OK;
}

// Whether the all-terms-in-one-launch kernel serves this plan (order 8, N_T = 4, Nz a multiple of its tile).
static bool envelope_use_fused(envelope_plan_t p) {
  return envelope_fused_supported(p->order, p->NT) && p->Nz % 32 == 0;
}

// n steps of the fused kernel between the caller's state and a plan buffer (the kernel reads halos of its
// input, so input and output alternate), optionally damped around each step (absorbing layer); the result
// ends in the caller's state.
static int envelope_steps_fused(envelope_plan_t p, float2* psi, const float* chi, int nsteps, const float* sigma,
                                float damp, cudaStream_t st) {
  const size_t plane = (size_t)p->Nz * p->Nr;
  float2* buf = p->d_buf;  // two planes: a, a~
  float2* cur = psi;
  float2* nxt = buf;
  EnvArgs g = p->base;
  g.chi = chi;
  g.scale = 0.f;
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = cudaSuccess;
    if (sigma) e = launch_envelope_damp(cur, sigma, damp, plane, st);
    if (e == cudaSuccess) e = launch_envelope_fused(g, cur, cur + plane, nxt, nxt + plane, p->NT, st);
    if (e == cudaSuccess && sigma) e = launch_envelope_damp(nxt, sigma, damp, plane, st);
    if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("envelope: ") + cudaGetErrorString(e));
    std::swap(cur, nxt);
  }
  if (cur != psi) {
    cudaError_t e = cudaMemcpyAsync(psi, cur, 2 * plane * sizeof(float2), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, cudaGetErrorString(e));
  }
  return FDETD_OK;
}

extern "C" int envelope_step(envelope_plan_t p, void* a, const float* chi, int nsteps, void* stream) {
  if (!p || !a || !chi) return fail(FDETD_ERR_ARG, "null argument");
  if (nsteps < 0) return fail(FDETD_ERR_ARG, "nsteps < 0");
  if (((uintptr_t)a & 15) || ((uintptr_t)chi & 15)) return fail(FDETD_ERR_ARG, "pointers must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t plane = (size_t)p->Nz * p->Nr;
  float2* psi_a = (float2*)a;
  for (int s = 0; s < nsteps; ++s) {
    int rc = envelope_taylor(p, psi_a, psi_a + plane, chi, st);
    if (rc) return rc;
  }
  return FDETD_OK;
}

extern "C" int envelope_step_fused(envelope_plan_t p, void* a, const float* chi, int nsteps, void* stream) {
  if (!p || !a || !chi) return fail(FDETD_ERR_ARG, "null argument");
  if (nsteps < 0) return fail(FDETD_ERR_ARG, "nsteps < 0");
  if (((uintptr_t)a & 15) || ((uintptr_t)chi & 15)) return fail(FDETD_ERR_ARG, "pointers must be 16-byte aligned");
  if (!envelope_use_fused(p)) return fail(FDETD_ERR_UNSUPPORTED, "the fused step takes order 8, N_T = 4, Nz = 32 k");
  return envelope_steps_fused(p, (float2*)a, chi, nsteps, nullptr, 0.f, (cudaStream_t)stream);
}

extern "C" int envelope_step_absorbing(envelope_plan_t p, void* a, const float* chi, const float* sigma, int nsteps,
                                       void* stream) {
  if (!p || !a || !chi || !sigma) return fail(FDETD_ERR_ARG, "null argument");
  if (nsteps < 0) return fail(FDETD_ERR_ARG, "nsteps < 0");
  if (((uintptr_t)a & 15) || ((uintptr_t)chi & 15) || ((uintptr_t)sigma & 15))
    return fail(FDETD_ERR_ARG, "pointers must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t plane = (size_t)p->Nz * p->Nr;
  float2* psi_a = (float2*)a;
  cudaError_t e = launch_envelope_chit(chi, sigma, p->d_chit, plane, st);
  if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("envelope: ") + cudaGetErrorString(e));
  const float damp = (float)(-0.25 * p->dt);
  for (int s = 0; s < nsteps; ++s) {
    e = launch_envelope_damp(psi_a, sigma, damp, plane, st);
    if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("envelope: ") + cudaGetErrorString(e));
    int rc = envelope_taylor(p, psi_a, psi_a + plane, p->d_chit, st);
    if (rc) return rc;
    e = launch_envelope_damp(psi_a, sigma, damp, plane, st);
    if (e != cudaSuccess) return fail(FDETD_ERR_CUDA, std::string("envelope: ") + cudaGetErrorString(e));
  }
  return FDETD_OK;
}

extern "C" int envelope_plan_launches_per_step(envelope_plan_t p) { return p ? p->NT : 0; }

extern "C" size_t envelope_plan_device_bytes(envelope_plan_t p) { return p ? p->bytes : 0; }

extern "C" int envelope_plan_destroy(envelope_plan_t p) {
  if (!p) return FDETD_OK;
  if (p->d_lr) cudaFree(p->d_lr);
  if (p->d_buf) cudaFree(p->d_buf);
  if (p->d_chit) cudaFree(p->d_chit);
  delete p;
  return FDETD_OK;
}

extern "C" int fdetd_last_error(char* buf, size_t len) {
  if (!buf || !len) return FDETD_ERR_ARG;
  snprintf(buf, len, "%s", g_err.c_str());
  return FDETD_OK;
}
