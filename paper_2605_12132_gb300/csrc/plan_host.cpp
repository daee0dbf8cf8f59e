// Host-side FP64 plan builder (see plan_host.h).
#include "plan_host.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <future>
#include <list>
#include <memory>
#include <mutex>
#include <thread>

#include "eig.h"

namespace fdetd {

// --------------------------------------------------------------------------
// Exact rational products for the stencil coefficients
// --------------------------------------------------------------------------
namespace {

typedef __int128 i128;

i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) {
    i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

struct Rat {
  i128 p = 0, q = 1;
  Rat() {}
  Rat(long long a, long long b = 1) : p(a), q(b) { norm(); }
  void norm() {
    if (q < 0) {
      p = -p;
      q = -q;
    }
    i128 g = gcd128(p, q);
    if (g > 1) {
      p /= g;
      q /= g;
    }
  }
  Rat mul(const Rat& o) const {
    // cross-reduce before multiplying to keep the intermediates small
    Rat a = *this, b = o;
    i128 g1 = gcd128(a.p, b.q), g2 = gcd128(b.p, a.q);
    if (g1 > 1) { a.p /= g1; b.q /= g1; }
    if (g2 > 1) { b.p /= g2; a.q /= g2; }
    Rat r;
    r.p = a.p * b.p;
    r.q = a.q * b.q;
    r.norm();
    return r;
  }
  Rat add(const Rat& o) const {
    i128 g = gcd128(q, o.q);
    Rat r;
    r.p = p * (o.q / g) + o.p * (q / g);
    r.q = (q / g) * o.q;
    r.norm();
    return r;
  }
  double val() const {
    long double v = (long double)p / (long double)q;
    return (double)v;
  }
};

}  // namespace

std::vector<double> staggered_coeffs(int order) {
  // c_n = 1/(2n-1) prod_{k != n} (2k-1)^2 / ((2k-1)^2 - (2n-1)^2)
  const int N = order / 2;
  std::vector<double> c(N);
  for (int n = 1; n <= N; ++n) {
    Rat r(1, 2 * n - 1);
    const long long on = (long long)(2 * n - 1) * (2 * n - 1);
    for (int k = 1; k <= N; ++k) {
      if (k == n) continue;
      const long long ok = (long long)(2 * k - 1) * (2 * k - 1);
      r = r.mul(Rat(ok, ok - on));
    }
    c[n - 1] = r.val();
  }
  return c;
}

static Rat centred_d1_rat(int N, int n) {
  // d_n = (-1)^(n+1)/n prod_{k=1..n} (N-n+k)/(N+k)
  Rat r((n % 2) ? 1 : -1, n);
  for (int k = 1; k <= n; ++k) r = r.mul(Rat(N - n + k, N + k));
  return r;
}

std::vector<double> centred_d1_coeffs(int order) {
  const int N = order / 2;
  std::vector<double> d(N);
  for (int n = 1; n <= N; ++n) d[n - 1] = centred_d1_rat(N, n).val();
  return d;
}

std::vector<double> centred_d2_coeffs(int order, double* e0) {
  // e_n = (2/n) d_n, e_0 = -2 sum e_n
  const int N = order / 2;
  std::vector<double> e(N);
  Rat s(0, 1);
  for (int n = 1; n <= N; ++n) {
    Rat en = centred_d1_rat(N, n).mul(Rat(2, n));
    e[n - 1] = en.val();
    s = s.add(en);
  }
  if (e0) *e0 = s.mul(Rat(-2, 1)).val();
  return e;
}

int centred_coeffs_fixed(int order, double* d1, double* e2, double* e0) {
  if (order < 2 || order > 32 || (order & 1)) return -1;
  const int N = order / 2;
  Rat s(0, 1);
  for (int n = 1; n <= N; ++n) {
    const Rat d = centred_d1_rat(N, n);
    const Rat en = d.mul(Rat(2, n));
    d1[n - 1] = d.val();
    e2[n - 1] = en.val();
    s = s.add(en);
  }
  *e0 = s.mul(Rat(-2, 1)).val();
  return N;
}

std::vector<double> axis_coeffs(int N) {
  // c_k = prod_{j != k} j^2 / (j^2 - k^2)   (Lagrange in rho^2 at rho = 0, Sec. 2.4)
  std::vector<double> c(N);
  for (int k = 1; k <= N; ++k) {
    Rat r(1, 1);
    for (int j = 1; j <= N; ++j) {
      if (j == k) continue;
      r = r.mul(Rat((long long)j * j, (long long)j * j - (long long)k * k));
    }
    c[k - 1] = r.val();
  }
  return c;
}

// --------------------------------------------------------------------------
// Radial operators (Sec. 2.3-2.4)
// --------------------------------------------------------------------------

// D^(-): primary-grid operand -> staggered grid; mirror j<0 -> -1-j with sign (-1)^parity.
static Mat d_minus(int n, const std::vector<double>& c, double dr, int parity) {
  Mat D(n, n);
  const double sg = (parity & 1) ? -1.0 : 1.0;
  for (int k = 0; k < n; ++k)
    for (int t = 1; t <= (int)c.size(); ++t) {
      int js[2] = {k + t - 1, k - t};
      double ws[2] = {c[t - 1], -c[t - 1]};
      for (int s = 0; s < 2; ++s) {
        int j = js[s];
        double w = ws[s];
        if (j < 0) {
          j = -1 - j;
          w *= sg;
        }
        if (j < n) D(k, j) += w / dr;
      }
    }
  return D;
}

// D^(+): staggered-grid operand (slot 0 = axis) -> primary grid; mirror j<0 -> -j.
static Mat d_plus(int n, const std::vector<double>& c, double dr, int parity) {
  Mat D(n, n);
  const double sg = (parity & 1) ? -1.0 : 1.0;
  for (int k = 0; k < n; ++k)
    for (int t = 1; t <= (int)c.size(); ++t) {
      int js[2] = {k + t, k - t + 1};
      double ws[2] = {c[t - 1], -c[t - 1]};
      for (int s = 0; s < 2; ++s) {
        int j = js[s];
        double w = ws[s];
        if (j < 0) {
          j = -j;
          w *= sg;
        }
        if (j < n) D(k, j) += w / dr;
      }
    }
  return D;
}

// ---------------------------------------------------------------- double-double helpers
namespace {
struct DD {
  double hi, lo;
};
inline DD quick_two_sum(double a, double b) {
  const double s = a + b;
  return {s, b - (s - a)};
}
inline DD two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
inline DD two_prod(double a, double b) {
  const double p = a * b;
  return {p, std::fma(a, b, -p)};
}
inline DD dd_add(DD a, DD b) {
  DD s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + a.lo + b.lo);
}
inline DD dd_mul_d(DD a, double b) {
  DD p = two_prod(a.hi, b);
  return quick_two_sum(p.hi, p.lo + a.lo * b);
}
inline DD dd_div_d(DD a, double b) {
  const double q1 = a.hi / b;
  DD p = two_prod(q1, b);
  const double r = ((a.hi - p.hi) - p.lo + a.lo) / b;
  return quick_two_sum(q1, r);
}
}  // namespace

// Two-sided Rayleigh-quotient refinement of eigenvalues w_j of a matrix applied through
// `apply` (double-double residual): w_j <- w_j + y_j.(A x_j - w_j x_j) / y_j.x_j with x_j the
// right eigenvector (column j of V) and y_j the left one (row j of V^-1).  The residual of a
// squared radial operator cancels to ~eps |A| in FP64, which is large relative to its small
// eigenvalues; evaluating it in double-double restores their relative accuracy.
template <typename F>
static void refine_eigs(std::vector<double>& w, const Mat& V, const Mat& Vi, F apply) {
  const int n = V.n;
  std::vector<double> x(n);
  std::vector<DD> ax(n);
  for (int j = 0; j < n; ++j) {
    for (int k = 0; k < n; ++k) x[k] = V(k, j);
    apply(x, ax);
    DD num = {0, 0}, den = {0, 0};
    for (int k = 0; k < n; ++k) {
      const DD r = dd_add(ax[k], two_prod(-w[j], x[k]));
      num = dd_add(num, dd_mul_d(r, Vi(j, k)));
      den = dd_add(den, two_prod(Vi(j, k), x[k]));
    }
    w[j] += (num.hi + num.lo) / (den.hi + den.lo);
  }
}

void phase_coeffs(double w, double t, double* A1, double* A2) {
  const double x = w * t;
  if (x < 1e-3) {
    const double x2 = x * x;
    *A1 = t * (1.0 - x2 / 6.0 * (1.0 - x2 / 20.0));
    *A2 = 0.5 * t * t * (1.0 - x2 / 12.0 * (1.0 - x2 / 30.0));
  } else {
    const double s = std::sin(0.5 * x);
    *A1 = std::sin(x) / w;
    *A2 = 2.0 * s * s / (w * w);
  }
}

// f on another thread (std::async), or deferred to get() where no thread can be started
template <typename F>
static auto run_async(F f) -> std::future<decltype(f())> {
  try {
    return std::async(std::launch::async, f);
  } catch (...) {
    return std::async(std::launch::deferred, f);
  }
}

static int build_mode(ModePlan& P, int n, int order, double dr, int m, std::string& msg) {
  P.m = m;
  P.n = n;
  const std::vector<double> c = staggered_coeffs(order);
  const int ND = order / 2;
  const int parity = m & 1;  // every radial derivative acts on a parity-m operand
  Mat Dm = d_minus(n, c, dr, parity), Dp = d_plus(n, c, dr, parity);
  std::vector<double> rho(n), rhom(n);
  for (int k = 0; k < n; ++k) {
    rho[k] = (k + 0.5) * dr;
    rhom[k] = k * dr;
  }
  const std::vector<double> ax = axis_coeffs(ND);
  std::vector<double> w_scalar(n - 1, 0.0), w_polar(n - 1, 0.0);
  for (int k = 0; k < ND; ++k) {
    if (m == 0) w_scalar[k] = ax[k];  // B_z-type constant on the axis for m = 0
    if (m == 1) w_polar[k] = ax[k];   // E_rho / B_theta constant on the axis for m = 1
  }
  const int n1 = n - 1;
  Mat DivP(n, n1), GradR(n1, n), DivM(n1, n), DpBz(n, n1);
  for (int k = 0; k < n; ++k)
    for (int j = 1; j < n; ++j) {
      DivP(k, j - 1) = Dp(k, j) * rhom[j] / rho[k];
      DpBz(k, j - 1) = Dp(k, j) + Dp(k, 0) * w_scalar[j - 1];
    }
  for (int k = 1; k < n; ++k)
    for (int j = 0; j < n; ++j) {
      GradR(k - 1, j) = Dm(k, j);
      DivM(k - 1, j) = Dm(k, j) * rho[j] / rhom[k];
    }
  Mat L0 = matmul(DivP, GradR), L2 = matmul(DivM, DpBz);
  for (int k = 0; k < n; ++k) L0(k, k) -= (double)m * m / (rho[k] * rho[k]);
  for (int k = 0; k < n1; ++k) L2(k, k) -= (double)m * m / (rhom[k + 1] * rhom[k + 1]);

  std::vector<double> w0, w2;
  Mat U, Psi, Ui, Psii;
  double im0 = 0, im2 = 0;
  // the TM (L0) and TE (L2) eigenbases are independent: the TE one is computed on a second thread
  // (1 = eigen-decomposition failed, 2 = singular basis)
  auto te = run_async([&]() -> int {
    if (eig_real(L2, w2, Psi, 1e-8, &im2) != 0) return 1;
    return invert(Psi, Psii) != 0 ? 2 : 0;
  });
  const int rc0 = eig_real(L0, w0, U, 1e-8, &im0) != 0 ? 1 : (invert(U, Ui) != 0 ? 2 : 0);
  const int rc2 = te.get();
  if (rc0 == 1 || rc2 == 1) {
    msg = "radial eigen-decomposition failed (complex or non-convergent spectrum) for mode " + std::to_string(m);
    return 4;
  }
  P.max_imag = std::max(im0, im2);
  if (rc0 == 2 || rc2 == 2) {
    msg = "singular radial eigenbasis for mode " + std::to_string(m);
    return 4;
  }
  {
    // L0 x = rho^-1 D^+ (rho_- (D^- x)) - m^2 x / rho^2 in factored form (double-double)
    const double m2 = (double)m * m;
    auto apply_L0 = [&](const std::vector<double>& x, std::vector<DD>& out) {
      std::vector<DD> t(n, DD{0, 0});
      for (int k = 1; k < n; ++k) {
        DD acc = {0, 0};
        for (int j = 0; j < n; ++j)
          if (Dm(k, j) != 0.0) acc = dd_add(acc, two_prod(Dm(k, j), x[j]));
        t[k] = dd_mul_d(acc, rhom[k]);
      }
      for (int k = 0; k < n; ++k) {
        DD acc = {0, 0};
        for (int j = 1; j < n; ++j)
          if (Dp(k, j) != 0.0) acc = dd_add(acc, dd_mul_d(t[j], Dp(k, j)));
        out[k] = dd_add(dd_div_d(acc, rho[k]), dd_div_d(dd_div_d(two_prod(-m2, x[k]), rho[k]), rho[k]));
      }
    };
    // L2 psi = rho_-^-1 D^- (rho (D^+ X0 psi)) - m^2 psi / rho_-^2 (double-double)
    auto apply_L2 = [&](const std::vector<double>& x, std::vector<DD>& out) {
      std::vector<DD> g(n, DD{0, 0}), u(n, DD{0, 0});
      for (int k = 1; k < n; ++k) g[k] = DD{x[k - 1], 0};
      for (int k = 0; k < n1; ++k)
        if (w_scalar[k] != 0.0) g[0] = dd_add(g[0], two_prod(w_scalar[k], x[k]));
      for (int k = 0; k < n; ++k) {
        DD acc = {0, 0};
        for (int j = 0; j < n; ++j)
          if (Dp(k, j) != 0.0) acc = dd_add(acc, dd_mul_d(g[j], Dp(k, j)));
        u[k] = dd_mul_d(acc, rho[k]);
      }
      for (int k = 1; k < n; ++k) {
        DD acc = {0, 0};
        for (int j = 0; j < n; ++j)
          if (Dm(k, j) != 0.0) acc = dd_add(acc, dd_mul_d(u[j], Dm(k, j)));
        out[k - 1] = dd_add(dd_div_d(acc, rhom[k]),
                            dd_div_d(dd_div_d(two_prod(-m2, x[k - 1]), rhom[k]), rhom[k]));
      }
    };
    auto te_refine = run_async([&]() -> int {
      refine_eigs(w2, Psi, Psii, apply_L2);
      return 0;
    });
    refine_eigs(w0, U, Ui, apply_L0);
    te_refine.get();
  }
  P.lam.assign(n, 0.0);
  P.mu.assign(n, 0.0);
  P.tm_live.assign(n, 1);
  P.te_live.assign(n, 1);
  double lmax = 0.0;
  for (int j = 0; j < n; ++j) lmax = std::max(lmax, std::fabs(w0[j]));
  int nzero = 0;
  for (int j = 0; j < n; ++j) {
    P.lam[j] = -w0[j];
    if (std::fabs(w0[j]) < 1e-9 * lmax) {
      P.tm_live[j] = 0;
      P.lam[j] = 0.0;
      ++nzero;
    } else if (P.lam[j] <= 0.0) {
      msg = "non-positive TM eigenvalue for mode " + std::to_string(m);
      return 4;
    }
  }
  if (nzero != (m == 0 ? 1 : 0)) {
    msg = "unexpected TM null space for mode " + std::to_string(m);
    return 4;
  }
  for (int j = 0; j < n1; ++j) {
    P.mu[j] = -w2[j];
    if (P.mu[j] <= 0.0) {
      msg = "non-positive TE eigenvalue for mode " + std::to_string(m);
      return 4;
    }
  }
  P.mu[n1] = 0.0;
  P.te_live[n1] = (m == 0) ? 1 : 0;

  // projection pieces
  Mat LiUi(n, n), MiPsii(n1, n1);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) LiUi(j, k) = P.tm_live[j] ? -Ui(j, k) / P.lam[j] : 0.0;
  for (int j = 0; j < n1; ++j)
    for (int k = 0; k < n1; ++k) MiPsii(j, k) = Psii(j, k) / P.mu[j];
  Mat A_Er = matmul(LiUi, DivP);   // n x n1 (acts on Er slots 1..)
  Mat C_Et = matmul(MiPsii, DivM);  // n1 x n
  Mat GU = matmul(GradR, U);        // n1 x n
  Mat DPsi = matmul(DpBz, Psi);     // n x n1

  const int N3 = 3 * n;
  P.PE.assign((size_t)N3 * N3, 0.0);
  P.PB.assign((size_t)N3 * N3, 0.0);
  P.QE.assign((size_t)N3 * N3, 0.0);
  P.QB.assign((size_t)N3 * N3, 0.0);
  auto at = [N3](std::vector<double>& M, int blk_r, int r, int blk_c, int cc) -> double& {
    return M[(size_t)(blk_r * (N3 / 3) + r) * N3 + blk_c * (N3 / 3) + cc];
  };
  // E group forward: rows (e, a, c^), cols (Er, Et^, Ez)
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      at(P.PE, 0, j, 2, k) = Ui(j, k);
      at(P.PE, 1, j, 1, k) = LiUi(j, k) * m / rho[k];
      if (k >= 1) at(P.PE, 1, j, 0, k) = A_Er(j, k - 1);
    }
  for (int j = 0; j < n1; ++j)
    for (int k = 0; k < n; ++k) {
      at(P.PE, 2, j, 1, k) = C_Et(j, k);
      if (k >= 1) at(P.PE, 2, j, 0, k) = MiPsii(j, k - 1) * m / rhom[k];
    }
  // B group forward: rows (b, d^, f^), cols (Bt, Br^, Bz^); same transverse map on w = (Bt, -Br^)
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < n; ++k) {
      at(P.PB, 0, r, 0, k) = at(P.PE, 1, r, 0, k);
      at(P.PB, 0, r, 1, k) = -at(P.PE, 1, r, 1, k);
      at(P.PB, 1, r, 0, k) = at(P.PE, 2, r, 0, k);
      at(P.PB, 1, r, 1, k) = -at(P.PE, 2, r, 1, k);
    }
  for (int j = 0; j < n1; ++j)
    for (int k = 1; k < n; ++k) at(P.PB, 2, j, 2, k) = Psii(j, k - 1);
  // E group backward: rows (Er, Et^, Ez), cols (e, a, c^)
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) {
      at(P.QE, 2, k, 0, j) = U(k, j);
      at(P.QE, 1, k, 1, j) = -(double)m / rho[k] * U(k, j);
      if (k >= 1) at(P.QE, 0, k, 1, j) = GU(k - 1, j);
    }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n1; ++j) {
      at(P.QE, 1, k, 2, j) = -DPsi(k, j);
      if (k >= 1) at(P.QE, 0, k, 2, j) = (double)m / rhom[k] * Psi(k - 1, j);
    }
  if (m == 0) {
    // radially uniform TE pair (curl- and divergence-free E_theta / B_rho component):
    // h spans ker D_div^(-), l spans the left null space of D^(+) with the axis fill, l.h = 1.
    std::vector<double> h(n, 0.0), l(n, 0.0), x, b(n1);
    Mat A(n1, n1);
    for (int i = 0; i < n1; ++i) {
      for (int j = 0; j < n1; ++j) A(i, j) = DivM(i, j + 1);
      b[i] = -DivM(i, 0);
    }
    if (solve(A, x, b) != 0) {
      msg = "null vector of D_div^(-) not found";
      return 4;
    }
    h[0] = 1.0;
    for (int i = 0; i < n1; ++i) h[i + 1] = x[i];
    for (int i = 0; i < n1; ++i) {
      for (int j = 0; j < n1; ++j) A(i, j) = DpBz(j + 1, i);
      b[i] = -DpBz(0, i);
    }
    if (solve(A, x, b) != 0) {
      msg = "left null vector of D^(+) not found";
      return 4;
    }
    l[0] = 1.0;
    for (int i = 0; i < n1; ++i) l[i + 1] = x[i];
    double lh = 0.0;
    for (int i = 0; i < n; ++i) lh += l[i] * h[i];
    for (int i = 0; i < n; ++i) {
      at(P.PE, 2, n1, 1, i) = l[i] / lh;
      at(P.QE, 1, i, 2, n1) = h[i];
    }
  }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) {
      at(P.QB, 0, k, 0, j) = at(P.QE, 0, k, 1, j);
      at(P.QB, 0, k, 1, j) = at(P.QE, 0, k, 2, j);
      at(P.QB, 1, k, 0, j) = -at(P.QE, 1, k, 1, j);
      at(P.QB, 1, k, 1, j) = -at(P.QE, 1, k, 2, j);
    }
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < n; ++k) at(P.PB, 1, r, 1, k) = -at(P.PE, 2, r, 1, k);  // includes -l^T row
  for (int k = 1; k < n; ++k)
    for (int j = 0; j < n1; ++j) at(P.QB, 2, k, 2, j) = Psi(k - 1, j);
  // axis rows (Sec. 2.4): slot 0 of the staggered-grid fields from their interior slots
  for (int col = 0; col < N3; ++col) {
    double se = 0, sb = 0, sz = 0;
    for (int k = 1; k <= ND && k < n; ++k) {
      se += w_polar[k - 1] * P.QE[(size_t)k * N3 + col];
      sb += w_polar[k - 1] * P.QB[(size_t)k * N3 + col];
      sz += w_scalar[k - 1] * P.QB[(size_t)(2 * n + k) * N3 + col];
    }
    P.QE[(size_t)0 * N3 + col] = se;
    P.QB[(size_t)0 * N3 + col] = sb;
    P.QB[(size_t)(2 * n) * N3 + col] = sz;
  }
  return 0;
}

// Banded radial operators of the real-space operator H of one mode (Sec. 2.5), for the paper's
// Taylor scheme.  Row k of band b holds the coefficients of columns k - ND .. k + ND (zero outside
// 0..n-1), W = 2 ND + 1 per row, bands [4][n][W]:
//   0: D^+ acting on B_z with its axis value (the Sec. 2.4 extrapolation for m = 0) folded into
//      columns 1..ND, column 0 zero            (E_theta_t = D_z^+ B_rho - band0 B_z ...)
//   1: rho_k^-1 D^+ rho_-,j on B_theta         (E_z_t = ... + band1 B_theta)
//   2: D^- on E_z, row 0 zero                  (B_theta_t = ... + band2 E_z)
//   3: rho_-,k^-1 D^- rho_j on E_theta, row 0 zero (B_z_t = ... - band3 E_theta)
// axis[2][ND]: extrapolation weights of the axis slot from slots 1..ND for the polar fields
// (E_rho, B_theta; nonzero for m = 1) and the scalar field (B_z; nonzero for m = 0).
int taylor_bands(int n, int order, double dr, int m, std::vector<double>& bands, std::vector<double>& axis) {
  if (order < 2 || order > 32 || (order & 1) || n < order / 2 + 2) return 1;
  const std::vector<double> c = staggered_coeffs(order);
  const int ND = order / 2, W = 2 * ND + 1;
  const int parity = m & 1;
  Mat Dm = d_minus(n, c, dr, parity), Dp = d_plus(n, c, dr, parity);
  const std::vector<double> ax = axis_coeffs(ND);
  std::vector<double> w_scalar(n, 0.0);
  for (int k = 0; k < ND; ++k)
    if (m == 0) w_scalar[k + 1] = ax[k];  // weight of slot k + 1 in the B_z axis value
  bands.assign((size_t)4 * n * W, 0.0);
  auto B = [&](int b, int k, int j) -> double& { return bands[((size_t)b * n + k) * W + (j - k + ND)]; };
  for (int k = 0; k < n; ++k) {
    const double rho = (k + 0.5) * dr, rhom = k * dr;
    for (int j = std::max(0, k - ND); j <= std::min(n - 1, k + ND); ++j) {
      if (j >= 1) B(0, k, j) = Dp(k, j) + Dp(k, 0) * w_scalar[j];
      B(1, k, j) = Dp(k, j) * (j * dr) / rho;
      if (k >= 1) {
        B(2, k, j) = Dm(k, j);
        B(3, k, j) = Dm(k, j) * ((j + 0.5) * dr) / rhom;
      }
    }
  }
  axis.assign((size_t)2 * ND, 0.0);
  for (int k = 0; k < ND; ++k) {
    if (m == 1) axis[k] = ax[k];
    if (m == 0) axis[ND + k] = ax[k];
  }
  return 0;
}

// Banded radial operators of the planar current correction of mode m (Sec. 3, Eqs.
// shapesAM_currentRHS2m ... shapesAM_currentJth), rows k over columns k - ND .. k + ND (W = 2 ND + 1):
//   divp: rho_k^-1 D^+ rho_-,j       (staggered J_rho -> primary divergence; column 0 is zero)
//   dm:   D^-                        (primary phi -> staggered gradient, every row including the axis)
// and the LU factors (no pivoting; the pivots of this operator stay far from zero) of
//   A = L_rho^(mS) - m^2 rho^-2,  L_rho = D^2 + rho^-1 D^(C) centred (Eq. spatialAM_laplaceR),
// primary-grid mirror j < 0 -> -1 - j with the sign (-1)^m, taps past the outer edge dropped:
//   lo[k][d - 1] = l(k, k - d) (unit lower factor), up[k][d] = u(k, k + d), d = 0..ND.
// Returns 0, or 1 for bad arguments, 2 for a vanishing pivot.
int current_bands(int n, int order, double dr, int m, std::vector<double>& divp, std::vector<double>& dm,
                  std::vector<double>& lo, std::vector<double>& up) {
  if (order < 2 || order > 32 || (order & 1) || n < order / 2 + 2) return 1;
  const int ND = order / 2, W = 2 * ND + 1, parity = m & 1;
  const std::vector<double> c = staggered_coeffs(order);
  Mat Dm = d_minus(n, c, dr, parity), Dp = d_plus(n, c, dr, parity);
  divp.assign((size_t)n * W, 0.0);
  dm.assign((size_t)n * W, 0.0);
  for (int k = 0; k < n; ++k)
    for (int j = std::max(0, k - ND); j <= std::min(n - 1, k + ND); ++j) {
      divp[(size_t)k * W + (j - k + ND)] = Dp(k, j) * (j * dr) / ((k + 0.5) * dr);
      dm[(size_t)k * W + (j - k + ND)] = Dm(k, j);
    }
  // dense band of A (row k, column k + d for |d| <= ND)
  double e0 = 0;
  const std::vector<double> e = centred_d2_coeffs(order, &e0);
  const std::vector<double> d1 = centred_d1_coeffs(order);
  const double sg = parity ? -1.0 : 1.0;
  std::vector<double> A((size_t)n * W, 0.0);
  auto Aat = [&](int k, int j) -> double& { return A[(size_t)k * W + (j - k + ND)]; };
  for (int k = 0; k < n; ++k) {
    const double rho = (k + 0.5) * dr;
    Aat(k, k) += e0 / (dr * dr) - (double)m * m / (rho * rho);
    for (int t = 1; t <= ND; ++t) {
      const int js[2] = {k + t, k - t};
      const double ws[2] = {e[t - 1] / (dr * dr) + d1[t - 1] / (dr * rho), e[t - 1] / (dr * dr) - d1[t - 1] / (dr * rho)};
      for (int q = 0; q < 2; ++q) {
        int j = js[q];
        double w = ws[q];
        if (j < 0) {
          j = -1 - j;
          w *= sg;
        }
        if (j < n) Aat(k, j) += w;
      }
    }
  }
  // banded LU without pivoting (Doolittle)
  lo.assign((size_t)n * ND, 0.0);
  up.assign((size_t)n * (ND + 1), 0.0);
  double amax = 0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  for (int k = 0; k < n; ++k) {
    for (int j = k; j <= std::min(n - 1, k + ND); ++j) {
      double s = Aat(k, j);
      for (int q = std::max(0, j - ND); q < k; ++q)
        if (k - q <= ND) s -= lo[(size_t)k * ND + (k - q - 1)] * up[(size_t)q * (ND + 1) + (j - q)];
      up[(size_t)k * (ND + 1) + (j - k)] = s;
    }
    const double piv = up[(size_t)k * (ND + 1)];
    if (std::fabs(piv) < 1e-12 * amax) return 2;
    for (int i = k + 1; i <= std::min(n - 1, k + ND); ++i) {
      double s = Aat(i, k);
      for (int q = std::max(0, i - ND); q < k; ++q)
        if (k - q <= ND) s -= lo[(size_t)i * ND + (i - q - 1)] * up[(size_t)q * (ND + 1) + (k - q)];
      lo[(size_t)i * ND + (i - k - 1)] = s / piv;
    }
  }
  return 0;
}

// ------------------------------------------------------------------ cache of per-mode radial tables
// A mode's radial tables depend on (Nr, order, dr, m) only, not on Nz, dt or the precision, so plans that share a
// radial grid (repeated requests to a server, the instances of a batch) share one eigen-decomposition.  The cache
// holds immutable tables, keyed on those four values (dr by its bit pattern), bounded in bytes, least recently used
// evicted first; two threads that miss on the same key both build it and the first insert wins.
namespace {

struct ModeKey {
  int n, order, m;
  uint64_t dr_bits;
  bool operator==(const ModeKey& o) const {
    return n == o.n && order == o.order && m == o.m && dr_bits == o.dr_bits;
  }
};

struct ModeCache {
  std::mutex mu;
  std::list<std::pair<ModeKey, std::shared_ptr<const ModePlan>>> lru;  // front = most recently used
  size_t bytes = 0, limit = size_t(4) << 30;
  uint64_t hits = 0, misses = 0;
};

ModeCache& mode_cache() {
  static ModeCache c;
  return c;
}

size_t mode_plan_bytes(const ModePlan& P) {
  return sizeof(double) * (P.lam.size() + P.mu.size() + P.PE.size() + P.PB.size() + P.QE.size() + P.QB.size()) +
         P.tm_live.size() + P.te_live.size();
}

void evict_over_limit(ModeCache& c) {
  while (c.bytes > c.limit && !c.lru.empty()) {
    c.bytes -= mode_plan_bytes(*c.lru.back().second);
    c.lru.pop_back();
  }
}

int cached_mode(ModePlan& P, int n, int order, double dr, int m, std::string& msg) {
  ModeKey key{n, order, m, 0};
  std::memcpy(&key.dr_bits, &dr, sizeof(dr));
  ModeCache& c = mode_cache();
  std::shared_ptr<const ModePlan> hit;
  {
    std::lock_guard<std::mutex> lk(c.mu);
    for (auto it = c.lru.begin(); it != c.lru.end(); ++it)
      if (it->first == key) {
        c.lru.splice(c.lru.begin(), c.lru, it);
        hit = it->second;
        ++c.hits;
        break;
      }
    if (!hit) ++c.misses;
  }
  if (hit) {
    P = *hit;
    return 0;
  }
  const int rc = build_mode(P, n, order, dr, m, msg);
  if (rc) return rc;
  const size_t b = mode_plan_bytes(P);
  std::lock_guard<std::mutex> lk(c.mu);
  if (b > c.limit) return 0;
  for (const auto& e : c.lru)
    if (e.first == key) return 0;
  c.lru.emplace_front(key, std::make_shared<const ModePlan>(P));
  c.bytes += b;
  evict_over_limit(c);
  return 0;
}

}  // namespace

int mode_cache_warm(int n, int order, double dr, int m, std::string& msg) {
  ModeKey key{n, order, m, 0};
  std::memcpy(&key.dr_bits, &dr, sizeof(dr));
  {
    ModeCache& c = mode_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    for (const auto& e : c.lru)
      if (e.first == key) return 0;
  }
  ModePlan P;
  return cached_mode(P, n, order, dr, m, msg);
}

void mode_cache_set_limit(size_t bytes) {
  ModeCache& c = mode_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  c.limit = bytes;
  evict_over_limit(c);
}

void mode_cache_stats(size_t* bytes, size_t* limit, int* entries, uint64_t* hits, uint64_t* misses) {
  ModeCache& c = mode_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  if (bytes) *bytes = c.bytes;
  if (limit) *limit = c.limit;
  if (entries) *entries = (int)c.lru.size();
  if (hits) *hits = c.hits;
  if (misses) *misses = c.misses;
}

int build_host_plan(HostPlan& hp, int Nz, int Nr, const int* modes, int nmodes, int order, double dz,
                    double dr, double dt, std::string& msg) {
  if (order < 2 || order > 32 || (order & 1)) {
    msg = "order must be even, 2..32";
    return 1;
  }
  if (Nr < order / 2 + 2 || Nz < 2 || nmodes < 1 || !(dz > 0) || !(dr > 0) || !(dt > 0)) {
    msg = "invalid sizes or spacings";
    return 1;
  }
  hp.Nz = Nz;
  hp.Nr = Nr;
  hp.order = order;
  hp.dz = dz;
  hp.dr = dr;
  hp.dt = dt;
  hp.modes.assign(modes, modes + nmodes);
  hp.mp.resize(nmodes);
  for (int i = 0; i < nmodes; ++i)
    if (modes[i] < 0 || modes[i] > 64) {
      msg = "mode numbers must be 0..64";
      return 1;
    }
  // modes are independent: W workers take modes w, w + W, ...; the first failing mode (in mode order) reports
  {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int W = std::max(1, std::min(nmodes, (int)std::max(1u, hw / 2)));
    std::vector<int> rcs(nmodes, 0);
    std::vector<std::string> msgs(nmodes);
    auto work = [&](int w) -> int {
      for (int i = w; i < nmodes; i += W) rcs[i] = cached_mode(hp.mp[i], Nr, order, dr, modes[i], msgs[i]);
      return 0;
    };
    std::vector<std::future<int>> fs;
    for (int w = 1; w < W; ++w) fs.push_back(run_async([&work, w]() { return work(w); }));
    work(0);
    for (auto& f : fs) f.get();
    for (int i = 0; i < nmodes; ++i)
      if (rcs[i]) {
        msg = msgs[i];
        return rcs[i];
      }
  }
  // z symbols of the periodic staggered stencil: s+ = i kappa e^{+i th/2}, s- = i kappa e^{-i th/2},
  // kappa = (2/dz) sum_n c_n sin((2n-1) th / 2), th = 2 pi q / Nz.
  const std::vector<double> c = staggered_coeffs(order);
  hp.sp_re.resize(Nz);
  hp.sp_im.resize(Nz);
  hp.sm_re.resize(Nz);
  hp.sm_im.resize(Nz);
  hp.kappa2.resize(Nz);
  const double pi = 3.14159265358979323846;
  for (int q = 0; q < Nz; ++q) {
    double kap = 0.0;
    for (int t = 1; t <= (int)c.size(); ++t) {
      const long long num = ((long long)q * (2 * t - 1)) % (2LL * Nz);  // angle = pi * num / Nz
      kap += c[t - 1] * std::sin(pi * (double)num / Nz);
    }
    kap *= 2.0 / dz;
    const double half = pi * (double)q / Nz;
    const double ch = std::cos(half), sh = std::sin(half);
    hp.kappa2[q] = kap * kap;
    hp.sp_re[q] = -kap * sh;
    hp.sp_im[q] = kap * ch;
    hp.sm_re[q] = kap * sh;
    hp.sm_im[q] = kap * ch;
  }
  return 0;
}

}  // namespace fdetd
