// Dense FP64 eigen-decomposition and LU inversion for the plan builder.
//
// Textbook algorithms (Golub & Van Loan, "Matrix Computations", Sec. 7.4-7.6):
// Householder reduction to upper Hessenberg form, Francis double-shift QR with
// deflation to real Schur form (transformations accumulated), 2x2 blocks with
// real eigenvalues split by a Givens rotation, eigenvectors by back-substitution
// on the triangular factor.
#include "eig.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace fdetd {

static const double kEps = 2.220446049250313e-16;

Mat matmul(const Mat& A, const Mat& B) {
  Mat C(A.n, B.m);
  for (int i = 0; i < A.n; ++i) {
    double* c = &C.a[(size_t)i * C.m];
    for (int k = 0; k < A.m; ++k) {
      const double aik = A(i, k);
      if (aik == 0.0) continue;
      const double* b = &B.a[(size_t)k * B.m];
      for (int j = 0; j < B.m; ++j) c[j] += aik * b[j];
    }
  }
  return C;
}

static void hessenberg(Mat& H, Mat& Z) {
  const int n = H.n;
  Z = Mat(n, n);
  for (int i = 0; i < n; ++i) Z(i, i) = 1.0;
  std::vector<double> v(n);
  for (int k = 0; k < n - 2; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += H(i, k) * H(i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (H(k + 1, k) > 0) alpha = -alpha;
    double vn2 = 0.0;
    for (int i = k + 1; i < n; ++i) {
      v[i] = H(i, k) - (i == k + 1 ? alpha : 0.0);
      vn2 += v[i] * v[i];
    }
    if (vn2 == 0.0) continue;
    const double beta = 2.0 / vn2;
    for (int j = k; j < n; ++j) {
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * H(i, j);
      s *= beta;
      for (int i = k + 1; i < n; ++i) H(i, j) -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += H(i, j) * v[j];
      s *= beta;
      for (int j = k + 1; j < n; ++j) H(i, j) -= s * v[j];
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += Z(i, j) * v[j];
      s *= beta;
      for (int j = k + 1; j < n; ++j) Z(i, j) -= s * v[j];
    }
    H(k + 1, k) = alpha;
    for (int i = k + 2; i < n; ++i) H(i, k) = 0.0;
  }
}

// Householder vector for a length-len vector x: P = I - beta v v^T maps x to a multiple of e1.
static void house(const double* x, int len, double* v, double& beta) {
  double nrm = 0.0;
  for (int i = 0; i < len; ++i) nrm += x[i] * x[i];
  nrm = std::sqrt(nrm);
  for (int i = 0; i < len; ++i) v[i] = x[i];
  if (nrm == 0.0) {
    beta = 0.0;
    return;
  }
  v[0] += (x[0] >= 0 ? nrm : -nrm);
  double vn2 = 0.0;
  for (int i = 0; i < len; ++i) vn2 += v[i] * v[i];
  beta = vn2 > 0 ? 2.0 / vn2 : 0.0;
}

static void apply_left(Mat& H, int r0, int len, const double* v, double beta, int c0, int c1) {
  for (int j = c0; j <= c1; ++j) {
    double s = 0.0;
    for (int i = 0; i < len; ++i) s += v[i] * H(r0 + i, j);
    s *= beta;
    for (int i = 0; i < len; ++i) H(r0 + i, j) -= s * v[i];
  }
}

static void apply_right(Mat& H, int c0, int len, const double* v, double beta, int r0, int r1) {
  for (int i = r0; i <= r1; ++i) {
    double s = 0.0;
    for (int j = 0; j < len; ++j) s += H(i, c0 + j) * v[j];
    s *= beta;
    for (int j = 0; j < len; ++j) H(i, c0 + j) -= s * v[j];
  }
}

// Split a 2x2 diagonal block at (i, i) into upper-triangular form when its eigenvalues
// are real; returns the magnitude of the imaginary part otherwise (block left as is).
static double split2(Mat& H, Mat& Z, int i) {
  const int n = H.n;
  const double a = H(i, i), b = H(i, i + 1), c = H(i + 1, i), d = H(i + 1, i + 1);
  const double p = 0.5 * (a - d);
  const double disc = p * p + b * c;
  if (disc < 0) return std::sqrt(-disc);
  const double sq = std::sqrt(disc);
  const double l1 = 0.5 * (a + d) + (p >= 0 ? sq : -sq);
  double x, y;
  if (std::fabs(b) + std::fabs(l1 - a) >= std::fabs(l1 - d) + std::fabs(c)) {
    x = b;
    y = l1 - a;
  } else {
    x = l1 - d;
    y = c;
  }
  const double r = std::hypot(x, y);
  if (r == 0.0) {
    H(i + 1, i) = 0.0;
    return 0.0;
  }
  const double cs = x / r, sn = y / r;
  // rows i, i+1: G^T H
  for (int j = i; j < n; ++j) {
    const double h0 = H(i, j), h1 = H(i + 1, j);
    H(i, j) = cs * h0 + sn * h1;
    H(i + 1, j) = -sn * h0 + cs * h1;
  }
  // cols i, i+1: H G
  for (int k = 0; k <= i + 1; ++k) {
    const double h0 = H(k, i), h1 = H(k, i + 1);
    H(k, i) = cs * h0 + sn * h1;
    H(k, i + 1) = -sn * h0 + cs * h1;
  }
  for (int k = 0; k < n; ++k) {
    const double z0 = Z(k, i), z1 = Z(k, i + 1);
    Z(k, i) = cs * z0 + sn * z1;
    Z(k, i + 1) = -sn * z0 + cs * z1;
  }
  H(i + 1, i) = 0.0;
  return 0.0;
}

static int schur(Mat& H, Mat& Z, double& max_imag) {
  const int n = H.n;
  double norm = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = std::max(0, i - 1); j < n; ++j) norm += std::fabs(H(i, j));
  max_imag = 0.0;
  int p = n - 1, iter = 0, total = 0;
  double v[3], beta;
  while (p >= 0) {
    int l = p;
    while (l > 0) {
      double s = std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l));
      if (s == 0.0) s = norm;
      if (std::fabs(H(l, l - 1)) < kEps * s) {
        H(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == p) {
      --p;
      iter = 0;
      continue;
    }
    if (l == p - 1) {
      max_imag = std::max(max_imag, split2(H, Z, p - 1));
      p -= 2;
      iter = 0;
      continue;
    }
    if (++iter > 80 || ++total > 60 * n) return -1;
    double s, t;
    if (iter % 11 == 10) {  // exceptional shift
      const double w = std::fabs(H(p, p - 1)) + std::fabs(H(p - 1, p - 2));
      const double sg = H(p, p) + 0.75 * w;
      s = 2.0 * sg;
      t = sg * sg;
    } else {
      s = H(p - 1, p - 1) + H(p, p);
      t = H(p - 1, p - 1) * H(p, p) - H(p - 1, p) * H(p, p - 1);
    }
    double x = H(l, l) * H(l, l) + H(l, l + 1) * H(l + 1, l) - s * H(l, l) + t;
    double y = H(l + 1, l) * (H(l, l) + H(l + 1, l + 1) - s);
    double z = H(l + 1, l) * H(l + 2, l + 1);
    for (int k = l; k <= p - 2; ++k) {
      const double xv[3] = {x, y, z};
      house(xv, 3, v, beta);
      const int q = std::max(l, k - 1);
      apply_left(H, k, 3, v, beta, q, n - 1);
      const int r = std::min(k + 3, p);
      apply_right(H, k, 3, v, beta, 0, r);
      apply_right(Z, k, 3, v, beta, 0, n - 1);
      x = H(k + 1, k);
      y = H(k + 2, k);
      if (k < p - 2) z = H(k + 3, k);
    }
    const double xv[2] = {x, y};
    house(xv, 2, v, beta);
    apply_left(H, p - 1, 2, v, beta, std::max(l, p - 2), n - 1);
    apply_right(H, p - 1, 2, v, beta, 0, p);
    apply_right(Z, p - 1, 2, v, beta, 0, n - 1);
  }
  return 0;
}

int eig_real(const Mat& A, std::vector<double>& w, Mat& V, double imag_tol, double* max_imag_out) {
  const int n = A.n;
  Mat H = A, Z;
  hessenberg(H, Z);
  double max_imag = 0.0;
  if (schur(H, Z, max_imag) != 0) return -1;
  double lam_max = 0.0;
  for (int i = 0; i < n; ++i) lam_max = std::max(lam_max, std::fabs(H(i, i)));
  if (max_imag_out) *max_imag_out = max_imag;
  if (max_imag > imag_tol * std::max(lam_max, 1e-300)) return -2;
  for (int i = 0; i + 1 < n; ++i) H(i + 1, i) = 0.0;  // any leftover (tiny-imag) block
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) tnorm = std::max(tnorm, std::fabs(H(i, j)));
  // eigenvectors of the triangular factor, then back to the original basis
  Mat Y(n, n);
  std::vector<double> y(n);
  for (int k = 0; k < n; ++k) {
    std::fill(y.begin(), y.end(), 0.0);
    y[k] = 1.0;
    const double lk = H(k, k);
    for (int j = k - 1; j >= 0; --j) {
      double s = 0.0;
      for (int i = j + 1; i <= k; ++i) s += H(j, i) * y[i];
      double den = H(j, j) - lk;
      if (std::fabs(den) < kEps * tnorm) den = (den >= 0 ? 1.0 : -1.0) * kEps * tnorm;
      y[j] = -s / den;
      if (std::fabs(y[j]) > 1e100) {
        for (int i = j; i <= k; ++i) y[i] *= 1e-100;
      }
    }
    for (int i = 0; i <= k; ++i) Y(i, k) = y[i];
  }
  Mat X = matmul(Z, Y);
  // normalise, sort ascending by eigenvalue
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return H(a, a) < H(b, b); });
  w.assign(n, 0.0);
  V = Mat(n, n);
  for (int c = 0; c < n; ++c) {
    const int k = idx[c];
    w[c] = H(k, k);
    double nrm = 0.0, big = 0.0;
    int ib = 0;
    for (int i = 0; i < n; ++i) {
      nrm += X(i, k) * X(i, k);
      if (std::fabs(X(i, k)) > big) {
        big = std::fabs(X(i, k));
        ib = i;
      }
    }
    nrm = std::sqrt(nrm);
    const double sg = X(ib, k) >= 0 ? 1.0 : -1.0;
    for (int i = 0; i < n; ++i) V(i, c) = sg * X(i, k) / nrm;
  }
  return 0;
}

static int lu(Mat& A, std::vector<int>& piv) {
  const int n = A.n;
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double big = std::fabs(A(k, k));
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A(i, k)) > big) {
        big = std::fabs(A(i, k));
        p = i;
      }
    piv[k] = p;
    if (big == 0.0) return -1;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A(k, j), A(p, j));
    const double inv = 1.0 / A(k, k);
    for (int i = k + 1; i < n; ++i) {
      const double f = (A(i, k) *= inv);
      if (f == 0.0) continue;
      for (int j = k + 1; j < n; ++j) A(i, j) -= f * A(k, j);
    }
  }
  return 0;
}

static void lu_solve(const Mat& LU, const std::vector<int>& piv, double* b) {
  const int n = LU.n;
  for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
  for (int i = 1; i < n; ++i) {
    double s = b[i];
    for (int j = 0; j < i; ++j) s -= LU(i, j) * b[j];
    b[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= LU(i, j) * b[j];
    b[i] = s / LU(i, i);
  }
}

int invert(const Mat& A, Mat& Ainv) {
  const int n = A.n;
  Mat LU = A;
  std::vector<int> piv;
  if (lu(LU, piv) != 0) return -1;
  Ainv = Mat(n, n);
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    std::fill(col.begin(), col.end(), 0.0);
    col[c] = 1.0;
    lu_solve(LU, piv, col.data());
    for (int i = 0; i < n; ++i) Ainv(i, c) = col[i];
  }
  return 0;
}

int solve(const Mat& A, std::vector<double>& x, const std::vector<double>& b) {
  Mat LU = A;
  std::vector<int> piv;
  if (lu(LU, piv) != 0) return -1;
  x = b;
  lu_solve(LU, piv, x.data());
  return 0;
}

}  // namespace fdetd
