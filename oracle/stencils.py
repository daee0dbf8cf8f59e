"""Exact rational finite-difference coefficients (oracle; test infrastructure only).

All coefficients are derived here from Taylor-matching conditions solved in
exact rational arithmetic (``fractions.Fraction``), then converted to float64.

* Staggered first derivative of order 2N (Sec. 2.3, Eq. spatial_derivativeSt):
      (d phi/dx)(x) ~ h^-1 sum_{n=1..N} c_n [phi(x+(n-1/2)h) - phi(x-(n-1/2)h)]
  Taylor matching gives  sum_n c_n (2n-1)^(2p+1) = delta_{p,0},  p = 0..N-1.
* Centred first derivative D^(C) of order 2N (Sec. 2.3 Eq. spatialAM_laplaceR,
  Sec. 4.2 Eq. spatialAM_envelope_H):
      h^-1 sum_n d_n [phi(x+nh) - phi(x-nh)],   sum_n d_n n^(2p+1) = delta_{p,0}/2.
* Centred second derivative D^2 of order 2N:
      h^-2 [e_0 phi(x) + sum_n e_n (phi(x+nh) + phi(x-nh))],
      sum_n e_n n^2 = 1,  sum_n e_n n^(2p) = 0 (p = 2..N),  e_0 = -2 sum_n e_n.
* Axis extrapolation (Sec. 2.4): the value at rho = 0 of an even function from
  its samples at rho = k*dr, k = 1..N, by Lagrange interpolation in rho^2:
      c_k = prod_{j != k} j^2 / (j^2 - k^2).
  The paper prints the N = 5 (10th order) values 5/3, -20/21, 5/14, -5/63, 1/126.
"""
from fractions import Fraction

import numpy as np


def _solve_rational(a, b):
    """Gauss-Jordan elimination over the rationals: solve a x = b exactly."""
    n = len(b)
    m = [list(map(Fraction, row)) + [Fraction(bi)] for row, bi in zip(a, b)]
    for col in range(n):
        piv = next(r for r in range(col, n) if m[r][col] != 0)
        m[col], m[piv] = m[piv], m[col]
        pv = m[col][col]
        m[col] = [v / pv for v in m[col]]
        for r in range(n):
            if r != col and m[r][col] != 0:
                f = m[r][col]
                m[r] = [vr - f * vc for vr, vc in zip(m[r], m[col])]
    return [m[r][n] for r in range(n)]


def staggered_coeffs_exact(order):
    """c_1..c_N of the order-2N staggered first derivative (Sec. 2.3), as Fractions."""
    if order < 2 or order % 2:
        raise ValueError("order must be even and >= 2")
    N = order // 2
    a = [[(2 * n - 1) ** (2 * p + 1) for n in range(1, N + 1)] for p in range(N)]
    b = [1 if p == 0 else 0 for p in range(N)]
    return _solve_rational(a, b)


def centred_d1_coeffs_exact(order):
    """d_1..d_N of the order-2N centred first derivative D^(C), as Fractions."""
    N = order // 2
    a = [[n ** (2 * p + 1) for n in range(1, N + 1)] for p in range(N)]
    b = [Fraction(1, 2) if p == 0 else 0 for p in range(N)]
    return _solve_rational(a, b)


def centred_d2_coeffs_exact(order):
    """(e_0, [e_1..e_N]) of the order-2N centred second derivative D^2, as Fractions."""
    N = order // 2
    a = [[n ** (2 * p) for n in range(1, N + 1)] for p in range(1, N + 1)]
    b = [1 if p == 1 else 0 for p in range(1, N + 1)]
    e = _solve_rational(a, b)
    return -2 * sum(e), e


def axis_coeffs_exact(N):
    """c_1..c_N of the axis extrapolation (Sec. 2.4), as Fractions."""
    out = []
    for k in range(1, N + 1):
        c = Fraction(1)
        for j in range(1, N + 1):
            if j != k:
                c *= Fraction(j * j, j * j - k * k)
        out.append(c)
    return out


def staggered_coeffs(order):
    return np.array([float(c) for c in staggered_coeffs_exact(order)])


def centred_d1_coeffs(order):
    return np.array([float(c) for c in centred_d1_coeffs_exact(order)])


def centred_d2_coeffs(order):
    e0, e = centred_d2_coeffs_exact(order)
    return float(e0), np.array([float(c) for c in e])


def axis_coeffs(N):
    return np.array([float(c) for c in axis_coeffs_exact(N)])
