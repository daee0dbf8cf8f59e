"""Pins of the current-pipeline oracle (Sec. 2.5 current stagger, Sec. 3 planar current correction) and of
the host-built bands and LU factors the GPU kernels use."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import current as cur
from oracle.envelope import radial_laplacian
from oracle.maxwell import Radial

native = pytest.importorskip("paper_2605_12132_gb300._native")


@pytest.mark.parametrize("order", [4, 8])
def test_downstagger_parity_at_the_axis(order):
    # primary nodes (k + 1/2) dr -> staggered k dr including the axis: even functions with the
    # symmetric extension, odd with the antisymmetric one
    Nr, dr, a = 24, 0.1, 1.7
    rp, rm = (np.arange(Nr) + 0.5) * dr, np.arange(Nr) * dr
    inner = slice(0, Nr - order)
    N = order // 2   # twice the Lagrange remainder bound of the half-point value, |f^(2N)| <= a^(2N)
    tol = 2 * np.prod([abs(0.5 - t) for t in range(-N + 1, N + 1)]) / math.factorial(order) * (a * dr) ** order
    ge = cur.s_rho_minus(np.cos(a * rp)[None, :], order, True)[0]
    go = cur.s_rho_minus(np.sin(a * rp)[None, :], order, False)[0]
    assert np.abs(ge - np.cos(a * rm))[inner].max() < tol
    assert np.abs(go - np.sin(a * rm))[inner].max() < tol
    assert abs(go[0]) < 1e-15                       # an odd field vanishes on the axis


def _smooth(rng, Nz, Nr, m):
    z = np.arange(Nz) / Nz
    r = (np.arange(Nr) + 0.5) / Nr
    out = np.zeros((Nz, Nr), complex)
    for _ in range(3):
        kz, kr = rng.integers(1, 3), rng.uniform(0.5, 3)
        out += rng.standard_normal() * np.exp(2j * np.pi * kz * z)[:, None] * (r ** max(m, 1) * np.cos(kr * r))[None, :]
    return out


@pytest.mark.parametrize("m", [0, 1, 2])
def test_consistent_current_is_left_unchanged(m):
    # if rho_xy already equals the planar divergence of the staggered current, phi = 0 exactly
    rng = np.random.default_rng(m)
    Nz, Nr, order, dr = 16, 20, 8, 0.25
    J = np.stack([_smooth(rng, Nz, Nr, m) for _ in range(3)])
    rad = Radial(Nr, order, dr, m)
    Jr = cur.s_rho_minus(J[0], order, abs(m - 1) % 2 == 0)
    rho_xy = cur.divergence_perp(Jr, J[1], rad)
    out, phi = cur.current_pipeline(J, rho_xy, m, order, dr)
    assert np.abs(phi).max() < 1e-12 * np.abs(rho_xy).max()
    assert np.allclose(out[1], J[1]) and np.array_equal(out[2], J[2])


def _gradient_residual(m, order, Nr, dr):
    # J_perp = grad_perp psi = (d psi / d rho, (i sigma m / rho) psi), sigma = -1, for psi = rho^m exp(-(rho / w)^2)
    # (parity m, decayed long before the outer radius), J_z arbitrary, rho_xy = 0
    Nz, w = 8, 0.2 * Nr * dr
    rp = (np.arange(Nr) + 0.5) * dr
    ez = np.exp(2j * np.pi * np.arange(Nz) / Nz)[:, None]
    g = np.exp(-(rp / w) ** 2)
    psi = rp ** m * g
    dpsi = (m * rp ** (m - 1) if m else 0.0) * g - 2 * rp ** (m + 1) / w ** 2 * g
    J = np.stack([ez * dpsi, ez * (-1j) * m * psi / rp, ez * psi])
    out, _ = cur.current_pipeline(J, np.zeros((Nz, Nr), complex), m, order, dr)
    return max(np.abs(out[c]).max() for c in range(2)) / max(np.abs(J[c]).max() for c in range(2))


@pytest.mark.parametrize("m", [0, 1, 2, 3])
def test_gradient_current_without_density_is_removed(m):
    # A planar gradient current with no density is pure divergence error: the correction phi = -psi removes
    # J_rho and J_theta entirely, up to the difference between the centred L_rho - m^2 rho^-2 of the solve and
    # the staggered composite Div+ D- of the divergence (both order 2 N_D): halving dr divides the residual by
    # about 2^8 at order 8.
    order = 8
    coarse, fine = _gradient_residual(m, order, 48, 0.1), _gradient_residual(m, order, 96, 0.05)
    assert fine < 1e-8, (coarse, fine)
    assert np.log2(coarse / fine) > order - 1, (coarse, fine)


@pytest.mark.parametrize("m", [0, 1, 2])
def test_correction_removes_most_of_the_planar_divergence_error(m):
    # smooth current and density that disagree: after the correction the planar divergence matches the
    # density up to the difference between L_rho (centred) and Div+ D- (staggered), both order 2 N_D
    rng = np.random.default_rng(10 + m)
    Nz, Nr, order, dr = 16, 48, 8, 1 / 16
    J = np.stack([_smooth(rng, Nz, Nr, m) for _ in range(3)])
    rho_xy = _smooth(rng, Nz, Nr, m)
    rad = Radial(Nr, order, dr, m)
    Jr0 = cur.s_rho_minus(J[0], order, abs(m - 1) % 2 == 0)
    before = np.abs(rho_xy - cur.divergence_perp(Jr0, J[1], rad))[:, : Nr - order].max()
    out, _ = cur.current_pipeline(J, rho_xy, m, order, dr)
    after = np.abs(rho_xy - cur.divergence_perp(out[0], out[1], rad))[:, : Nr - order].max()
    assert after < 1e-3 * before, (before, after)


@pytest.mark.parametrize("m", [0, 1, 3])
@pytest.mark.parametrize("order", [4, 8, 16])
def test_host_bands_and_lu_reproduce_the_oracle_operators(m, order):
    Nr, dr = 23, 0.25
    N = order // 2
    divp, dm, lo, up = native.fdetd_current_host_bands(Nr, order, dr, m)
    rad = Radial(Nr, order, dr, m)
    dense = lambda b: np.array([[b[k, j - k + N] if abs(j - k) <= N else 0.0 for j in range(Nr)] for k in range(Nr)])
    Div = rad.Dp * rad.rhom[None, :] / rad.rho[:, None]
    assert np.allclose(dense(divp), Div, atol=1e-12 * np.abs(Div).max())
    assert np.allclose(dense(dm), rad.Dm, atol=1e-12 * np.abs(rad.Dm).max())
    L = np.eye(Nr)
    U = np.zeros((Nr, Nr))
    for k in range(Nr):
        for d in range(1, N + 1):
            if k - d >= 0:
                L[k, k - d] = lo[k, d - 1]
        for d in range(0, N + 1):
            if k + d < Nr:
                U[k, k + d] = up[k, d]
    A = radial_laplacian(Nr, order, dr, m)
    assert np.allclose(L @ U, A, atol=1e-10 * np.abs(A).max())
    # the LU solve agrees with LAPACK's banded solver
    b = np.random.default_rng(1).standard_normal(Nr)
    ab = np.zeros((2 * N + 1, Nr))
    for k in range(Nr):
        for j in range(max(0, k - N), min(Nr, k + N + 1)):
            ab[N + k - j, j] = A[k, j]
    x = scipy.linalg.solve_banded((N, N), ab, b)
    y = scipy.linalg.solve_triangular(U, scipy.linalg.solve_triangular(L, b, lower=True, unit_diagonal=True))
    assert np.allclose(x, y, rtol=1e-10, atol=1e-12)
