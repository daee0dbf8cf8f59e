"""Pins of the destagger oracle (Sec. 3 field interpolation, Eq. spatialAM_staggerS)."""
import os
from fractions import Fraction

import math

import numpy as np
import pytest
import scipy.interpolate

from oracle import destagger as ds
from paper_2605_12132_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "half_point_weights.txt")


def test_half_point_weights_match_the_classical_midpoint_formulas():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for order in (2, 4):
        nodes, w = ds.half_point_weights(order)
        want = {int(r[1]): Fraction(int(r[2]), int(r[3])) for r in rows if int(r[0]) == order}
        assert dict(zip(nodes, w)) == want


@pytest.mark.parametrize("order", [6, 8, 16])
def test_half_point_weights_equal_the_lagrange_interpolant(order):
    nodes, w = ds.half_point_weights(order)
    rng = np.random.default_rng(order)
    y = rng.standard_normal(len(nodes))
    poly = scipy.interpolate.lagrange(np.array(nodes, float), y)
    assert abs(poly(0.5) - sum(float(a) * b for a, b in zip(w, y))) < 1e-10 * np.abs(y).sum()


@pytest.mark.parametrize("order", [4, 8])
def test_z_upstagger_converges_at_its_order(order):
    errs = []
    for Nz in (32, 64):
        dz = 1.0 / Nz
        zs = (np.arange(Nz) - 0.5) * dz                      # staggered nodes (i - 1/2) dz
        f = np.cos(2 * np.pi * 3 * zs)[:, None] * np.ones((1, 3))
        got = ds.s_z_plus(f, order)
        exact = np.cos(2 * np.pi * 3 * np.arange(Nz) * dz)[:, None]
        errs.append(np.abs(got - exact).max())
    rate = np.log2(errs[0] / errs[1])
    assert rate > order - 0.7, (errs, rate)


def _lagrange_bound(order, h):
    """Twice the Lagrange remainder bound of the half-point value from the 2 N_D nodes t = -N_D+1 .. N_D
    for cos(a x) or sin(a x) sampled at spacing dr (|f^(2 N_D)| <= a^(2 N_D)), h = a dr."""
    N = order // 2
    prod = np.prod([abs(0.5 - t) for t in range(-N + 1, N + 1)])
    return 2 * prod / math.factorial(order) * h ** order


@pytest.mark.parametrize("order", [4, 8])
def test_radial_upstagger_parity_at_the_axis(order):
    # even function with the symmetric extension, odd function with the antisymmetric one: high-order
    # accurate at every radius including the first cells; the wrong extension fails near the axis
    Nr, dr, a = 24, 0.1, 1.7
    rm = np.arange(Nr) * dr                 # staggered nodes, slot 0 on the axis
    rp = (np.arange(Nr) + 0.5) * dr         # primary targets
    even, odd = np.cos(a * rm)[None, :], np.sin(a * rm)[None, :]
    inner = slice(0, Nr - order)            # away from the dropped outer taps
    ge = ds.s_rho_plus(even, order, True)[0]
    go = ds.s_rho_plus(odd, order, False)[0]
    tol = _lagrange_bound(order, a * dr)
    assert np.abs(ge - np.cos(a * rp))[inner].max() < tol
    assert np.abs(go - np.sin(a * rp))[inner].max() < tol
    assert np.abs(ds.s_rho_plus(even, order, False)[0] - np.cos(a * rp))[:2].max() > 1e-3
    assert np.abs(ds.s_rho_plus(odd, order, True)[0] - np.sin(a * rp))[:2].max() > 1e-3


@pytest.mark.parametrize("m", [0, 1, 2])
def test_destagger_moves_every_field_to_the_primary_grids(m):
    # smooth fields with the axis behaviour of Table tab:spatialAM_boundary, sampled on the Yee grid:
    # after destaggering they match the same functions sampled at (i dz, (k + 1/2) dr)
    Nz, Nr, dz, dr, order = 64, 32, 1 / 64, 1 / 16, 8
    kz, a = 2 * np.pi * 2, 2.3
    even = lambda r: np.cos(a * r)
    odd = lambda r: np.sin(a * r)
    polar = even if abs(m - 1) % 2 == 0 else odd
    scalar = even if m % 2 == 0 else odd
    radial = (polar, polar, scalar, polar, polar, scalar)
    F, want = np.zeros((6, Nz, Nr), complex), np.zeros((6, Nz, Nr), complex)
    for f in range(6):
        z, r = inputs.yee_positions(Nz, Nr, dz, dr, f)
        F[f] = np.exp(1j * kz * z)[:, None] * radial[f](r)[None, :]
        zp, rp = np.arange(Nz) * dz, (np.arange(Nr) + 0.5) * dr
        want[f] = np.exp(1j * kz * zp)[:, None] * radial[f](rp)[None, :]
    got = ds.destagger(F, m, order)
    inner = slice(0, Nr - order)
    for f in range(6):
        assert np.abs(got[f] - want[f])[:, inner].max() < 1e-6, f
