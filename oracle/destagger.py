"""Destaggering the Yee-grid field modes to the primary grids (oracle; test infrastructure only).

Follows the field-interpolation step of Sec. 3 (Eqs. shapesAM_destagger_E, _B, _Bth): every
staggered component is moved to the primary grids z_i = i dz, rho_k = (k + 1/2) dr with the
upstaggering Lagrange interpolation S^(+) of Eq. spatialAM_staggerS, of the same order 2 N_D as the
finite differences:
    E_rho -> S_rho^(+, mA) E_rho,   E_z -> S_z^(+) E_z,   B_rho -> S_z^(+) B_rho,
    B_z -> S_rho^(+, mS) B_z,       B_theta -> S_rho^(+, mA) S_z^(+) B_theta,   E_theta unchanged.
The value at the half point between nodes uses the 2 N_D nearest nodes, N_D on each side.  Along z
the grid is periodic, as for the field step.  Radially the operand sits on the staggered grid rho_-,j = j dr
with slot 0 on the axis holding the axis value (as the field step writes it); nodes j < 0 are the
mirror images rho_-,-j with the symmetric (S) or antisymmetric (A) extension chosen by the parity
rule of Eqs. spatialAM_derivativeS/A (mS: m even -> S; mA: |m - 1| even -> S); nodes beyond the
outer edge are dropped, as in the other radial operators (Sec. 2.2).
"""
from fractions import Fraction

import numpy as np


def half_point_weights(order):
    """Lagrange weights w_t, t = -N_D+1 .. N_D, of the value at t = 1/2 from the nodes t (exact)."""
    N = order // 2
    nodes = list(range(-N + 1, N + 1))
    w = []
    for i in nodes:
        num, den = Fraction(1), Fraction(1)
        for l in nodes:
            if l != i:
                num *= Fraction(1, 2) - l
                den *= i - l
        w.append(num / den)
    return nodes, w


def s_z_plus(f, order):
    """f[Nz][Nr] at z = (i - 1/2) dz -> values at z = i dz (periodic).

    Node i of the staggered array sits at (i - 1/2) dz, so the target i dz is the half point above
    node i: out[i] = sum_t w_t f[i + t] with the nodes t = -N_D+1 .. N_D.
    """
    nodes, w = half_point_weights(order)
    out = np.zeros_like(f)
    for t, wt in zip(nodes, w):
        out += float(wt) * np.roll(f, -t, axis=0)
    return out


def s_rho_plus(f, order, symmetric):
    """f[Nz][Nr] on rho_-,j = j dr (slot 0 = axis value) -> values at rho_k = (k + 1/2) dr."""
    nodes, w = half_point_weights(order)
    Nr = f.shape[-1]
    out = np.zeros_like(f)
    sign = 1.0 if symmetric else -1.0
    for k in range(Nr):
        for t, wt in zip(nodes, w):
            j = k + t
            if j < 0:
                out[..., k] += float(wt) * sign * f[..., -j]
            elif j < Nr:
                out[..., k] += float(wt) * f[..., j]
    return out


def destagger(F, m, order):
    """Fields [6][Nz][Nr] on the Yee grid (axis slots filled) -> the same fields on the primary grids."""
    sym_A = abs(m - 1) % 2 == 0
    sym_S = m % 2 == 0
    Er, Et, Ez, Br, Bt, Bz = F
    return np.stack([
        s_rho_plus(Er, order, sym_A),
        Et.copy(),
        s_z_plus(Ez, order),
        s_z_plus(Br, order),
        s_rho_plus(s_z_plus(Bt, order), order, sym_A),
        s_rho_plus(Bz, order, sym_S),
    ])
