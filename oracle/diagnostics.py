"""Discrete diagnostics of the Maxwell state (oracle; test infrastructure only).

* div E on the primary grid at integer z (Eq. spatialAM_divE, complex-mode form):
      D_div^(+) E_rho + i SIGMA m rho^-1 E_theta + D_z^(+) E_z
* div B on the staggered grid at half-integer z, the same construction applied to B
  (Br on the primary grid, Btheta and Bz on the staggered grid):
      D_div^(-) B_rho + i SIGMA m rho_(-)^-1 B_theta + D_z^(-) B_z        (rows k >= 1)
* energy W = dz dr sum (rho_(-) |Er|^2 + rho |Etheta|^2 + rho |Ez|^2
                       + rho |Br|^2 + rho_(-) |Btheta|^2 + rho_(-) |Bz|^2)
  over the state slots (the discrete form of the pulse energy of Eq. test_am_vacuum_E
  for one azimuthal mode, volume element rho drho dz).
"""
import numpy as np

from .maxwell import TAU, Radial, dz_minus, dz_plus


def div_E(F, rad, order, dz, truncated=False):
    Er, Et, Ez = F[0], F[1], F[2]
    div_r = ((rad.rhom[None, :] * Er) @ rad.Dp.T) / rad.rho
    return div_r + TAU * rad.m * Et / rad.rho + dz_plus(Ez, order, dz, truncated=truncated)


def div_J(J, rad, order, dz, truncated=False):
    return div_E(np.concatenate([J, np.zeros_like(J)]), rad, order, dz, truncated)


def div_B(F, rad, order, dz, truncated=False):
    Br, Bt, Bz = F[3], F[4], F[5]
    div_r = ((rad.rho[None, :] * Br) @ rad.Dm.T)[:, 1:] / rad.rhom[1:]
    return div_r + TAU * rad.m * Bt[:, 1:] / rad.rhom[1:] + dz_minus(Bz, order, dz, truncated=truncated)[:, 1:]


def energy(F, rad, dz):
    rho, rhom = rad.rho, rad.rhom
    w = 0.0
    for f, stag in zip(range(6), (True, False, False, False, True, True)):
        a = np.abs(F[f]) ** 2
        if stag:
            w += (a[:, 1:] * rhom[1:]).sum()
        else:
            w += (a * rho).sum()
    return w * dz * rad.dr


def radial_for(Nr, order, dr, m):
    return Radial(Nr, order, dr, m)
