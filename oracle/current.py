"""The current pipeline in front of the field step (oracle; test infrastructure only).

Follows Sec. 2.5 (Eqs. spatialAM_filter_Jr, _Jz) and the current correction of Sec. 3 (Eqs.
shapesAM_currentRHS2m ... shapesAM_currentJth), in the complex mode convention of the field step
(d/dtheta -> i sigma m, sigma = -1):

* the current is deposited on the primary grids; J_rho is moved down to the staggered radial grid
  of E_rho by the Lagrange downstagger S_rho^(-, mA) of Eq. spatialAM_staggerS (order 2 N_D, primary
  nodes below the axis mirror to -1-j with the mA sign, nodes past the outer edge dropped);
  the z filters F_z, F_z^(div) are the identity (the paper defines them in its companion work);
* the planar divergence error  delta = rho_xy - div_perp J,  div_perp J = Div^+ J_rho + (i sigma m / rho) J_theta;
* the planar Poisson equation  [L_rho^(mS) - m^2 rho^-2] phi = delta  per z row, with the centred
  radial Laplacian L_rho = D^2_rho + rho^-1 D^(C)_rho of Eq. spatialAM_laplaceR (the operator the paper
  uses for stability), solved by a dense solve here;
* the correction  J_rho += D^- phi,  J_theta += (i sigma m / rho) phi,  J_z unchanged
  (J + grad_perp phi: the vector form the paper states, with grad_perp in the complex convention above).
Arrays: J [3][Nz][Nr] complex (J_rho, J_theta at (z_i, rho_k); J_z at (z_i - dz/2, rho_k)),
rho_xy [Nz][Nr] complex at (z_i, rho_k).  The result is on the field step's Yee locations (J_rho at
rho_-,k, slot 0 = its value on the axis; J_theta, J_z unchanged positions).
"""
import numpy as np

from .destagger import half_point_weights
from .envelope import radial_laplacian
from .maxwell import Radial, TAU


def s_rho_minus(f, order, symmetric):
    """f[Nz][Nr] at rho_k = (k + 1/2) dr -> values at rho_-,k = k dr (Eq. spatialAM_staggerS, downward)."""
    nodes, w = half_point_weights(order)
    Nr = f.shape[-1]
    out = np.zeros_like(f)
    sign = 1.0 if symmetric else -1.0
    for k in range(Nr):
        # rho_-,k is the half point above primary node k - 1
        for t, wt in zip(nodes, w):
            j = k - 1 + t
            if j < 0:
                out[..., k] += float(wt) * sign * f[..., -1 - j]
            elif j < Nr:
                out[..., k] += float(wt) * f[..., j]
    return out


def divergence_perp(Jr, Jt, rad):
    """Div^+ J_rho + (i sigma m / rho) J_theta on the primary grid (J_rho staggered, slot 0 unused)."""
    return (rad.rhom[None, :] * Jr) @ rad.Dp.T / rad.rho[None, :] + TAU * rad.m * Jt / rad.rho[None, :]


def current_pipeline(J, rho_xy, m, order, dr):
    Nz, Nr = rho_xy.shape
    rad = Radial(Nr, order, dr, m)
    Jr = s_rho_minus(J[0], order, abs(m - 1) % 2 == 0)
    Jt, Jz = J[1].copy(), J[2].copy()
    delta = rho_xy - divergence_perp(Jr, Jt, rad)
    A = radial_laplacian(Nr, order, dr, m)
    phi = np.linalg.solve(A, delta.T).T
    Jr = Jr + phi @ rad.Dm.T
    Jt = Jt + TAU * m * phi / rad.rho[None, :]
    return np.stack([Jr, Jt, Jz]), phi
