"""Exponential laser-envelope propagator (oracle; test infrastructure only).

Follows Sec. 4.1-4.2 of the paper.  The envelope a and its auxiliary variable
a~ = da/dt (Eqs. laserA_envelope_equation_A/At) obey

    da/dt  = a~
    da~/dt = (L_rho + L_z - chi) a + 2 i k0 D_z^(C) a + 2 i k0 a~

(the complex form of Eq. laserA_envelope_equation; the 4x4 real matrix printed
in Eq. laserA_envelope_H has the opposite sign on its k0 terms, i.e. the complex
conjugate equation, and this oracle follows the complex equation together with
the field formula |E| = |a~ - i k0 a| of Eq. laserA_envelope_E, which it matches).

Discretisation (Eq. spatialAM_envelope_H), mode m = 0 by default:
* L_rho = D^2_rho + rho^-1 D^(C)_rho on the primary grid (Eq. spatialAM_laplaceR),
  centred differences of order 2N, symmetric (mS) mirror at the axis for even m,
  taps beyond the outer edge dropped; for m != 0 the term -m^2 rho^-2 is added;
* L_z = D^2_z and D_z^(C) centred, periodic in z;
* chi(z, rho) real and frozen over the step.
One step applies the truncated Taylor series sum_{n<=N_T} (dt H_a)^n / n!
(Eq. laserA_envelope_solution expanded as in Sec. 4.2).
"""
import numpy as np
import scipy.linalg

from .stencils import centred_d1_coeffs, centred_d2_coeffs

K0 = 2 * np.pi


def radial_laplacian(Nr, order, dr, m=0):
    """L_rho^(mS) - m^2 rho^-2 as a dense Nr x Nr matrix on the primary grid."""
    e0, e = centred_d2_coeffs(order)
    d = centred_d1_coeffs(order)
    rho = (np.arange(Nr) + 0.5) * dr
    parity = m % 2
    L = np.zeros((Nr, Nr))
    for k in range(Nr):
        L[k, k] += e0 / dr ** 2
        for n in range(1, len(e) + 1):
            for j, w2, w1 in ((k + n, e[n - 1], d[n - 1]), (k - n, e[n - 1], -d[n - 1])):
                w = w2 / dr ** 2 + w1 / (dr * rho[k])
                if j < 0:
                    j, w = -1 - j, w * (-1) ** parity
                if j < Nr:
                    L[k, j] += w
        L[k, k] -= m * m / rho[k] ** 2
    return L


def d2_z(f, order, dz):
    e0, e = centred_d2_coeffs(order)
    out = e0 * f
    for n in range(1, len(e) + 1):
        out = out + e[n - 1] * (np.roll(f, -n, axis=0) + np.roll(f, n, axis=0))
    return out / dz ** 2


def d1_z(f, order, dz):
    d = centred_d1_coeffs(order)
    out = np.zeros_like(f)
    for n in range(1, len(d) + 1):
        out = out + d[n - 1] * (np.roll(f, -n, axis=0) - np.roll(f, n, axis=0))
    return out / dz


def apply_Ha(a, at, chi, Lr, order, dz, k0=K0):
    """(da/dt, da~/dt) of the discrete envelope operator (Eq. spatialAM_envelope_H, complex form)."""
    lap = a @ Lr.T + d2_z(a, order, dz)
    return at, lap - chi * a + 2j * k0 * d1_z(a, order, dz) + 2j * k0 * at


def envelope_step(a, at, chi, order, taylor_order, dz, dr, dt, nsteps=1, k0=K0, m=0):
    """nsteps of the Taylor-N_T exponential propagator; a, at: [Nz][Nr] complex128, chi real."""
    Lr = radial_laplacian(a.shape[1], order, dr, m)
    for _ in range(nsteps):
        ta, tt = a, at
        sa, st = a.copy(), at.copy()
        for n in range(1, taylor_order + 1):
            ta, tt = apply_Ha(ta, tt, chi, Lr, order, dz, k0)
            ta, tt = ta * (dt / n), tt * (dt / n)
            sa, st = sa + ta, st + tt
        a, at = sa, st
    return a, at


def envelope_matrix(Nz, Nr, chi, order, dz, dr, k0=K0, m=0):
    """Dense matrix of H_a on the stacked vector (a, a~) (tiny grids only)."""
    Lr = radial_laplacian(Nr, order, dr, m)
    n = Nz * Nr
    A = np.zeros((2 * n, 2 * n), complex)
    for col in range(2 * n):
        x = np.zeros(2 * n, complex)
        x[col] = 1
        a, at = x[:n].reshape(Nz, Nr), x[n:].reshape(Nz, Nr)
        da, dat = apply_Ha(a, at, chi, Lr, order, dz, k0)
        A[:, col] = np.concatenate([da.ravel(), dat.ravel()])
    return A


def envelope_expm(a, at, chi, order, dz, dr, t, k0=K0, m=0):
    """exp(t H_a) by scipy's expm on the assembled matrix (brute force, tiny grids)."""
    Nz, Nr = a.shape
    A = envelope_matrix(Nz, Nr, chi, order, dz, dr, k0, m)
    x = scipy.linalg.expm(A * t) @ np.concatenate([a.ravel(), at.ravel()])
    n = Nz * Nr
    return x[:n].reshape(Nz, Nr), x[n:].reshape(Nz, Nr)


def envelope_step_absorbing(a, at, chi, sigma, order, taylor_order, dz, dr, dt, nsteps=1, k0=K0, m=0):
    """The envelope step with the scalar absorbing layer of the appendix (Eq. absorbingA_solution2).

    The absorbing wave equation (Eqs. absorbingA_Adt, absorbingA_waveA with h = 1) adds -sigma/2 to
    both components and -sigma^2 a to da~/dt; the split-operator step damps (a, a~) pointwise by
    exp(-sigma dt / 4), applies the Taylor step of H_a with chi + sigma^2 (the sigma^2 term merged
    into the susceptibility as the appendix suggests), and damps again.
    """
    damp = np.exp(-sigma * dt / 4)
    for _ in range(nsteps):
        a, at = a * damp, at * damp
        a, at = envelope_step(a, at, chi + sigma ** 2, order, taylor_order, dz, dr, dt, 1, k0, m)
        a, at = a * damp, at * damp
    return a, at
