"""Seeded synthetic inputs (shared by the tests, the bench and the oracle checks).

This module holds no arithmetic of the method itself: it only samples analytic
pulse shapes on the Yee grid, draws seeded smooth random currents and
susceptibility profiles, and describes the standard workloads.  Everything is
numpy on the host; callers move the arrays to the device themselves.

Units: c = 1, lengths in laser wavelengths, k0 = 2*pi (Sec. 1, normalised units).
Field layout per mode: [6][Nz][Nr] complex (Er, Etheta, Ez, Br, Btheta, Bz);
current layout per mode: [3][Nz][Nr] complex (Jr, Jtheta, Jz) on E's Yee locations.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

K0 = 2 * np.pi
_STAG_R = (True, False, False, False, True, True)
_STAG_Z = (False, False, True, True, True, False)


@dataclass
class Workload:
    name: str
    Nz: int
    Nr: int
    modes: List[int]
    order: int
    dz: float
    dr: float
    dt: float
    steps: int
    waist: float            # pulse waist (wavelengths)
    tau: float = 8.0        # pulse duration (wavelengths, 1/e amplitude half-width)
    pulse_mode: int = 1     # the mode carrying the x-polarised pulse
    with_J: bool = False
    J_rms: float = 1e-2
    J_corr: float = 8.0     # correlation length of J in cells
    seed: int = 0
    notes: str = ""


def workload(name):
    """The standard workloads (sizes of the vacuum, current-driven and precision-sweep cases)."""
    if name == "vacuum_m1_256x64":
        return Workload(name, 256, 64, [1], 8, 1 / 16, 1 / 4, 1 / 16, 200, waist=16 / 4)
    if name == "lwfa_m01_2048x256":
        return Workload(name, 2048, 256, [0, 1], 16, 1 / 16, 1 / 4, 1 / 16, 1000,
                        waist=40 / 4, with_J=True)
    if name == "sweep_m012_8192x512":
        return Workload(name, 8192, 512, [0, 1, 2], 16, 1 / 16, 1 / 4, 1 / 16, 1000,
                        waist=40 / 4, with_J=True)
    raise KeyError(name)


def yee_positions(Nz, Nr, dz, dr, f):
    """(z, rho) sample positions of field f (0..5) on the Yee grid (Table tab:spatialAM_boundary)."""
    z = (np.arange(Nz) - (0.5 if _STAG_Z[f] else 0.0)) * dz
    r = (np.arange(Nr) + (0.0 if _STAG_R[f] else 0.5)) * dr
    return z, r


def pulse_fields(Nz, Nr, dz, dr, waist, tau, zc=None, amp=1.0):
    """x-polarised Gaussian pulse in the m = 1 mode, sampled at each field's own Yee position.

    E(z, rho) = amp exp(-rho^2/w0^2) exp(-(z-zc)^2/tau^2) cos(k0 (z - zc));
    Er = E, Etheta = -iE, Br = iE, Btheta = E, Ez = Bz = 0 (a forward wave; with the
    exp(-i m theta) mode convention this is E_x = E, E_y = 0, B_y = E).
    """
    if zc is None:
        zc = Nz * dz / 2
    coef = (1.0, -1j, 0.0, 1j, 1.0, 0.0)
    F = np.zeros((6, Nz, Nr), complex)
    for f in range(6):
        if coef[f] == 0:
            continue
        z, r = yee_positions(Nz, Nr, dz, dr, f)
        zz = z[:, None] - zc
        E = amp * np.exp(-(r[None, :] ** 2) / waist ** 2) * np.exp(-zz ** 2 / tau ** 2) * np.cos(K0 * zz)
        F[f] = coef[f] * E
    return F


def _gauss_matrix_r(Nr, sigma):
    """Row-normalised Gaussian smoothing along rho, mirrored at the axis, zero beyond Nr."""
    k = np.arange(Nr)
    G = np.exp(-((k[:, None] - k[None, :]) ** 2) / (2 * sigma ** 2))
    G += np.exp(-((k[:, None] + k[None, :] + 1) ** 2) / (2 * sigma ** 2))   # mirror image
    return G


def smooth_random(shape_zr, sigma, rng):
    """Complex white noise smoothed by a Gaussian of width sigma cells (periodic z, mirrored rho)."""
    Nz, Nr = shape_zr
    w = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    kz = np.fft.fftfreq(Nz)
    gz = np.exp(-2 * (np.pi * kz * sigma) ** 2)
    w = np.fft.ifft(np.fft.fft(w, axis=0) * gz[:, None], axis=0)
    return w @ _gauss_matrix_r(Nr, sigma).T


def random_current(Nz, Nr, mode, sigma=8.0, rms=1e-2, seed=0):
    """Seeded smooth random current of one mode: [3][Nz][Nr], component RMS = rms.

    Seed of component c of mode m is seed + 3*m + c.
    """
    J = np.zeros((3, Nz, Nr), complex)
    for c in range(3):
        rng = np.random.default_rng(seed + 3 * mode + c)
        w = smooth_random((Nz, Nr), sigma, rng)
        J[c] = w * (rms / np.sqrt(np.mean(np.abs(w) ** 2)))
    return J


def random_fields(Nz, Nr, seed=0, scale=1.0):
    """Seeded complex white-noise fields [6][Nz][Nr] (axis slots of staggered fields zeroed)."""
    rng = np.random.default_rng(seed)
    F = scale * (rng.standard_normal((6, Nz, Nr)) + 1j * rng.standard_normal((6, Nz, Nr)))
    for f in range(6):
        if _STAG_R[f]:
            F[f, :, 0] = 0
    return F


def workload_inputs(w: Workload, modes: Optional[List[int]] = None):
    """Fields [nmodes][6][Nz][Nr] and currents [nmodes][3][Nz][Nr] (or None) for a workload."""
    modes = w.modes if modes is None else modes
    F = np.zeros((len(modes), 6, w.Nz, w.Nr), complex)
    J = np.zeros((len(modes), 3, w.Nz, w.Nr), complex) if w.with_J else None
    for i, m in enumerate(modes):
        if m == w.pulse_mode:
            F[i] = pulse_fields(w.Nz, w.Nr, w.dz, w.dr, w.waist, w.tau)
        if w.with_J:
            J[i] = random_current(w.Nz, w.Nr, m, w.J_corr, w.J_rms, w.seed)
    for f in range(6):
        if _STAG_R[f]:
            F[:, f, :, 0] = 0
    return F, J


# ---------------------------------------------------------------------------
# Envelope inputs
# ---------------------------------------------------------------------------

@dataclass
class EnvelopeWorkload:
    name: str
    Nz: int
    Nr: int
    order: int
    taylor_order: int
    dz: float
    dr: float
    dt: float
    steps: int
    a0: float
    waist: float
    tau: float
    chi0: float
    chi_var: float = 0.1
    seed: int = 0


def envelope_workload(name):
    if name == "envelope_4096x256":
        dz = 1 / 5
        return EnvelopeWorkload(name, 4096, 256, 8, 4, dz, 1 / 4, 0.25 * dz, 100,
                                a0=2.0, waist=30 / 4, tau=12.5, chi0=(2 * np.pi) ** 2 * 1e-3)
    raise KeyError(name)


def envelope_inputs(w: EnvelopeWorkload, zc=None):
    """(a, a_tilde, chi): Gaussian envelope moving forward, seeded smooth chi(z, rho) >= 0.

    a = a0 exp(-rho^2/w0^2) exp(-(z-zc)^2/tau^2) on the primary grid; a_tilde = -da/dz
    (analytic), the forward-moving choice; chi = chi0 (1 + chi_var g), g in [-1, 1].
    """
    if zc is None:
        zc = w.Nz * w.dz / 2
    z = np.arange(w.Nz) * w.dz - zc
    r = (np.arange(w.Nr) + 0.5) * w.dr
    a = w.a0 * np.exp(-(r[None, :] ** 2) / w.waist ** 2) * np.exp(-(z[:, None] ** 2) / w.tau ** 2)
    at = (2 * z[:, None] / w.tau ** 2) * a
    rng = np.random.default_rng(w.seed + 1000)
    g = smooth_random((w.Nz, w.Nr), 8.0, rng).real
    g = g / np.abs(g).max()
    chi = w.chi0 * (1 + w.chi_var * g)
    return a.astype(complex), at.astype(complex), chi


# ---------------------------------------------------------------------------
# Uneven-instance mix (batched and served field requests)
# ---------------------------------------------------------------------------

NZ_POW2 = (512, 1024, 2048, 4096)


def uneven_instances(count, seed=0, nz_values=NZ_POW2):
    """Seeded draw of the uneven-instance mix: Nz from nz_values, even Nr in [64, 512], M in {1, 2, 3},
    order 8 or 16, m = 1 pulse with waist 10-40 dr (dz = 1/16, dr = 1/4, dt = dz), seeded current."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        Nz = int(rng.choice(list(nz_values)))
        Nr = 2 * int(rng.integers(32, 257))
        M = int(rng.integers(1, 4))
        order = int(rng.choice([8, 16]))
        waist = float(rng.uniform(10, 40)) * 0.25
        out.append(dict(Nz=Nz, Nr=Nr, M=M, order=order, waist=waist, seed=seed * 1000 + k))
    return out


def instance_inputs(c, tau=8.0):
    """Fields [M+1][6][Nz][Nr] and currents [M+1][3][Nz][Nr] (complex128) of one instance of the mix: the
    x-polarised pulse on m = 1, zero fields on the other modes, a seeded smooth random current (RMS 1e-2,
    correlation length 8 cells) on every mode."""
    Nz, Nr, M = c["Nz"], c["Nr"], c["M"]
    F = np.zeros((M + 1, 6, Nz, Nr), complex)
    F[1] = pulse_fields(Nz, Nr, 1 / 16, 1 / 4, c["waist"], tau)
    for f in range(6):
        if _STAG_R[f]:
            F[:, f, :, 0] = 0
    J = np.stack([random_current(Nz, Nr, m, 8.0, 1e-2, c["seed"]) for m in range(M + 1)])
    return F, J


# Three instances at the sizes of the uneven mix, used for parity of the batched launch against the oracle:
# the largest radial size with the most modes and order 16, a mid-size order-8 case, the longest z.
PARITY_INSTANCES = (
    dict(Nz=512, Nr=512, M=3, order=16, waist=10.0, seed=901),
    dict(Nz=1024, Nr=200, M=2, order=8, waist=6.25, seed=902),
    dict(Nz=4096, Nr=96, M=1, order=16, waist=2.5, seed=903),
)
