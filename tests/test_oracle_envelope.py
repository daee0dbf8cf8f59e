"""Pins of the envelope oracle (Sec. 4.1-4.2) against closed forms and a library expm (CPU only)."""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.special

from oracle import envelope as ev
from oracle import stencils as st


@pytest.mark.parametrize("order", [4, 8])
def test_radial_laplacian_on_bessel(order):
    # L_rho J0(k rho) = -k^2 J0(k rho) (m = 0, symmetric axis mirror), converging at order 2N
    k = 2.0
    errs = []
    for Nr in (24, 48):
        dr = 6.0 / Nr
        L = ev.radial_laplacian(Nr, order, dr)
        rho = (np.arange(Nr) + 0.5) * dr
        f = scipy.special.j0(k * rho)
        r = L @ f + k * k * f
        win = rho < 3.5
        errs.append(np.abs(r[win]).max())
    assert math.log2(errs[0] / errs[1]) > order - 1.5, errs


def test_radial_laplacian_m2_on_bessel():
    k, order = 2.0, 8
    errs = []
    for Nr in (24, 48):
        dr = 6.0 / Nr
        L = ev.radial_laplacian(Nr, order, dr, m=2)
        rho = (np.arange(Nr) + 0.5) * dr
        f = scipy.special.jv(2, k * rho)
        errs.append(np.abs((L @ f + k * k * f)[rho < 3.5]).max())
    assert math.log2(errs[0] / errs[1]) > order - 2.5, errs


def test_taylor_converges_to_expm():
    rng = np.random.default_rng(5)
    Nz, Nr, order, dz, dr = 8, 6, 4, 0.2, 0.25
    a = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    at = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    chi = 0.5 + rng.random((Nz, Nr))
    t = 0.05
    ra, rt = ev.envelope_expm(a, at, chi, order, dz, dr, t)
    sa, stt = ev.envelope_step(a, at, chi, order, 40, dz, dr, t / 8, nsteps=8)
    s = max(np.abs(ra).max(), np.abs(rt).max())
    assert np.abs(sa - ra).max() < 1e-12 * s and np.abs(stt - rt).max() < 1e-12 * s


@pytest.mark.parametrize("NT", [1, 2, 4])
def test_taylor_NT_is_the_truncated_series(NT):
    # On tiny grids the oracle's N_T-term step equals sum_{n<=N_T} (dt A)^n/n! with A the
    # assembled matrix (independent check of the term recursion and the dt/n scaling).
    rng = np.random.default_rng(9)
    Nz, Nr, order, dz, dr, dt = 6, 5, 4, 0.2, 0.25, 0.01
    a = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    at = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    chi = rng.random((Nz, Nr))
    A = ev.envelope_matrix(Nz, Nr, chi, order, dz, dr)
    P = sum(np.linalg.matrix_power(dt * A, n) / math.factorial(n) for n in range(NT + 1))
    x = P @ np.concatenate([a.ravel(), at.ravel()])
    sa, stt = ev.envelope_step(a, at, chi, order, NT, dz, dr, dt)
    n = Nz * Nr
    np.testing.assert_allclose(sa.ravel(), x[:n], atol=1e-12)
    np.testing.assert_allclose(stt.ravel(), x[n:], atol=1e-12)


@pytest.mark.parametrize("q", [1, 3, 7])
def test_separable_mode_closed_form(q):
    # a = alpha v(rho) e^{i theta i}, a~ = beta v(rho) e^{i theta i} with L_rho v = -nu v and uniform chi:
    # H_a reduces to [[0, 1], [-nu - K2 - chi0 - 2 k0 K1, 2 i k0]], K2, K1 the z-stencil symbols,
    # so N_T Taylor terms act as the 2x2 polynomial (complex form of Eq. spatialAM_envelope_H).
    Nz, Nr, order, dz, dr, dt, NT = 16, 10, 8, 0.2, 0.25, 0.05, 4
    chi0, k0 = 0.7, 2 * np.pi
    L = ev.radial_laplacian(Nr, order, dr)
    w, V = np.linalg.eig(L)
    j = int(np.argmax(w.real))
    nu, v = -w[j].real, V[:, j].real
    th = 2 * np.pi * q / Nz
    e0, e = st.centred_d2_coeffs(order)
    d = st.centred_d1_coeffs(order)
    K2 = -(e0 + 2 * sum(e[n - 1] * np.cos(n * th) for n in range(1, len(e) + 1))) / dz ** 2
    K1 = 2 * sum(d[n - 1] * np.sin(n * th) for n in range(1, len(d) + 1)) / dz
    M = np.array([[0, 1], [-nu - K2 - chi0 - 2 * k0 * K1, 2j * k0]])
    P = sum(np.linalg.matrix_power(dt * M, n) / math.factorial(n) for n in range(NT + 1))
    alpha, beta = 0.3 - 0.2j, 1.1 + 0.4j
    phase = np.exp(1j * th * np.arange(Nz))[:, None]
    a, at = alpha * phase * v[None, :], beta * phase * v[None, :]
    sa, stt = ev.envelope_step(a, at, np.full((Nz, Nr), chi0), order, NT, dz, dr, dt)
    na, nb = P @ np.array([alpha, beta])
    np.testing.assert_allclose(sa, na * phase * v[None, :], atol=1e-12)
    np.testing.assert_allclose(stt, nb * phase * v[None, :], atol=1e-12)


def test_absorbing_step_without_layer_is_the_plain_step():
    rng = np.random.default_rng(7)
    Nz, Nr = 32, 12
    a = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    at = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    chi = 0.3 * rng.random((Nz, Nr))
    x = ev.envelope_step_absorbing(a, at, chi, np.zeros((Nz, Nr)), 4, 4, 0.2, 0.25, 0.05, nsteps=2)
    y = ev.envelope_step(a, at, chi, 4, 4, 0.2, 0.25, 0.05, nsteps=2)
    assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])


def test_absorbing_step_with_a_uniform_layer_factorises():
    # a constant sigma commutes with H_a: the step is exp(-sigma dt / 2) times the plain step with chi + sigma^2
    rng = np.random.default_rng(8)
    Nz, Nr, s0, dt = 32, 12, 0.7, 0.05
    a = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    at = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    chi = 0.3 * rng.random((Nz, Nr))
    x = ev.envelope_step_absorbing(a, at, chi, np.full((Nz, Nr), s0), 4, 4, 0.2, 0.25, dt, nsteps=3)
    y = ev.envelope_step(a, at, chi + s0 ** 2, 4, 4, 0.2, 0.25, dt, nsteps=3)
    f = np.exp(-s0 * dt / 2) ** 3
    assert np.allclose(x[0], f * y[0], rtol=1e-13, atol=0) and np.allclose(x[1], f * y[1], rtol=1e-13, atol=0)


def test_absorbing_layer_absorbs_an_outgoing_pulse():
    # a pulse travelling in +z (at ~c) through a layer occupying the upper part of the periodic box is
    # absorbed there, while without the layer it keeps nearly all of its norm
    Nz, Nr, order, NT, dz, dr, dt = 192, 12, 4, 4, 0.25, 0.5, 0.05
    z = np.arange(Nz) * dz
    r = (np.arange(Nr) + 0.5) * dr
    zc, tau, w0, z0 = 20.0, 2.0, 3.0, 28.0
    a = (np.exp(-((z - zc) / tau) ** 2)[:, None] * np.exp(-(r / w0) ** 2)[None, :]).astype(complex)
    at = np.zeros_like(a)
    chi = np.zeros((Nz, Nr))
    ramp = np.clip((z - z0) / (z[-1] - z0), 0.0, None)
    sigma = np.repeat((4.0 * ramp ** 2)[:, None], Nr, axis=1)
    nsteps = 600                      # 30 time units: the pulse crosses the whole layer
    x = ev.envelope_step_absorbing(a, at, chi, sigma, order, NT, dz, dr, dt, nsteps=nsteps)
    y = ev.envelope_step(a, at, chi, order, NT, dz, dr, dt, nsteps=nsteps)
    kept = np.linalg.norm(y[0]) / np.linalg.norm(a)
    absorbed = np.linalg.norm(x[0]) / np.linalg.norm(a)
    # >= 50x in amplitude, >= 2500x in energy (a stronger layer reflects more of the pulse)
    assert kept > 0.5 and absorbed < 0.02 * kept, (kept, absorbed)


def _centroid_delay(w0, chi0, dz=1 / 16, Nz=320, T=4.0):
    # 1 - v_g of a forward Gaussian envelope (a~ = -D_z a) in a uniform plasma chi0, from its |a|^2 centroid
    dr, Nr, order, NT = 0.25, 56, 8, 4
    dt = dz / 4
    z = np.arange(Nz) * dz
    rho = (np.arange(Nr) + 0.5) * dr
    zc = Nz * dz / 2 - T / 2 - 1
    a = np.exp(-(z[:, None] - zc) ** 2 / 4.0) * np.exp(-rho[None, :] ** 2 / w0 ** 2) + 0j
    at = -ev.d1_z(a, order, dz)

    def centroid(x):
        w = np.abs(x) ** 2 * rho[None, :]
        return (w.sum(axis=1) @ z) / w.sum()
    n = int(round(T / dt))
    a1, _ = ev.envelope_step(a, at, np.full((Nz, Nr), chi0), order, NT, dz, dr, dt, nsteps=n)
    return 1 - (centroid(a1) - centroid(a)) / (n * dt)


def test_envelope_group_velocity_in_a_uniform_plasma():
    # 1 - v_g = n0 / (2 n_c) + (lambda / 2 pi w0)^2 (Sec. 5.2, Eq. test_am_plasma_vg; the paper notes the formula is
    # analytical but not exact): chi0 = k0^2 n0 / n_c, so n0 / (2 n_c) = chi0 / (2 k0^2); centroid as in
    # Eq. test_am_vacuum_Z, of |a|^2 weighted by rho
    k0 = ev.K0
    runs = {(3.0, 0.01): None, (3.0, 0.02): None, (4.0, 0.01): None}
    for w0, dens in runs:
        runs[(w0, dens)] = _centroid_delay(w0, k0 ** 2 * dens)
    for (w0, dens), d in runs.items():
        pred = dens / 2 + 1 / (k0 * w0) ** 2
        assert abs(d / pred - 1) < 0.03, (w0, dens, d, pred)
    # the density and waist dependences separately
    dd = runs[(3.0, 0.02)] - runs[(3.0, 0.01)]
    assert abs(dd / 0.005 - 1) < 0.02, dd
    dw = runs[(3.0, 0.01)] - runs[(4.0, 0.01)]
    assert abs(dw / (1 / (k0 * 3.0) ** 2 - 1 / (k0 * 4.0) ** 2) - 1) < 0.02, dw
