"""Pins of the oracle's truncated-z option (the paper's own z boundary, Sec. 2.2 after Eq. bandedmatricesAM_Az:
stencil taps beyond the ends of the z grid dropped), which only the real-space evaluators (ii) and (iii) take."""
import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import maxwell as mx

pytestmark = pytest.mark.filterwarnings("ignore")


def _matrix(op, Nz, order, truncated):
    return np.stack([op(np.eye(Nz)[:, k], order, 1.0, truncated=truncated) for k in range(Nz)], axis=1)


@pytest.mark.parametrize("order", [2, 4, 8])
def test_truncated_z_differences_are_negative_transposes(order):
    # the integer -> half and half -> integer differences with the ends dropped are the restrictions of the two
    # infinite Toeplitz operators, which are negative transposes of each other (summation by parts): a tap kept
    # or dropped on one side only, or a stencil shifted by one, breaks it; the periodic pair keeps it too
    Nz = 13
    for truncated in (False, True):
        Dm = _matrix(mx.dz_minus, Nz, order, truncated)
        Dp = _matrix(mx.dz_plus, Nz, order, truncated)
        assert np.abs(Dp + Dm.T).max() < 1e-13
    # truncation changes only rows whose stencil reaches past an end
    N = order // 2
    Dm_t, Dm_p = _matrix(mx.dz_minus, Nz, order, True), _matrix(mx.dz_minus, Nz, order, False)
    diff_rows = np.flatnonzero(np.abs(Dm_t - Dm_p).max(axis=1) > 0)
    assert set(diff_rows) == set(range(N)) | set(range(Nz - N + 1, Nz))


def test_truncation_is_invisible_away_from_the_ends():
    # the Taylor polynomial of a banded operator spreads a field by (terms x half-width) cells: a pulse whose
    # spread stays inside the grid advances identically under both z boundaries
    rng = np.random.default_rng(3)
    Nz, Nr, order, dz, dr, m = 64, 8, 4, 0.25, 0.3, 1
    F = np.zeros((6, Nz, Nr), complex)
    F[:, 28:36, :] = rng.standard_normal((6, 8, Nr)) + 1j * rng.standard_normal((6, 8, Nr))
    a = mx.step_taylor(F, None, Nz, Nr, m, order, dz, dr, 0.05, taylor_order=6, substeps=1)
    b = mx.step_taylor(F, None, Nz, Nr, m, order, dz, dr, 0.05, taylor_order=6, substeps=1, truncated=True)
    assert np.abs(a - b).max() < 1e-14 * np.abs(a).max()
    # while a pulse at an end does see the boundary
    G = np.roll(F, -30, axis=1)
    a = mx.step_taylor(G, None, Nz, Nr, m, order, dz, dr, 0.05, taylor_order=6, substeps=1)
    b = mx.step_taylor(G, None, Nz, Nr, m, order, dz, dr, 0.05, taylor_order=6, substeps=1, truncated=True)
    assert np.abs(a - b).max() > 1e-3 * np.abs(a).max()


@pytest.mark.parametrize("m", [0, 1, 2])
def test_truncated_evaluators_agree(m):
    rng = np.random.default_rng(11 + m)
    Nz, Nr, order, dz, dr, dt = 8, 7, 4, 0.25, 0.3, 0.2
    F = rng.standard_normal((6, Nz, Nr)) + 1j * rng.standard_normal((6, Nz, Nr))
    J = rng.standard_normal((3, Nz, Nr)) + 1j * rng.standard_normal((3, Nz, Nr))
    b = mx.step_expm_realspace(F, J, Nz, Nr, m, order, dz, dr, dt, nsteps=3, truncated=True)
    c = mx.step_taylor(F, J, Nz, Nr, m, order, dz, dr, dt, nsteps=3, truncated=True)
    p = mx.step_expm_realspace(F, J, Nz, Nr, m, order, dz, dr, dt, nsteps=3)
    s = np.abs(b).max()
    assert np.abs(c - b).max() < 1e-12 * s
    assert np.abs(p - b).max() > 1e-3 * s          # a different operator from the periodic one


@pytest.mark.parametrize("m", [0, 1, 3])
def test_truncated_divergences_evolve_exactly(m):
    # the z and radial differences act on different axes, so the discrete div (curl) = 0 identities hold with
    # the truncated z differences too: div B is conserved and div E changes by -n dt div J exactly
    rng = np.random.default_rng(5 + m)
    Nz, Nr, order, dz, dr, dt, n = 10, 8, 4, 0.25, 0.3, 0.15, 2
    rad = mx.Radial(Nr, order, dr, m)
    F = mx.fill_axis(mx._zero_axis_slots(rng.standard_normal((6, Nz, Nr)) + 1j * rng.standard_normal((6, Nz, Nr))),
                     rad)
    J = rng.standard_normal((3, Nz, Nr)) + 1j * rng.standard_normal((3, Nz, Nr))
    J[0, :, 0] = 0
    G = mx.step_expm_realspace(F, J, Nz, Nr, m, order, dz, dr, dt, nsteps=n, truncated=True)
    scale = np.abs(F).max() * (1 / dz + 1 / dr) * 10
    dB0, dB1 = dg.div_B(F, rad, order, dz, True), dg.div_B(G, rad, order, dz, True)
    assert np.abs(dB1 - dB0).max() < 1e-11 * scale
    dE0, dE1 = dg.div_E(F, rad, order, dz, True), dg.div_E(G, rad, order, dz, True)
    dJ = dg.div_J(J, rad, order, dz, True)
    assert np.abs(dE1 - (dE0 - n * dt * dJ)).max() < 1e-11 * scale
