"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in the oracle - a flipped sign, a wrong mirror index, a dropped term, a
transposed operand, a wrong phase - through monkeypatch, runs a pin that should see it, and expects that
pin to fail.  Nothing here touches the CUDA path.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

from oracle import current as cur
from oracle import destagger as ds
from oracle import envelope as ev
from oracle import maxwell as mx
from oracle import stencils as st
from tests import test_oracle_current as PC
from tests import test_oracle_destagger as PD
from tests import test_oracle_envelope as PE
from tests import test_oracle_pins as P
from tests import test_oracle_truncated_z as PT


def _c2_sign_flipped(mp):
    orig = st.staggered_coeffs_exact

    def bad(order):
        c = list(orig(order))
        if len(c) > 1:
            c[1] = -c[1]
        return c
    mp.setattr(st, "staggered_coeffs_exact", bad)


def _dminus_parity_ignored(mp):
    orig = mx.d_minus
    mp.setattr(mx, "d_minus", lambda Nr, order, dr, parity: orig(Nr, order, dr, 0))


def _dplus_primary_mirror(mp):
    # the staggered-grid operand mirrored as if it sat on the primary grid (-1 - j instead of -j)
    def bad(Nr, order, dr, parity):
        c = mx.staggered_coeffs(order)
        D = np.zeros((Nr, Nr))
        for k in range(Nr):
            for n in range(1, len(c) + 1):
                for j, w in ((k + n, c[n - 1]), (k - n + 1, -c[n - 1])):
                    if j < 0:
                        j, w = -1 - j, w * (-1) ** parity
                    if j < Nr:
                        D[k, j] += w
        return D / dr
    mp.setattr(mx, "d_plus", bad)


def _axis_value_dropped(mp):
    mp.setattr(mx, "axis_value_row", lambda Nr, order, constant_on_axis: np.zeros(Nr - 1))


def _z_symbol_phase_conjugated(mp):
    orig = mx.z_symbols

    def bad(Nz, order, dz):
        sp, sm = orig(Nz, order, dz)
        return -np.conj(sp), -np.conj(sm)   # i kappa e^{-i theta/2} for s+ and vice versa
    mp.setattr(mx, "z_symbols", bad)


def _kz_operator_transposed(mp):
    orig = mx.kz_operator
    mp.setattr(mx, "kz_operator", lambda rad, sp, sm: orig(rad, sp, sm).T)


def _half_step_propagator_dropped(mp):
    orig = mx._propagators

    def bad(H, dt, method):
        E1, Eh = orig(H, dt, method)
        return E1, np.eye(E1.shape[0])
    mp.setattr(mx, "_propagators", bad)


def _envelope_k0_drift_sign(mp):
    orig = ev.d1_z
    mp.setattr(ev, "d1_z", lambda f, order, dz: -orig(f, order, dz))


def _current_tau_term_dropped(mp):
    def bad(Jr, Jt, rad):
        return (rad.rhom[None, :] * Jr) @ rad.Dp.T / rad.rho[None, :]
    mp.setattr(cur, "divergence_perp", bad)


def _half_point_nodes_shifted(mp):
    def bad(order):
        N = order // 2
        nodes = list(range(-N, N))
        w = []
        for i in nodes:
            num, den = Fraction(1), Fraction(1)
            for l in nodes:
                if l != i:
                    num *= Fraction(1, 2) - l
                    den *= i - l
            w.append(num / den)
        return nodes, w
    mp.setattr(ds, "half_point_weights", bad)


def _correction_sign_flipped(mp):
    orig = cur.current_pipeline

    def bad(J, rho_xy, m, order, dr):
        out, phi = orig(J, rho_xy, m, order, dr)
        # J_rho -= D^- phi and J_theta -= (i sigma m / rho) phi instead of +=: undo the correction twice
        rad = mx.Radial(rho_xy.shape[1], order, dr, m)
        out = out.copy()
        out[0] = out[0] - 2 * phi @ rad.Dm.T
        out[1] = out[1] - 2 * cur.TAU * m * phi / rad.rho[None, :]
        return out, phi
    mp.setattr(cur, "current_pipeline", bad)


def _downstagger_mirror_index(mp):
    # the primary-grid operand mirrored as if it sat on the staggered grid (-j instead of -1 - j)
    def bad(f, order, symmetric):
        nodes, w = ds.half_point_weights(order)
        Nr = f.shape[-1]
        out = np.zeros_like(f)
        sign = 1.0 if symmetric else -1.0
        for k in range(Nr):
            for t, wt in zip(nodes, w):
                j = k - 1 + t
                if j < 0:
                    out[..., k] += float(wt) * sign * f[..., -j]
                elif j < Nr:
                    out[..., k] += float(wt) * f[..., j]
        return out
    mp.setattr(cur, "s_rho_minus", bad)


def _upstagger_mirror_index(mp):
    # the staggered operand mirrored as if it sat on the primary grid (-1 - j instead of -j)
    def bad(f, order, symmetric):
        nodes, w = ds.half_point_weights(order)
        Nr = f.shape[-1]
        out = np.zeros_like(f)
        sign = 1.0 if symmetric else -1.0
        for k in range(Nr):
            for t, wt in zip(nodes, w):
                j = k + t
                if j < 0:
                    out[..., k] += float(wt) * sign * f[..., -1 - j]
                elif j < Nr:
                    out[..., k] += float(wt) * f[..., j]
        return out
    mp.setattr(ds, "s_rho_plus", bad)


def _polar_axis_value_dropped(mp):
    def bad(F, rad):
        F = F.copy()
        F[0, :, 0] = 0
        F[4, :, 0] = 0
        F[5, :, 0] = F[5, :, 1:] @ rad.axis_scalar
        return F
    mp.setattr(mx, "fill_axis", bad)


def _full_step_uses_the_half_step(mp):
    orig = mx._propagators

    def bad(H, dt, method):
        E1, Eh = orig(H, dt, method)
        return Eh, Eh
    mp.setattr(mx, "_propagators", bad)


def _realspace_faraday_sign(mp):
    # dB_theta/dt = +D_z^- E_rho + D^- E_z instead of -D_z^- E_rho + D^- E_z in the real-space operator
    orig = mx.apply_H

    def bad(F, rad, order, dz, truncated=False):
        out = orig(F, rad, order, dz, truncated)
        out[4, :, 1:] += 2 * mx.dz_minus(F[0], order, dz, truncated=truncated)[:, 1:]
        return out
    mp.setattr(mx, "apply_H", bad)


def _absorbing_damping_once(mp):
    # exp(-sigma dt / 4) applied once per step instead of on both sides of the Taylor step
    def bad(a, at, chi, sigma, order, taylor_order, dz, dr, dt, nsteps=1, k0=ev.K0, m=0):
        damp = np.exp(-sigma * dt / 4)
        for _ in range(nsteps):
            a, at = a * damp, at * damp
            a, at = ev.envelope_step(a, at, chi + sigma ** 2, order, taylor_order, dz, dr, dt, 1, k0, m)
        return a, at
    mp.setattr(ev, "envelope_step_absorbing", bad)


def _truncation_at_one_end(mp):
    # the truncated z stencils drop the taps below the first point but wrap those past the last one
    def bad(f, s, axis, truncated):
        g = np.roll(f, -s, axis=axis)
        if truncated and s < 0:
            Nz = f.shape[axis]
            idx = np.arange(Nz) + s
            shape = [1] * f.ndim
            shape[axis] = Nz
            g = np.where((idx < 0).reshape(shape), 0, g)
        return g
    mp.setattr(mx, "_shift", bad)


def _exact_current_left_endpoint(mp):
    # the constant-current integral replaced by dt exp(dt H) J (the current taken at the start of the step)
    def bad(H, j, dt):
        return dt * (scipy.linalg.expm(H * dt) @ j)
    mp.setattr(mx, "_exact_current_source", bad)


def _envelope_chi_sign(mp):
    # the susceptibility entering with the wrong sign, (L - chi) a -> (L + chi) a
    orig = ev.apply_Ha

    def bad(a, at, chi, Lr, order, dz, k0=ev.K0):
        return orig(a, at, -chi, Lr, order, dz, k0)
    mp.setattr(ev, "apply_Ha", bad)


CASES = [
    ("staggered c_2 sign", _c2_sign_flipped, lambda: P.test_staggered_textbook_values()),
    ("D- mirror sign ignored", _dminus_parity_ignored, lambda: P.test_radial_derivative_convergence_near_axis(1, 4)),
    ("D+ mirrored like a primary-grid operand", _dplus_primary_mirror, lambda: P.test_L2_on_bessel(0)),
    ("B_z axis value dropped", _axis_value_dropped, lambda: P.test_axis_output_values()),
    ("z-symbol half-cell phase conjugated", _z_symbol_phase_conjugated, lambda: P.test_z_symbol_is_kappa(4)),
    ("per-kz operator transposed", _kz_operator_transposed, lambda: P.test_three_evaluators_agree(1)),
    ("half-step exponential on the current dropped", _half_step_propagator_dropped,
     lambda: P.test_three_evaluators_agree(1)),
    ("envelope 2 i k0 D_z term sign", _envelope_k0_drift_sign, lambda: PE.test_separable_mode_closed_form(3)),
    ("tau term of the planar divergence dropped", _current_tau_term_dropped,
     lambda: PC.test_gradient_current_without_density_is_removed(1)),
    ("upstagger nodes shifted by one", _half_point_nodes_shifted,
     lambda: PD.test_half_point_weights_match_the_classical_midpoint_formulas()),
    ("current correction applied with the wrong sign", _correction_sign_flipped,
     lambda: PC.test_gradient_current_without_density_is_removed(2)),
    ("downstagger mirror index", _downstagger_mirror_index, lambda: PC.test_downstagger_parity_at_the_axis(4)),
    ("upstagger mirror index", _upstagger_mirror_index, lambda: PD.test_radial_upstagger_parity_at_the_axis(4)),
    ("E_rho / B_theta axis value dropped for m = 1", _polar_axis_value_dropped, lambda: P.test_axis_output_values()),
    ("full step advanced by the half-step exponential", _full_step_uses_the_half_step,
     lambda: P.test_three_evaluators_agree(2)),
    ("Faraday sign in the real-space operator", _realspace_faraday_sign, lambda: P.test_three_evaluators_agree(0)),
    ("absorbing-layer damping on one side only", _absorbing_damping_once,
     lambda: PE.test_absorbing_step_with_a_uniform_layer_factorises()),
    ("truncated z stencil wraps at one end", _truncation_at_one_end,
     lambda: PT.test_truncated_z_differences_are_negative_transposes(4)),
    ("constant-current integral taken at the left end", _exact_current_left_endpoint,
     lambda: P.test_exact_current_variant_integrates_the_ode(1)),
    ("envelope susceptibility sign", _envelope_chi_sign, lambda: PE.test_envelope_group_velocity_in_a_uniform_plasma()),
]


@pytest.mark.parametrize("name,plant,pin", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(name, plant, pin, monkeypatch):
    pin()                      # the pin passes on the oracle as written
    with monkeypatch.context() as mp:
        plant(mp)
        with pytest.raises(AssertionError):
            pin()
