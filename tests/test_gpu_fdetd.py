"""GPU parity of the exact exponential field step against the FP64 oracle (through the C-ABI)."""
import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import maxwell as mx
from paper_2605_12132_gb300 import inputs
from tests.gpu_util import check_report, column_report, field_report, format_report, kz_columns, zero_axis

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

# Per-step relative error budget of each precision against the FP64 oracle, for fields that carry at
# least 10% of the state (relative L2 per field, floor 1e-12 of the state's norm):
#  fp64   - FP64 round trip: single-step agreement ~1e-13; the projection/back-projection pair
#           reproduces the identity only to ~1e-14 entrywise (it divides by the small radial
#           eigenvalues), so over many steps the difference grows ~1e-13 per step;
#  fp32   - FP32 storage + FP32 CUDA-core GEMMs + FP32 FFT: ~5e-7 per step;
#  bf16x6 - 3-piece bf16 operands (24 bits); the leading product and the correction products in separate
#           tensor-core accumulators (each MMA truncates its FP32 sum toward zero): <= 1e-6 per step up
#           to Nr = 256 (2e-6 at Nr = 512: the leading accumulation chain is twice as long);
#  bf16x3 - 2-piece bf16 operands (16 bits): representation error 2^-17 per operand, ~1e-5 per step.
TOL = {"fp64": 1e-12, "fp32": 1e-6, "bf16x6": 1e-6, "bf16x3": 2.5e-5}
# Fields under 10% of the state carry the state-scale absolute error of the radial transforms: measured on
# the 256 x 64 vacuum pulse, whose E_z and B_z hold 0.8% of the state, after one step (true relative
# error): fp32 1.2e-6, bf16x6 1.0e-6, bf16x3 1.2e-4 (element-wise at the axis slot, where the axis
# extrapolation adds its own amplification: 5e-6, 4.9e-6, 6.3e-4).
TOL_WEAK = {"fp64": 1e-12, "fp32": 3e-6, "bf16x6": 3e-6, "bf16x3": 3e-4}
ALL = ["fp64", "fp32", "bf16x3", "bf16x6"]


def _run(prec, F, J, Nz, Nr, modes, order, dz, dr, dt, nsteps):
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, order, dz, dr, dt, precision=prec)
    dt_c = plan.complex_dtype
    f = torch.from_numpy(F).to(dt_c).cuda()
    j = torch.from_numpy(J).to(dt_c).cuda() if J is not None else None
    fd.fdetd_step(plan, f, j, nsteps)
    torch.cuda.synchronize()
    return f.cpu().numpy().astype(np.complex128)


def _oracle(F, J, Nz, Nr, modes, order, dz, dr, dt, nsteps):
    return np.stack([mx.step_spectral(F[i], None if J is None else J[i], Nz, Nr, m, order, dz, dr, dt, nsteps=nsteps)
                     for i, m in enumerate(modes)])


@pytest.fixture(scope="module")
def ragged_case():
    # several z tiles, a ragged radial tail (70 = 64 + 6), modes 0..3, current on; the oracle runs once
    # for all precisions
    rng = np.random.default_rng(1)
    Nz, Nr, modes, order, dz, dr, dt = 128, 70, [0, 1, 2, 3], 8, 1 / 16, 1 / 4, 1 / 16
    F = zero_axis(rng.standard_normal((4, 6, Nz, Nr)) + 1j * rng.standard_normal((4, 6, Nz, Nr)))
    J = 0.3 * (rng.standard_normal((4, 3, Nz, Nr)) + 1j * rng.standard_normal((4, 3, Nz, Nr)))
    args = (Nz, Nr, modes, order, dz, dr, dt, 3)
    return F, J, args, _oracle(F, J, *args)


@pytest.mark.parametrize("prec", ALL)
def test_parity_small_ragged(prec, ragged_case):
    # random fields on every component (all fields strong), 3 steps: per-field L2, element-wise, and the
    # axis slot, the first N_D radii and the last N_D radii separately
    F, J, args, ref = ragged_case
    modes, order, nsteps = args[2], args[3], args[7]
    got = _run(prec, F, J, *args)
    for i in range(len(modes)):
        rows = field_report(got[i], ref[i], nd=order // 2)
        print("\n" + format_report(rows, f"{prec} m={modes[i]}"))
        check_report(rows, TOL[prec] * nsteps, TOL_WEAK[prec] * nsteps, label=f"{prec} m={modes[i]}")


@pytest.fixture(scope="module")
def vacuum_ref():
    w = inputs.workload("vacuum_m1_256x64")
    F, _ = inputs.workload_inputs(w)
    r1, r200 = mx.step_spectral(F[0], None, w.Nz, w.Nr, 1, w.order, w.dz, w.dr, w.dt, nsteps=[1, w.steps],
                                method="expm")
    return w, F, r1, r200


@pytest.mark.parametrize("prec", ALL)
def test_parity_vacuum_pulse_256x64(prec, vacuum_ref):
    # the 256 x 64 vacuum pulse (m = 1, order 8, dt = dz): after 1 step and after 200 steps
    w, F, r1, r200 = vacuum_ref
    nd = w.order // 2
    g1 = _run(prec, F, None, w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, 1)
    rows = field_report(g1[0], r1, nd=nd)
    print("\n" + format_report(rows, f"{prec} 1 step"))
    check_report(rows, TOL[prec], TOL_WEAK[prec], label=f"{prec} 1 step")
    g200 = _run(prec, F, None, w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, w.steps)
    rows = field_report(g200[0], r200, nd=nd)
    print(format_report(rows, f"{prec} {w.steps} steps"))
    # error grows at most linearly with the step count (fp64: a quarter of that, ~1e-13 per step)
    t = TOL[prec] * (0.25 if prec == "fp64" else 1) * w.steps
    check_report(rows, t, t, label=f"{prec} {w.steps} steps")


def test_zero_steps_and_null_current():
    rng = np.random.default_rng(2)
    Nz, Nr, modes = 64, 20, [1]
    F = zero_axis(rng.standard_normal((1, 6, Nz, Nr)) + 1j * rng.standard_normal((1, 6, Nz, Nr)))
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, 4, 0.1, 0.2, 0.05, precision="fp64")
    f = torch.from_numpy(F).cuda()
    fd.fdetd_step(plan, f, None, 0)
    assert np.array_equal(f.cpu().numpy(), F)
    f1 = torch.from_numpy(F).cuda()
    f2 = torch.from_numpy(F).cuda()
    fd.fdetd_step(plan, f1, None, 2)
    fd.fdetd_step(plan, f2, torch.zeros((1, 3, Nz, Nr), dtype=torch.complex128, device="cuda"), 2)
    torch.cuda.synchronize()
    assert np.abs(f1.cpu().numpy() - f2.cpu().numpy()).max() < 1e-14


def test_argument_errors():
    with pytest.raises(fd.FdetdError):
        fd.fdetd_plan_modes(100, 32, [0], 8, 0.1, 0.1, 0.1)          # Nz not a multiple of 64
    with pytest.raises(fd.FdetdError):
        fd.fdetd_plan_modes(64, 32, [0], 7, 0.1, 0.1, 0.1)           # odd order
    with pytest.raises(fd.FdetdError):
        fd.fdetd_plan_modes(64, 3, [0], 8, 0.1, 0.1, 0.1)            # Nr too small
    plan = fd.fdetd_plan_modes(64, 32, [0], 8, 0.1, 0.1, 0.1, precision="fp32")
    with pytest.raises(fd.FdetdError):
        fd.fdetd_step(plan, torch.zeros((1, 6, 64, 32), dtype=torch.complex128, device="cuda"))  # wrong dtype
    with pytest.raises(fd.FdetdError):
        fd.fdetd_step(plan, torch.zeros((1, 6, 64, 31), dtype=torch.complex64, device="cuda"))   # wrong shape


def test_host_entry_point_matches_device():
    rng = np.random.default_rng(3)
    Nz, Nr, modes = 64, 24, [0, 1]
    F = zero_axis(rng.standard_normal((2, 6, Nz, Nr)) + 1j * rng.standard_normal((2, 6, Nz, Nr)))
    J = rng.standard_normal((2, 3, Nz, Nr)) + 0j
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, 8, 1 / 16, 1 / 4, 1 / 16, precision="fp64")
    dev = torch.from_numpy(F).cuda()
    fd.fdetd_step(plan, dev, torch.from_numpy(J).cuda(), 3)
    host = torch.from_numpy(F.copy()).pin_memory()
    fd.fdetd_step_host(plan, host, torch.from_numpy(J).pin_memory(), 3)
    assert np.abs(host.numpy() - dev.cpu().numpy()).max() < 1e-14


# The 2048 x 256 current-driven workload after 2 steps, on sampled kz columns.  Columns where a mode has
# content (the pulse band around the carrier kz = 2 pi, q = Nz dz = 128, and the low-kz band of the smooth
# current) are compared per field, relative to the field's norm in those columns (floor 1e-12).  Mode 0
# starts at zero and is driven by the current alone, so its B_r and B_theta carry about 1% of its state;
# their true relative error is bounded separately (measured levels x 3).  Columns far outside both bands hold
# only rounding-level values: there the error is checked against the state's RMS column norm (an absolute,
# state-scale bound, reported as such).
TOL_WEAK_2048 = {"fp64": 1e-10, "fp32": 6e-5, "bf16x6": 3e-5, "bf16x3": 1e-3}


@pytest.mark.parametrize("prec", ALL)
def test_full_size_2048x256_sampled_kz(prec):
    w = inputs.workload("lwfa_m01_2048x256")
    F, J = inputs.workload_inputs(w)
    nsteps = 2
    got = _run(prec, F, J, w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, nsteps)
    rng = np.random.default_rng(4)
    qs = [0, 1, 20, 120, 128, 136, w.Nz // 2, int(rng.integers(400, 900))]
    for i, m in enumerate(w.modes):
        ref = mx.step_spectral(F[i], J[i], w.Nz, w.Nr, m, w.order, w.dz, w.dr, w.dt, nsteps=nsteps,
                               kz_subset=qs, method="eig")
        Gq = kz_columns(got[i], qs)                           # [6][nq][Nr]
        col_rms = np.linalg.norm(got[i])   # Parseval: the RMS norm of a kz column equals the real-space norm
        norms = np.array([np.linalg.norm(mx.gather(ref[q])) for q in qs])
        inb = [k for k in range(len(qs)) if norms[k] >= 1e-2 * norms.max()]
        rows = column_report([Gq[:, k, :] for k in inb], [ref[qs[k]] for k in inb])
        print("\n" + format_report(rows, f"{prec} m={m} columns {[qs[k] for k in inb]}"))
        # two steps, with a factor 2 of margin over the per-step tolerance (the FP64 path agrees to ~1e-12
        # per step on the pulse band of this 256-point radial basis)
        check_report(rows, TOL[prec] * nsteps * 2, TOL_WEAK_2048[prec], label=f"{prec} m={m}")
        for k in range(len(qs)):
            if k in inb:
                continue
            e = np.linalg.norm(mx.gather(Gq[:, k, :]) - mx.gather(ref[qs[k]])) / col_rms
            print(f"{prec} m={m} q={qs[k]} (outside the bands): error / RMS column norm = {e:.2e}")
            assert e < TOL[prec] * nsteps * 2, (m, qs[k], e)


@pytest.mark.parametrize("prec", ALL)
def test_full_size_invariants(prec):
    # div B is conserved exactly by the discrete operator; div E changes by -n dt div J
    w = inputs.workload("lwfa_m01_2048x256")
    F, J = inputs.workload_inputs(w)
    nsteps = 4
    got = _run(prec, F, J, w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, nsteps)
    for i, m in enumerate(w.modes):
        rad = mx.Radial(w.Nr, w.order, w.dr, m)
        F0 = mx.fill_axis(F[i], rad)
        dE0 = dg.div_E(F0, rad, w.order, w.dz)
        dJ = dg.div_J(J[i], rad, w.order, w.dz)
        dB0 = dg.div_B(F0, rad, w.order, w.dz)
        # A divergence is a difference stencil: rounding an O(|F|) field by a relative error e
        # perturbs it by up to e |F|_max times the stencil's absolute row sum (~2 sum|c_n| (1/dz + 2/dr)).
        from oracle.stencils import staggered_coeffs
        stencil = 2 * np.abs(staggered_coeffs(w.order)).sum() * (1 / w.dz + 2 / w.dr)
        fmax = np.abs(got[i]).max()
        tol = TOL[prec] * nsteps * stencil * fmax
        assert np.abs(dg.div_E(got[i], rad, w.order, w.dz) - (dE0 - nsteps * w.dt * dJ)).max() < tol
        assert np.abs(dg.div_B(got[i], rad, w.order, w.dz) - dB0).max() < tol


@pytest.mark.parametrize("prec", ALL)
@pytest.mark.parametrize("Nz", [192, 320, 448, 576])
def test_parity_non_power_of_two_nz(prec, Nz):
    # z lengths 64 k with odd factors 3, 5, 7, 9: the mixed-radix transform (radix 3, 5, 7 stages before the
    # power-of-two ones), full field against the oracle after 2 steps, current on, modes 0 and 2
    rng = np.random.default_rng(Nz)
    Nr, modes, order, dz, dr, dt = 40, [0, 2], 8, 1 / 16, 1 / 4, 1 / 16
    F = zero_axis(rng.standard_normal((2, 6, Nz, Nr)) + 1j * rng.standard_normal((2, 6, Nz, Nr)))
    J = 0.3 * (rng.standard_normal((2, 3, Nz, Nr)) + 1j * rng.standard_normal((2, 3, Nz, Nr)))
    nsteps = 2
    got = _run(prec, F, J, Nz, Nr, modes, order, dz, dr, dt, nsteps)
    ref = _oracle(F, J, Nz, Nr, modes, order, dz, dr, dt, nsteps)
    for i, m in enumerate(modes):
        rows = field_report(got[i], ref[i], nd=order // 2)
        print("\n" + format_report(rows, f"{prec} Nz={Nz} m={m}"))
        check_report(rows, TOL[prec] * nsteps, TOL_WEAK[prec] * nsteps, label=f"{prec} Nz={Nz} m={m}")


def test_unsupported_z_lengths_are_refused():
    for Nz in (100, 64 * 11, 4093):
        with pytest.raises(fd.FdetdError):
            fd.fdetd_plan_modes(Nz, 32, [0], 8, 0.1, 0.1, 0.1, precision="fp32")
