"""The column-split form of the z transform (three launches, one column in shared memory at a time): the form
FP64 takes where the three field columns of a family do not fit in shared memory (Nz = 8192).  Forced at small
Nz it must give bitwise the single-pass (fused) form's FP64 result; on the tensor-core paths it feeds the
back-projection's split pieces; at Nz = 8192 in FP64 it is checked against the oracle's per-kz evaluator."""
import numpy as np
import pytest

from oracle import maxwell as mx
from tests.gpu_util import check_report, column_report, field_report, format_report, kz_columns, zero_axis

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402
from paper_2605_12132_gb300 import _native as nat  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-6, "bf16x6": 1e-6, "bf16x3": 2.5e-5}
TOL_WEAK = {"fp64": 1e-12, "fp32": 3e-6, "bf16x6": 3e-6, "bf16x3": 3e-4}


def _case(Nz, Nr, nm, seed, with_J=True):
    rng = np.random.default_rng(seed)
    F = zero_axis(rng.standard_normal((nm, 6, Nz, Nr)) + 1j * rng.standard_normal((nm, 6, Nz, Nr)))
    J = 0.3 * (rng.standard_normal((nm, 3, Nz, Nr)) + 1j * rng.standard_normal((nm, 3, Nz, Nr))) if with_J else None
    return F, J


def _step(plan, F, J, nsteps):
    cdt = plan.complex_dtype
    f = torch.from_numpy(F).to(cdt).cuda()
    j = torch.from_numpy(J).to(cdt).cuda() if J is not None else None
    fd.fdetd_step(plan, f, j, nsteps)
    plan.status()
    return f


@pytest.mark.parametrize("with_J", [True, False])
def test_column_form_is_bitwise_the_fused_form_fp64(with_J):
    Nz, Nr, modes = 256, 40, [0, 1, 3]
    F, J = _case(Nz, Nr, len(modes), 17, with_J)
    a = fd.fdetd_plan_modes(Nz, Nr, modes, 8, 1 / 16, 1 / 4, 1 / 16, precision="fp64")
    b = fd.fdetd_plan_modes(Nz, Nr, modes, 8, 1 / 16, 1 / 4, 1 / 16, precision="fp64", flags=nat.SPECTRAL_COLUMNS)
    assert b.launches_per_step == a.launches_per_step + 2
    assert torch.equal(_step(a, F, J, 3), _step(b, F, J, 3))


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6"])
def test_column_form_matches_oracle(prec):
    Nz, Nr, modes, order, dz, dr, dt = 512, 40, [0, 2], 8, 1 / 16, 1 / 4, 1 / 16
    F, J = _case(Nz, Nr, len(modes), 23)
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, order, dz, dr, dt, precision=prec, flags=nat.SPECTRAL_COLUMNS)
    got = _step(plan, F, J, 2).cpu().numpy().astype(np.complex128)
    for i, m in enumerate(modes):
        ref = mx.step_spectral(F[i], J[i], Nz, Nr, m, order, dz, dr, dt, nsteps=2)
        rows = field_report(got[i], ref, nd=order // 2)
        print("\n" + format_report(rows, f"columns {prec} m={m}"))
        check_report(rows, TOL[prec] * 2, TOL_WEAK[prec] * 2, label=f"columns {prec} m={m}")


def test_fp64_at_8192_sampled_kz():
    # the FP64 row at the sweep's z length: one step of modes 0 and 1, current on, against the oracle's per-kz
    # dense evaluator on sampled columns (white-noise fields: every kz column carries energy)
    Nz, Nr, modes, order, dz, dr, dt = 8192, 24, [0, 1], 16, 1 / 16, 1 / 4, 1 / 16
    F, J = _case(Nz, Nr, len(modes), 29)
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, order, dz, dr, dt, precision="fp64")
    assert plan.launches_per_step == 5          # projection, three column-split launches, back-projection
    got = _step(plan, F, J, 1).cpu().numpy()
    qs = [0, 1, 777, 2048, 4095, 4096, 6000, 8191]
    for i, m in enumerate(modes):
        ref = mx.step_spectral(F[i], J[i], Nz, Nr, m, order, dz, dr, dt, nsteps=1, kz_subset=qs, method="eig")
        Gq = kz_columns(got[i], qs)
        rows = column_report([Gq[:, k, :] for k in range(len(qs))], [ref[q] for q in qs])
        print("\n" + format_report(rows, f"fp64 Nz=8192 m={m} columns {qs}"))
        check_report(rows, 2 * TOL["fp64"], 2 * TOL_WEAK["fp64"], label=f"fp64 8192 m={m}")
