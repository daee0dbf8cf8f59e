"""The paper's Taylor-polynomial stepper on the GPU against the oracle's Taylor evaluator (same N, S).

Parity: the oracle's step_taylor with taylor_order = N and substeps = S computes exactly what the
kernels compute (Eq. maxwellAM_solution2 with T_N exponentials), in FP64; the GPU path is FP32.
Property: with more terms and substeps the Taylor step converges to the exact exponential step."""
import numpy as np
import pytest

from oracle import maxwell as mx
from paper_2605_12132_gb300 import inputs
from tests.gpu_util import check_report, field_report, format_report, zero_axis

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

# FP32 state and arithmetic: a few e-7 relative per stencil application, N applications per step
TOL_PER_STEP = 3e-6


def _run(F, J, Nz, Nr, modes, order, dz, dr, dt, N, S, nsteps):
    plan = fd.fdetd_taylor_plan(Nz, Nr, modes, order, dz, dr, dt, N, S)
    f = torch.from_numpy(F).to(torch.complex64).cuda()
    j = torch.from_numpy(J).to(torch.complex64).cuda() if J is not None else None
    fd.fdetd_taylor_step(plan, f, j, nsteps)
    torch.cuda.synchronize()
    return f.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("N,S", [(4, 1), (6, 2), (2, 3)])
def test_taylor_parity_small_ragged(N, S):
    rng = np.random.default_rng(10 + N + S)
    Nz, Nr, modes, order, dz, dr, dt = 64, 37, [0, 1, 2], 8, 1 / 16, 1 / 4, 1 / 64
    F = zero_axis(rng.standard_normal((3, 6, Nz, Nr)) + 1j * rng.standard_normal((3, 6, Nz, Nr)))
    J = 0.3 * (rng.standard_normal((3, 3, Nz, Nr)) + 1j * rng.standard_normal((3, 3, Nz, Nr)))
    nsteps = 3
    got = _run(F, J, Nz, Nr, modes, order, dz, dr, dt, N, S, nsteps)
    for i, m in enumerate(modes):
        ref = mx.step_taylor(F[i], J[i], Nz, Nr, m, order, dz, dr, dt, nsteps=nsteps, taylor_order=N, substeps=S)
        rows = field_report(got[i], ref, nd=order // 2)
        check_report(rows, TOL_PER_STEP * nsteps, TOL_PER_STEP * nsteps, label=f"N={N} S={S} m={m}")


def test_taylor_no_current_and_zero_steps():
    rng = np.random.default_rng(3)
    Nz, Nr = 64, 20
    F = zero_axis(rng.standard_normal((1, 6, Nz, Nr)) + 1j * rng.standard_normal((1, 6, Nz, Nr)))
    plan = fd.fdetd_taylor_plan(Nz, Nr, [1], 4, 1 / 16, 1 / 4, 1 / 64, 4, 1)
    f = torch.from_numpy(F).to(torch.complex64).cuda()
    f0 = f.clone()
    fd.fdetd_taylor_step(plan, f, None, 0)
    assert torch.equal(f, f0)
    fd.fdetd_taylor_step(plan, f, None, 2)
    torch.cuda.synchronize()
    ref = mx.step_taylor(F[0], None, Nz, Nr, 1, 4, 1 / 16, 1 / 4, 1 / 64, nsteps=2, taylor_order=4, substeps=1)
    rows = field_report(f.cpu().numpy()[0].astype(np.complex128), ref, nd=2)
    check_report(rows, TOL_PER_STEP * 2, TOL_PER_STEP * 2, label="no current")


def test_taylor_converges_to_the_exact_step():
    # vacuum pulse, m = 1: the Taylor truncation error of every field falls with the number of terms
    w = inputs.workload("vacuum_m1_256x64")
    F, _ = inputs.workload_inputs(w)
    exact = mx.step_spectral(F[0], None, w.Nz, w.Nr, 1, w.order, w.dz, w.dr, w.dt, nsteps=1)
    errs = []
    for N in (2, 4, 8):
        got = _run(F, None, w.Nz, w.Nr, [1], w.order, w.dz, w.dr, w.dt, N, 4, 1)
        rows = field_report(got[0], exact)
        print(format_report(rows, f"N={N}"))
        errs.append(np.array([r["l2"] for r in rows]))
    assert np.all(errs[0] > errs[1]) and np.all(errs[1] > errs[2]), errs
    # N = 8 with 4 substeps: the truncation is below the FP32 rounding of the strong fields; E_z and B_z
    # (0.8% of the state) carry the state-scale FP32 error
    assert errs[2].max() < 2e-5, errs


def test_taylor_argument_errors():
    with pytest.raises(fd.FdetdError):
        fd.fdetd_taylor_plan(64, 20, [0], 4, 1 / 16, 1 / 4, 1 / 64, 1, 1)     # N < 2
    with pytest.raises(fd.FdetdError):
        fd.fdetd_taylor_plan(64, 2, [0], 8, 1 / 16, 1 / 4, 1 / 64, 4, 1)      # Nr too small for the order
    with pytest.raises(fd.FdetdError):
        fd.fdetd_taylor_plan(64, 20, [0], 4, 1 / 16, 1 / 4, -1.0, 4, 1)       # dt <= 0
