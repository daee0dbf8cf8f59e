"""Destagger to the primary grids on the GPU against the oracle (Sec. 3, Eqs. shapesAM_destagger_*)."""
import numpy as np
import pytest

from oracle import destagger as ds
from paper_2605_12132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

TOL = {"fp64": 1e-13, "fp32": 1e-6, "bf16x3": 1e-6}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [4, 8, 16])
def test_destagger_matches_oracle(prec, order):
    rng = np.random.default_rng(order)
    Nz, Nr, modes = 64, 37, [0, 1, 2, 3]
    F = rng.standard_normal((4, 6, Nz, Nr)) + 1j * rng.standard_normal((4, 6, Nz, Nr))
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, order, 1 / 16, 1 / 4, 1 / 16, precision=prec)
    f = torch.from_numpy(F).to(plan.complex_dtype).cuda()
    got = fd.fdetd_destagger(plan, f).cpu().numpy().astype(np.complex128)
    Fin = f.cpu().numpy().astype(np.complex128)
    for i, m in enumerate(modes):
        ref = ds.destagger(Fin[i], m, order)
        err = np.abs(got[i] - ref).max() / np.abs(ref).max()
        assert err < TOL[prec], (m, err)


def test_destagger_after_a_step_uses_the_axis_values():
    # the step writes the axis slots; the destaggered pulse matches the oracle on the same state
    w = inputs.workload("vacuum_m1_256x64")
    F, _ = inputs.workload_inputs(w)
    plan = fd.fdetd_plan_modes(w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, precision="bf16x3")
    f = torch.from_numpy(F).to(torch.complex64).cuda()
    fd.fdetd_step(plan, f, None, 3)
    out = fd.fdetd_destagger(plan, f)
    state = f.cpu().numpy().astype(np.complex128)
    ref = ds.destagger(state[0], 1, w.order)
    err = np.abs(out.cpu().numpy()[0] - ref).max() / np.abs(ref).max()
    assert err < TOL["bf16x3"], err


def test_destagger_rejects_aliasing():
    plan = fd.fdetd_plan(64, 16, 0, 4, 1 / 16, 1 / 4, 1 / 16, precision="fp32")
    f = torch.zeros((1, 6, 64, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(fd.FdetdError):
        fd.fdetd_destagger(plan, f, f)
