"""The bounded-wait timeout path of the tensor-core pipelines, driven without breaking anything: a plan's wait
limit set to 0 makes every mbarrier wait of its next step's kernels give up at once on a healthy pipeline.
The kernels must then stop, drain what they issued, release their tensor memory and return; the plan reports
FDETD_ERR_TIMEOUT; and the same plan and device context keep working: with the default limit restored, a step
gives bitwise the result of a fresh plan."""
import numpy as np
import pytest

from tests.gpu_util import zero_axis

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

FDETD_ERR_TIMEOUT = 6


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_expired_waits_report_timeout_and_the_context_stays_usable(prec):
    rng = np.random.default_rng(8)
    Nz, Nr, modes = 256, 64, [0, 1]
    F = zero_axis(rng.standard_normal((2, 6, Nz, Nr)) + 1j * rng.standard_normal((2, 6, Nz, Nr)))
    J = 0.1 * (rng.standard_normal((2, 3, Nz, Nr)) + 1j * rng.standard_normal((2, 3, Nz, Nr)))
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, 8, 1 / 16, 1 / 4, 1 / 16, precision=prec)
    j = torch.from_numpy(J).to(torch.complex64).cuda()
    f = torch.from_numpy(F).to(torch.complex64).cuda()
    fd.fdetd_step(plan, f, j, 1)                  # a healthy step first (builds the plan's launch tables)
    plan.status()
    plan.set_wait_limit(0)
    f = torch.from_numpy(F).to(torch.complex64).cuda()
    fd.fdetd_step(plan, f, j, 1)
    with pytest.raises(fd.FdetdError) as info:
        plan.status()
    assert info.value.code == FDETD_ERR_TIMEOUT
    # the status call cleared the record; the default limit restores normal operation
    plan.set_wait_limit(-1)
    f = torch.from_numpy(F).to(torch.complex64).cuda()
    fd.fdetd_step(plan, f, j, 2)
    plan.status()
    fresh = fd.fdetd_plan_modes(Nz, Nr, modes, 8, 1 / 16, 1 / 4, 1 / 16, precision=prec)
    g = torch.from_numpy(F).to(torch.complex64).cuda()
    fd.fdetd_step(fresh, g, j, 2)
    fresh.status()
    assert torch.equal(f, g)


def test_wait_limit_is_refused_on_cuda_core_plans():
    plan = fd.fdetd_plan(64, 16, 0, 4, 1 / 16, 1 / 4, 1 / 16, precision="fp32")
    with pytest.raises(fd.FdetdError):
        plan.set_wait_limit(0)
