"""Pipeline accounting of the tensor-core kernels: with profiling on, the projection and back-projection count
the clock cycles their roles wait on each kind of barrier.  Counting changes no result (bitwise equal steps with
and without it), every share lies in [0, 1], and the accounting covers both kernels, for one plan and for a
captured batch."""
import numpy as np
import pytest

from tests.gpu_util import zero_axis

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402
from paper_2605_12132_gb300 import _native as nat  # noqa: E402


def _inputs(Nz, Nr, nm, seed):
    rng = np.random.default_rng(seed)
    F = zero_axis(rng.standard_normal((nm, 6, Nz, Nr)) + 1j * rng.standard_normal((nm, 6, Nz, Nr)))
    J = 0.1 * (rng.standard_normal((nm, 3, Nz, Nr)) + 1j * rng.standard_normal((nm, 3, Nz, Nr)))
    return F, J


def _check_shares(rep):
    for kern in ("projection", "backprojection"):
        r = rep[kern]
        assert r["cycles"] > 0, kern
        for slot in nat.PIPELINE_SLOTS[1:]:
            if slot in r:
                assert 0.0 <= r[slot] <= 1.0 + 1e-9, (kern, slot, r[slot])
    assert rep["projection"]["converter_busy"] > 0 and rep["backprojection"]["epilogue_busy"] > 0
    if rep["spectral"]["cycles"]:
        assert abs(sum(rep["spectral"][k] for k in nat.SPECTRAL_PHASES[1:6]) - 1.0) < 1e-6


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_counting_changes_no_result_and_reports_shares(prec):
    Nz, Nr, modes = 512, 200, [0, 1, 2]
    F, J = _inputs(Nz, Nr, len(modes), 31)
    j = torch.from_numpy(J).to(torch.complex64).cuda()
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, 16, 1 / 16, 1 / 4, 1 / 16, precision=prec)
    a = torch.from_numpy(F).to(torch.complex64).cuda()
    fd.fdetd_step(plan, a, j, 3)
    plan.status()
    plan.set_profiling(True)
    b = torch.from_numpy(F).to(torch.complex64).cuda()
    fd.fdetd_step(plan, b, j, 3)
    rep = plan.pipeline_waits()
    plan.set_profiling(False)
    plan.status()
    assert torch.equal(a, b)
    _check_shares(rep)
    # off again: the counters stop (a further step leaves them where they were)
    before = plan.pipeline_waits()
    fd.fdetd_step(plan, b, j, 1)
    plan.status()
    assert plan.pipeline_waits() == before


def test_batch_counters_cover_the_grouped_kernels():
    shapes = [(512, 96, [0, 1]), (1024, 200, [0, 1, 2])]
    plans, dev = [], []
    for k, (Nz, Nr, modes) in enumerate(shapes):
        F, J = _inputs(Nz, Nr, len(modes), 40 + k)
        plans.append(fd.fdetd_plan_modes(Nz, Nr, modes, 8, 1 / 16, 1 / 4, 1 / 16, precision="bf16x6"))
        dev.append((torch.from_numpy(F).to(torch.complex64).cuda(), torch.from_numpy(J).to(torch.complex64).cuda()))
    batch = fd.FdetdBatch()
    for p, (f, j) in zip(plans, dev):
        batch.add(p, f, j)
    batch.set_profiling(True)
    batch.capture(1)
    for _ in range(2):
        batch.launch()
    torch.cuda.synchronize()
    for p in plans:
        p.status()
    _check_shares(batch.pipeline_waits())
    batch.close()
    for p in plans:
        p.close()


def test_cuda_core_plans_count_only_the_spectral_phases():
    Nz, Nr = 256, 48
    F, J = _inputs(Nz, Nr, 2, 5)
    plan = fd.fdetd_plan(Nz, Nr, 1, 8, 1 / 16, 1 / 4, 1 / 16, precision="fp32")
    f = torch.from_numpy(F).to(torch.complex64).cuda()
    j = torch.from_numpy(J).to(torch.complex64).cuda()
    plan.set_profiling(True)
    fd.fdetd_step(plan, f, j, 2)
    rep = plan.pipeline_waits()
    plan.set_profiling(False)
    plan.status()
    assert rep["projection"]["cycles"] == 0 and rep["backprojection"]["cycles"] == 0
    sp = rep["spectral"]
    assert sp["blocks"] == 2 * 2 * 2 * Nr          # steps x modes x families x j
    shares = [sp[k] for k in nat.SPECTRAL_PHASES[1:6]]
    assert all(0.0 <= x <= 1.0 for x in shares) and abs(sum(shares) - 1.0) < 1e-6
