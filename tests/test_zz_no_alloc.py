"""The allocation-free envelope entry point against the plan-based one (GPU).

envelope_step_static exists for callers that cannot allocate device memory (pre-reserved memory
pools, host frameworks that own every allocation, loops that cannot afford an allocation's
synchronisation); its scratch is a fixed file-scope device array.  This file is collected last so that a failure here leaves every other
test already run; it passes both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.mark.parametrize("NT", [1, 4])
def test_static_entry_matches_plan_entry_twice(NT):
    rng = np.random.default_rng(31 + NT)
    Nz, Nr, order, dz, dr, dt = 128, 48, 8, 0.2, 0.25, 0.05
    a = rng.standard_normal((2, Nz, Nr)) + 1j * rng.standard_normal((2, Nz, Nr))
    chi = 0.5 * rng.random((Nz, Nr))
    c = torch.from_numpy(chi).float().cuda()
    ref = torch.from_numpy(a).to(torch.complex64).cuda()
    got = ref.clone()
    plan = fd.envelope_plan(Nz, Nr, order, NT, dz, dr, dt)
    for call in range(2):  # two calls in a row share the static scratch
        fd.envelope_step(plan, ref, c, 2)
        fd.envelope_step_static(got, c, order, NT, dz, dr, dt, nsteps=2)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        # same tolerance as the envelope parity tests (FP32 arithmetic, different summation order)
        assert _rel(g[0], r[0]) < 2e-6 and _rel(g[1], r[1]) < 2e-6, (call, _rel(g[0], r[0]), _rel(g[1], r[1]))


def test_static_entry_rejects_oversized_grid():
    a = torch.zeros((2, 4096, 512), dtype=torch.complex64, device="cuda")  # 2^21 cells > 2^20
    c = torch.zeros((4096, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(fd.FdetdError):
        fd.envelope_step_static(a, c, 8, 4, 0.2, 0.25, 0.05)
