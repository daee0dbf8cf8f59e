"""Batches of uneven instances under one captured CUDA graph: each instance's result equals
the same plan stepped alone (bitwise: same kernels, same inputs, private scratch)."""
import numpy as np
import pytest

from paper_2605_12132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402


def _instances(seed, count, prec):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        Nz = int(rng.choice([64, 128, 256, 512]))
        Nr = int(rng.integers(12, 80)) * 2
        M = int(rng.integers(1, 4))
        order = int(rng.choice([8, 16]))
        waist = float(rng.uniform(10, 40)) * 0.25
        F = np.zeros((M + 1, 6, Nz, Nr), complex)
        F[1] = inputs.pulse_fields(Nz, Nr, 1 / 16, 1 / 4, waist, 2.0)
        for f in (0, 4, 5):
            F[:, f, :, 0] = 0
        J = np.stack([inputs.random_current(Nz, Nr, m, 4.0, 1e-2, seed + k) for m in range(M + 1)])
        plan = fd.fdetd_plan(Nz, Nr, M, order, 1 / 16, 1 / 4, 1 / 16, precision=prec)
        out.append((plan, F, J))
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_batch_graph_matches_individual_steps(prec):
    inst = _instances(7, 6, prec)
    nsteps = 3
    batch = fd.FdetdBatch()
    tensors = []
    for plan, F, J in inst:
        f = torch.from_numpy(F).to(torch.complex64).cuda()
        j = torch.from_numpy(J).to(torch.complex64).cuda()
        tensors.append((f, j))
        batch.add(plan, f, j)
    batch.capture(1)
    for _ in range(nsteps):
        batch.launch()
    torch.cuda.synchronize()
    for (plan, F, J), (f, j) in zip(inst, tensors):
        ref = torch.from_numpy(F).to(torch.complex64).cuda()
        fd.fdetd_step(plan, ref, torch.from_numpy(J).to(torch.complex64).cuda(), nsteps)
        plan.status()
        torch.cuda.synchronize()
        assert torch.equal(ref, f)


def test_batch_rejects_duplicate_plan():
    plan = fd.fdetd_plan(64, 16, 0, 4, 0.1, 0.1, 0.1, precision="fp32")
    f = torch.zeros((1, 6, 64, 16), dtype=torch.complex64, device="cuda")
    batch = fd.FdetdBatch()
    batch.add(plan, f)
    with pytest.raises(fd.FdetdError):
        batch.add(plan, f)
