"""Batches of uneven instances under one captured CUDA graph.

* Each instance's result equals the same plan stepped alone (bitwise: same kernels, same inputs,
  private scratch).
* Instances at the sizes of the uneven mix (the largest radial size with the most modes and order 16, a
  mid-size order-8 case, the longest z) advanced inside one batch match the FP64 oracle on sampled kz
  columns after 1 and 100 steps.  The oracle's columns are precomputed by
  tests/golden/make_batch_instances.py (a dense (6 Nr - 3)^2 exponential per column) into
  tests/golden/batch_instances_ref.npz."""
import os

import numpy as np
import pytest

from paper_2605_12132_gb300 import inputs
from tests.gpu_util import check_report, column_report, format_report, kz_columns

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


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6"])
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


REF = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_instances_ref.npz")
# per-step tolerance of fields with >= 10% of the state (relative L2, floor 1e-12 of the state) and measured
# bounds of the weak fields (the azimuthal and axial fields of the modes driven by the current alone)
TOL_BATCH = {"fp32": (1e-6, 1e-4), "bf16x6": (3e-6, 1e-4), "bf16x3": (3e-5, 3e-3)}


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "fp32"])
def test_batch_instances_match_oracle(prec):
    d = np.load(REF)
    counts = list(d["counts"])
    cfgs = list(inputs.PARITY_INSTANCES)
    batch = fd.FdetdBatch()
    keep = []
    for c in cfgs:
        F, J = inputs.instance_inputs(c)
        plan = fd.fdetd_plan(c["Nz"], c["Nr"], c["M"], c["order"], 1 / 16, 1 / 4, 1 / 16, precision=prec)
        f = torch.from_numpy(F).to(torch.complex64).cuda()
        j = torch.from_numpy(J).to(torch.complex64).cuda()
        batch.add(plan, f, j)
        keep.append((plan, f, j))
    batch.capture(1)
    done = 0
    for ci, n in enumerate(counts):
        for _ in range(int(n) - done):
            batch.launch()
        done = int(n)
        torch.cuda.synchronize()
        for k, (c, (plan, f, _)) in enumerate(zip(cfgs, keep)):
            plan.status()
            qs = list(d[f"qs{k}"])
            G = kz_columns(f.cpu().numpy().astype(np.complex128), qs)      # [M+1][6][nq][Nr]
            ref = d[f"ref{k}"][ci]                                          # [M+1][nq][6][Nr]
            for m in range(c["M"] + 1):
                rows = column_report([G[m][:, q, :] for q in range(len(qs))], list(ref[m]))
                label = f"{prec} Nz={c['Nz']} Nr={c['Nr']} order={c['order']} m={m} after {n}"
                print("\n" + format_report(rows, label))
                tol, weak = TOL_BATCH[prec]
                check_report(rows, tol * n, weak * n, label=label)


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_host_step_pipeline_parts_give_the_same_bits(prec):
    # the host-buffer step in its serial form and split into parts (copies overlapping compute) advances every
    # instance exactly as the device-resident graph does; a graph of two steps per launch is replayed as two
    # one-step part graphs
    inst = _instances(11, 5, prec)
    batch = fd.FdetdBatch()
    dev = []
    for plan, F, J in inst:
        f = torch.from_numpy(F).to(torch.complex64).cuda()
        j = torch.from_numpy(J).to(torch.complex64).cuda()
        dev.append((f, j))
        batch.add(plan, f, j)
    batch.capture(2)
    batch.launch()
    torch.cuda.synchronize()
    ref = [f.cpu().clone() for f, _ in dev]
    for parts in (1, 2, 3, 8):
        batch.set_host_pipeline(parts)
        hf = [torch.from_numpy(F).to(torch.complex64).pin_memory() for _, F, _ in inst]
        hj = [torch.from_numpy(J).to(torch.complex64).pin_memory() for _, _, J in inst]
        batch.step_host(hf, hj, 1)
        for k, (h, r) in enumerate(zip(hf, ref)):
            assert torch.equal(h, r), (parts, k)
    for plan, _, _ in inst:
        plan.status()
    batch.close()
