"""Error of the FP32-state precisions against the FP64 oracle after 1, 100 and 1000 steps on the 8192 x 512
three-mode current-driven workload (the full-size precision sweep), on sampled kz columns inside and outside
the pulse band.  The oracle's columns are precomputed by tests/golden/make_sweep_8192x512.py (a dense 3069^2
exponential per column takes minutes) and read from tests/golden/sweep_8192x512_ref.npz.  FP64 is absent here:
it runs at Nz = 8192 through the column-split z transform, checked against the oracle in
tests/test_gpu_spectral_columns.py on a narrower radial grid, but its 1000 steps at Nr = 512 would take about ten
GPU-minutes per run.

Per mode and field: relative L2 with a floor of 1e-12 of the state's norm, and the element-wise error.  Fields
carrying at least 10% of the state are checked against the strong bound, the others (the radial and
azimuthal magnetic fields of mode 0, which the current alone drives, and E_z, B_z of the pulse mode) against
the weak bound.  Bounds are the measured levels (GB300) x 2-3; the table is printed (pytest -s).
"""
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

REF = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_8192x512_ref.npz")
# (strong, weak) per step count 1, 100, 1000
BOUND = {"fp32": [(1e-6, 6e-5), (1.5e-5, 3e-5), (1.5e-4, 1.5e-4)],
         "bf16x6": [(3e-6, 3e-5), (5e-4, 5e-4), (4e-3, 4e-3)],
         "bf16x3": [(3e-5, 1e-3), (1.5e-3, 1.5e-3), (1.2e-2, 1.2e-2)]}
W = inputs.workload("sweep_m012_8192x512")


@pytest.fixture(scope="module")
def case():
    d = np.load(REF)
    F, J = inputs.workload_inputs(W)
    return F, J, d["ref"], list(d["counts"]), list(d["qs"])


@pytest.mark.parametrize("prec", ["bf16x6", "fp32", "bf16x3"])
def test_sweep_8192x512(prec, case):
    F, J, ref, counts, qs = case
    plan = fd.fdetd_plan_modes(W.Nz, W.Nr, W.modes, W.order, W.dz, W.dr, W.dt, precision=prec)
    f = torch.from_numpy(F).to(plan.complex_dtype).cuda()
    j = torch.from_numpy(J).to(plan.complex_dtype).cuda()
    done = 0
    failures = []
    for ci, n in enumerate(counts):
        fd.fdetd_step(plan, f, j, int(n) - done)
        done = int(n)
        plan.status()
        G = kz_columns(f.cpu().numpy().astype(np.complex128), qs)      # [modes][6][nq][Nr]
        for i, m in enumerate(W.modes):
            rows = column_report([G[i][:, k, :] for k in range(len(qs))], list(ref[ci, i]))
            label = f"{prec} {int(n):5d} steps m={m}"
            print("\n" + format_report(rows, label))
            try:
                check_report(rows, *BOUND[prec][ci], label=label)
            except AssertionError as e:
                failures.append(str(e))
    assert not failures, "\n".join(failures)
