"""Error of the FP32-state precisions against the FP64 oracle after 1, 100 and 1000 steps on the 8192 x 512
three-mode current-driven workload (the full-size precision sweep), on sampled kz columns inside and outside
the pulse band.  The oracle's columns are precomputed by tests/golden/make_sweep_8192x512.py (a dense 3069^2
exponential per column takes minutes) and read from tests/golden/sweep_8192x512_ref.npz.  FP64 is absent: its
single-pass z transform stops at Nz = 4096.

Opt-in (several minutes of device and host time): FDETD_FULL_SWEEP=1 pytest -m gpu -s tests/test_gpu_sweep_8192x512.py
The bounds are ten times the measured 2048 x 256 levels until this size has been measured.
"""
import os

import numpy as np
import pytest

from oracle import maxwell as mx
from paper_2605_12132_gb300 import inputs

pytestmark = pytest.mark.gpu

if os.environ.get("FDETD_FULL_SWEEP") != "1":
    pytest.skip("full-size sweep is opt-in (FDETD_FULL_SWEEP=1)", allow_module_level=True)
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

REF = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_8192x512_ref.npz")
BOUND = {"fp32": [1e-5, 1.5e-4, 2e-3], "bf16x6": [1e-5, 2.5e-3, 2.5e-2], "bf16x3": [3e-4, 1.2e-2, 1.2e-1]}
W = inputs.workload("sweep_m012_8192x512")


@pytest.fixture(scope="module")
def case():
    d = np.load(REF)
    F, J = inputs.workload_inputs(W)
    return F, J, d["ref"], list(d["counts"]), list(d["qs"])


def _errors(G, ref, qs):
    """per-field error on the sampled columns, fields under 10% of the state measured against 10% of it"""
    Gh = np.fft.fft(G, axis=1)
    err = np.zeros(6)
    tot = np.sqrt(sum(np.linalg.norm(ref[k]) ** 2 for k in range(len(qs))))
    for f in range(6):
        num = np.sqrt(sum(np.linalg.norm(mx.gather_field(Gh[:, q, :], f) - mx.gather_field(ref[k], f)) ** 2
                          for k, q in enumerate(qs)))
        den = np.sqrt(sum(np.linalg.norm(mx.gather_field(ref[k], f)) ** 2 for k in range(len(qs))))
        err[f] = num / max(den, 0.1 * tot)
    return err


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6", "fp32"])
def test_sweep_8192x512(prec, case):
    F, J, ref, counts, qs = case
    plan = fd.fdetd_plan_modes(W.Nz, W.Nr, W.modes, W.order, W.dz, W.dr, W.dt, precision=prec)
    f = torch.from_numpy(F).to(plan.complex_dtype).cuda()
    j = torch.from_numpy(J).to(plan.complex_dtype).cuda()
    done = 0
    rows = []
    for ci, n in enumerate(counts):
        fd.fdetd_step(plan, f, j, int(n) - done)
        done = int(n)
        plan.status()
        G = f.cpu().numpy()
        for i, m in enumerate(W.modes):
            e = _errors(G[i].astype(np.complex128), ref[ci, i], qs)
            rows.append((n, m, e))
    print(f"\n{prec}: steps, mode, per-field error (Er, Et, Ez, Br, Bt, Bz)")
    for n, m, e in rows:
        print(f"  {prec} {n:5d} m={m} " + " ".join(f"{x:.2e}" for x in e))
    for ci, n in enumerate(counts):
        worst = max(e.max() for nn, _, e in rows if nn == n)
        assert worst < BOUND[prec][ci], (prec, n, worst)
