"""The library's continuous-batching server on the GPU: requests of different sizes and precisions admitted
under an HBM budget, the resident field requests advanced together as one batch (grouped launches under a
CUDA graph, re-captured as requests join and leave), envelope requests alongside.  Each result equals the
same request run alone (bitwise: the batch runs the same kernels on the same data), the served field results
match the FP64 oracle on sampled kz columns, and the server's device-footprint estimate covers what the
plans and resident state actually hold."""
import numpy as np
import pytest

from oracle import maxwell as mx
from paper_2605_12132_gb300 import inputs
from tests.gpu_util import check_report, column_report, format_report, kz_columns

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402
from paper_2605_12132_gb300 import serve  # noqa: E402

# per-step tolerance of the strong fields and the weak-field bound, relative L2 per field
TOL = {"bf16x3": (3e-5, 1e-3), "bf16x6": (3e-6, 1e-4), "fp32": (1e-6, 1e-4), "fp64": (1e-12, 1e-10)}


def _requests():
    reqs = []
    for k, (Nz, Nr, M, prec, steps) in enumerate([(256, 64, 1, "bf16x3", 20), (128, 96, 2, "fp32", 13),
                                                   (512, 40, 1, "bf16x6", 9), (64, 32, 0, "fp64", 7),
                                                   (256, 128, 2, "bf16x6", 6)]):
        F = np.zeros((M + 1, 6, Nz, Nr), complex)
        F[min(1, M)] = inputs.pulse_fields(Nz, Nr, 1 / 16, 1 / 4, 2.5, 2.0)
        for f in (0, 4, 5):
            F[:, f, :, 0] = 0
        J = np.stack([inputs.random_current(Nz, Nr, m, 4.0, 1e-2, 50 + k) for m in range(M + 1)])
        reqs.append(serve.FieldRequest(Nz, Nr, list(range(M + 1)), 8, 1 / 16, 1 / 4, 1 / 16, steps, F, J, prec))
    w = inputs.EnvelopeWorkload("small", 256, 64, 8, 4, 0.2, 0.25, 0.05, 11, a0=1.0, waist=4.0, tau=6.0,
                                chi0=0.04)
    a, at, chi = inputs.envelope_inputs(w)
    reqs.append(serve.EnvelopeRequest(w.Nz, w.Nr, w.order, w.taylor_order, w.dz, w.dr, w.dt, w.steps,
                                      np.stack([a, at]), chi))
    return reqs


def _alone(req):
    if req.kind == "envelope":
        plan = fd.envelope_plan(req.Nz, req.Nr, req.order, req.taylor_order, req.dz, req.dr, req.dt, req.k0)
        st = torch.from_numpy(req.a).to(torch.complex64).cuda()
        fd.envelope_step(plan, st, torch.from_numpy(req.chi.astype(np.float32)).cuda(), req.steps)
    else:
        plan = fd.fdetd_plan_modes(req.Nz, req.Nr, req.modes, req.order, req.dz, req.dr, req.dt,
                                   precision=req.precision)
        st = torch.from_numpy(req.F).to(plan.complex_dtype).cuda()
        fd.fdetd_step(plan, st, torch.from_numpy(req.J).to(plan.complex_dtype).cuda(), req.steps)
    torch.cuda.synchronize()
    return st.cpu().numpy()


def test_mix_equals_alone_and_oracle_under_budget():
    reqs = _requests()
    alone = [_alone(r) for r in reqs]
    need = [serve.estimate_bytes(r) for r in reqs]
    budget = int(max(need) * 1.6)          # forces queueing: not everything fits at once
    srv = serve.Server(budget, chunk_steps=4)
    tickets = [srv.submit(r) for r in reqs]
    for t in tickets:
        t.wait(300)
    st = srv.stats()
    assert st["peak_bytes"] <= budget and st["used_bytes"] == 0 and st["completed"] == len(reqs)
    assert st["recaptures"] >= 2           # the batch changed membership while requests were served
    for t, ref in zip(tickets, alone):
        assert t.state == serve.DONE and t.latency >= 0
        assert np.array_equal(t.result, ref), t.id
    srv.close()
    # the served field results against the oracle (kz = 0, the carrier, one outside the band)
    for t in tickets:
        r = t.request
        if r.kind != "field":
            continue
        qs = [0, r.Nz // 16, r.Nz // 3]
        G = kz_columns(t.result.astype(np.complex128), qs)
        for i, m in enumerate(r.modes):
            ref = mx.step_spectral(r.F[i], r.J[i], r.Nz, r.Nr, m, r.order, r.dz, r.dr, r.dt, nsteps=r.steps,
                                   kz_subset=qs, method="expm")
            rows = column_report([G[i][:, k, :] for k in range(len(qs))], [ref[q] for q in qs])
            label = f"served {r.precision} {r.Nz}x{r.Nr} m={m} after {r.steps}"
            print("\n" + format_report(rows, label))
            tol, weak = TOL[r.precision]
            check_report(rows, tol * r.steps, weak * r.steps, label=label)


def test_request_larger_than_budget_is_rejected():
    reqs = _requests()
    srv = serve.Server(1024)
    with pytest.raises(fd.FdetdError):
        srv.submit(reqs[0])
    srv.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "bf16x6"])
def test_footprint_estimate_covers_plan_and_state(prec):
    for Nz, Nr, M in [(256, 64, 1), (512, 200, 2), (8192, 48, 1)]:
        if prec == "fp64" and Nz > 4096:
            continue
        F = np.zeros((M + 1, 6, Nz, Nr), complex)
        J = np.zeros((M + 1, 3, Nz, Nr), complex)
        req = serve.FieldRequest(Nz, Nr, list(range(M + 1)), 8, 1 / 16, 1 / 4, 1 / 16, 5, F, J, prec)
        plan = fd.fdetd_plan(Nz, Nr, M, 8, 1 / 16, 1 / 4, 1 / 16, precision=prec)
        elt = 16 if prec == "fp64" else 8
        state = (M + 1) * 9 * Nz * Nr * elt
        assert serve.estimate_bytes(req) >= plan.device_bytes + state, (prec, Nz, Nr, M)
        plan.close()
    ew = inputs.envelope_workload("envelope_4096x256")
    a, at, chi = inputs.envelope_inputs(ew)
    req = serve.EnvelopeRequest(ew.Nz, ew.Nr, ew.order, ew.taylor_order, ew.dz, ew.dr, ew.dt, 10,
                                np.stack([a, at]), chi)
    plan = fd.envelope_plan(ew.Nz, ew.Nr, ew.order, ew.taylor_order, ew.dz, ew.dr, ew.dt)
    assert serve.estimate_bytes(req) >= plan.device_bytes + ew.Nz * ew.Nr * (16 + 4)
    plan.close()
