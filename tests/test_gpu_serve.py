"""Continuous-batching server: requests admitted under an HBM budget, interleaved on the device,
each result identical (bitwise) to the same request run alone."""
import numpy as np
import pytest

from paper_2605_12132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402
from paper_2605_12132_gb300 import serve  # noqa: E402


def _requests():
    rng = np.random.default_rng(11)
    reqs = []
    for k, (Nz, Nr, M, prec, steps) in enumerate([(256, 64, 1, "bf16x3", 20), (128, 96, 2, "fp32", 13),
                                                   (512, 40, 1, "bf16x6", 9), (64, 32, 0, "fp64", 7)]):
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


def test_mix_equals_alone_under_budget():
    reqs = _requests()
    alone = [_alone(r) for r in reqs]
    need = [serve.estimate_bytes(r) for r in reqs]
    budget = int(max(need) * 1.6)          # forces queueing: not everything fits at once
    srv = serve.Server(budget, chunk_steps=4)
    tickets = [srv.submit(r) for r in reqs]
    srv.drain(timeout=300)
    srv.close()
    assert srv.peak_used <= budget and srv.used == 0
    for t, ref in zip(tickets, alone):
        assert t.completed is not None and t.latency >= 0
        assert np.array_equal(t.result, ref), t.id
    stats = serve.latency_stats(tickets)
    assert stats["count"] == len(reqs) and stats["p99_s"] >= stats["p50_s"]


def test_request_larger_than_budget_is_rejected():
    reqs = _requests()
    srv = serve.Server(1024)
    with pytest.raises(fd.FdetdError):
        srv.submit(reqs[0])
    srv.close()
