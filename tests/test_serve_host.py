"""Host-side logic of the continuous-batching server (CPU only): the device work is replaced by a fake that
completes a chunk per scheduling round, so admission, ordering, memory accounting and the latency statistics
are checked without a GPU."""
import time

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2605_12132_gb300 import _native as nat  # noqa: E402
from paper_2605_12132_gb300 import serve  # noqa: E402


def _field(Nz=64, Nr=32, modes=(0, 1), steps=5, prec="bf16x3", with_J=True):
    F = np.zeros((len(modes), 6, Nz, Nr), complex)
    J = np.zeros((len(modes), 3, Nz, Nr), complex) if with_J else None
    return serve.FieldRequest(Nz, Nr, list(modes), 8, 0.1, 0.1, 0.1, steps, F, J, prec)


class FakeServer(serve.Server):
    """The scheduler with the device replaced: plans are dummies, a chunk completes at once."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.admission_order = []
        self.max_used = 0

    @staticmethod
    def _build_plan(req):
        return object()

    def _admit(self):
        before = {t.id for t in self.building}
        super()._admit()
        self.admission_order += [t.id for t in self.building if t.id not in before]
        self.max_used = max(self.max_used, self.used)
        assert self.used <= self.budget

    def _start_ready(self):
        still = []
        for t in self.building:
            if t._future.done():
                t._plan = t._future.result()
                self.active.append(t)
            else:
                still.append(t)
        self.building = still

    def _launch_chunks(self):
        still = []
        for t in self.active:
            t._done_steps += min(self.chunk, t.request.steps - t._done_steps)
            (self.finishing if t._done_steps >= t.request.steps else still).append(t)
        self.active = still

    def _reap(self):
        for t in self.finishing:
            t.completed = time.perf_counter()
            self.used -= t.bytes
            self.done.append(t)
        self.finishing = []


def test_estimate_bytes_grows_with_precision_current_and_size():
    b3, b6 = serve.estimate_bytes(_field(prec="bf16x3")), serve.estimate_bytes(_field(prec="bf16x6"))
    f32, f64 = serve.estimate_bytes(_field(prec="fp32")), serve.estimate_bytes(_field(prec="fp64"))
    assert b6 > b3 and f64 > f32
    noJ = serve.estimate_bytes(_field(with_J=False))
    assert b3 - noJ == 2 * 3 * 64 * 32 * 8          # the resident current: modes x 3 x Nz x Nr complex64
    assert serve.estimate_bytes(_field(Nz=128)) > b3


def test_first_come_first_served_within_the_budget():
    reqs = [_field(Nz=int(Nz), steps=int(s)) for Nz, s in zip([64, 256, 64, 128, 512, 64, 128, 256],
                                                                [5, 40, 3, 17, 9, 1, 33, 2])]
    sizes = [serve.estimate_bytes(r) for r in reqs]
    budget = max(sizes) + min(sizes)                 # the largest fits, but never next to a mid-sized one
    srv = FakeServer(budget, chunk_steps=4, plan_workers=2)
    tickets = [srv.submit(r, arrival=0.0) for r in reqs]
    srv.drain(timeout=60)
    srv.close()
    assert srv.admission_order == [t.id for t in tickets]          # no overtaking
    assert srv.used == 0 and len(srv.done) == len(reqs)
    assert srv.max_used <= budget
    assert all(t.completed is not None and t._done_steps == t.request.steps for t in tickets)


def test_a_request_larger_than_the_budget_is_refused():
    srv = FakeServer(1000)
    with pytest.raises(nat.FdetdError):
        srv.submit(_field())
    srv.close()


def test_latency_statistics():
    tickets = []
    for i, lat in enumerate([1.0, 2.0, 3.0, 4.0, 100.0]):
        t = serve.Ticket(i, None, arrival=10.0)
        t.completed = 10.0 + lat
        tickets.append(t)
    s = serve.latency_stats(tickets)
    assert s["count"] == 5 and s["p50_s"] == 3.0 and s["max_s"] == 100.0
    assert s["p99_s"] == pytest.approx(np.percentile([1, 2, 3, 4, 100], 99))
    assert serve.latency_stats([serve.Ticket(0, None, 0.0)]) == {}
