"""Host-side logic of the library's continuous-batching server (CPU only): in dry-run mode the server makes no
CUDA call (plans are only checked on the host and a chunk takes a fixed host time per step), so admission
order, the HBM budget, memory accounting, failure handling and the latency statistics are checked without a
GPU."""
import numpy as np
import pytest

from paper_2605_12132_gb300 import _native as nat
from paper_2605_12132_gb300 import serve


def _field(Nz=64, Nr=32, modes=(0, 1), steps=5, prec="bf16x3", with_J=True, order=8):
    F = np.zeros((len(modes), 6, Nz, Nr), complex)
    J = np.zeros((len(modes), 3, Nz, Nr), complex) if with_J else None
    return serve.FieldRequest(Nz, Nr, list(modes), order, 0.1, 0.1, 0.1, steps, F, J, prec)


def _envelope(Nz=64, Nr=32, steps=7):
    a = np.zeros((2, Nz, Nr), complex)
    return serve.EnvelopeRequest(Nz, Nr, 8, 4, 0.2, 0.25, 0.05, steps, a, np.zeros((Nz, Nr)))


def test_estimate_bytes_grows_with_precision_current_and_size():
    b3, b6 = serve.estimate_bytes(_field(prec="bf16x3")), serve.estimate_bytes(_field(prec="bf16x6"))
    f32, f64 = serve.estimate_bytes(_field(prec="fp32")), serve.estimate_bytes(_field(prec="fp64"))
    assert b6 > b3 and f64 > f32
    noJ = serve.estimate_bytes(_field(with_J=False))
    assert b3 - noJ >= 2 * 3 * 64 * 32 * 8          # the resident current: modes x 3 x Nz x Nr complex64
    assert serve.estimate_bytes(_field(Nz=128)) > b3
    # envelope: state, chi, the plan's three Taylor buffers and the chi + sigma^2 plane
    assert serve.estimate_bytes(_envelope()) >= 64 * 32 * (16 + 4 + 48 + 4)


def test_first_come_first_served_within_the_budget():
    reqs = [_field(Nz=int(Nz), steps=int(s)) for Nz, s in zip([64, 256, 64, 128, 512, 64, 128, 256],
                                                                [5, 40, 3, 17, 9, 1, 33, 2])]
    reqs.insert(3, _envelope(steps=11))
    sizes = [serve.estimate_bytes(r) for r in reqs]
    budget = max(sizes) + min(sizes)                 # the largest fits, but never next to a mid-sized one
    srv = serve.Server(budget, chunk_steps=4, plan_workers=2, dry_run=True)
    tickets = [srv.submit(r) for r in reqs]
    srv.drain(timeout=60)
    st = srv.stats()
    admitted = [t.times()[1] for t in tickets]
    assert admitted == sorted(admitted)              # admission in submission order: no overtaking
    assert all(t.state == serve.DONE for t in tickets)
    assert st["used_bytes"] == 0 and st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_bytes"] <= budget
    assert all(t.latency is not None and t.latency >= 0 for t in tickets)
    srv.close()


def test_a_request_larger_than_the_budget_is_refused():
    srv = serve.Server(1000, dry_run=True)
    with pytest.raises(nat.FdetdError):
        srv.submit(_field())
    srv.close()


def test_a_failed_request_returns_its_budget_and_the_server_keeps_running():
    # order 16 needs Nr > 8: the plan rejects Nr = 6, after admission
    bad = _field(Nr=6, order=16)
    good = [_field(steps=3), _envelope(steps=5), _field(Nz=128, steps=9)]
    srv = serve.Server(10 * max(serve.estimate_bytes(r) for r in good), chunk_steps=4, dry_run=True)
    tb = srv.submit(bad)
    tg = [srv.submit(r) for r in good]
    with pytest.raises(nat.FdetdError):
        tb.wait(30)
    for t in tg:
        t.wait(30)
    st = srv.stats()
    assert tb.state == serve.FAILED and all(t.state == serve.DONE for t in tg)
    assert st["failed"] == 1 and st["completed"] == 3 and st["used_bytes"] == 0
    srv.close()


def test_destroy_finishes_what_was_submitted():
    srv = serve.Server(1 << 30, chunk_steps=2, dry_run=True)
    tickets = [srv.submit(_field(steps=s)) for s in (3, 8, 5)]
    srv.close()                                      # joins after every submitted request is done
    assert srv.handle is None


class _T:
    def __init__(self, lat):
        self.latency = lat


def test_latency_statistics():
    tickets = [_T(x) for x in [1.0, 2.0, 3.0, 4.0, 100.0]]
    s = serve.latency_stats(tickets)
    assert s["count"] == 5 and s["p50_s"] == 3.0 and s["max_s"] == 100.0
    assert s["p99_s"] == pytest.approx(np.percentile([1, 2, 3, 4, 100], 99))
    assert serve.latency_stats([_T(None)]) == {"count": 0}


def test_cancel_queued_ends_only_the_waiting_requests():
    reqs = [_field(Nz=256, steps=400) for _ in range(6)]
    one = serve.estimate_bytes(reqs[0])
    srv = serve.Server(one * 2, chunk_steps=2, dry_run=True)   # two fit at a time
    tickets = [srv.submit(r) for r in reqs]
    import time
    time.sleep(0.05)
    n = srv.cancel_queued()
    srv.drain(timeout=60)
    states = [t.state for t in tickets]
    assert n >= 1 and states.count(serve.FAILED) == n
    assert states.count(serve.DONE) == len(reqs) - n
    st = srv.stats()
    assert st["used_bytes"] == 0 and st["failed"] == n
    srv.close()


def test_prewarm_fills_the_radial_table_cache_once_per_grid():
    nat.fdetd_plan_cache_set_limit(0)
    nat.fdetd_plan_cache_set_limit(1 << 30)
    reqs = [_field(Nr=48, modes=(0, 1)), _field(Nr=48, modes=(1, 2), Nz=128), _envelope(), _field(Nr=40, modes=(0,))]
    srv = serve.Server(1 << 30, dry_run=True)
    assert srv.prewarm(reqs, workers=3) == 4          # (48, m) for m = 0, 1, 2 and (40, 0)
    st = nat.fdetd_plan_cache_stats()
    assert st["entries"] == 4 and st["misses"] >= 4
    hits = st["hits"]
    assert srv.prewarm(reqs) == 4
    assert nat.fdetd_plan_cache_stats()["misses"] == st["misses"]   # already there: no new builds
    assert nat.fdetd_plan_cache_stats()["hits"] == hits
    srv.close()
    nat.fdetd_plan_cache_set_limit(4 << 30)
