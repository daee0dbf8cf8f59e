"""Continuous-batching server for field-advance and envelope-advance requests: the Python face of the
library's fdetd_server_* calls (include/fdetd.h).

The scheduling lives in the library (one scheduler thread and plan-builder threads in C++): requests are
admitted first-come first-served by HBM budget, field requests that are resident on the device advance
together as the instances of one batch (one CUDA graph per step with grouped tensor-core launches,
re-captured when a request joins or leaves), envelope requests advance on their own streams alongside,
and each result is copied back to a host buffer when its request finishes.  This module only marshals
requests, keeps their host buffers alive until they finish, and feeds Poisson arrivals.
"""
import ctypes
import time
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import _native as nat

REQUEST_FIELD, REQUEST_ENVELOPE = 0, 1
QUEUED, ADMITTED, RUNNING, DONE, FAILED = range(5)
DRY_RUN = 1
_PREC = {"fp64": 0, "fp32": 1, "bf16x3": 2, "bf16x6": 3}


class _Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("Nz", ctypes.c_int), ("Nr", ctypes.c_int), ("nmodes", ctypes.c_int),
                ("modes", ctypes.POINTER(ctypes.c_int)), ("order", ctypes.c_int), ("precision", ctypes.c_int),
                ("taylor_order", ctypes.c_int), ("steps", ctypes.c_int), ("dz", ctypes.c_double),
                ("dr", ctypes.c_double), ("dt", ctypes.c_double), ("k0", ctypes.c_double),
                ("fields", ctypes.c_void_p), ("J", ctypes.c_void_p), ("chi", ctypes.c_void_p),
                ("out", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("queued", ctypes.c_size_t), ("building", ctypes.c_size_t), ("running", ctypes.c_size_t),
                ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("recaptures", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("served_cell_steps", ctypes.c_double)]


def _bind():
    L = nat.lib()
    if getattr(L, "_server_bound", False):
        return L
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    L.fdetd_request_device_bytes.argtypes = [ctypes.POINTER(_Request)]
    L.fdetd_request_device_bytes.restype = ctypes.c_size_t
    L.fdetd_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, ctypes.c_int, ctypes.c_int, u64]
    L.fdetd_server_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(u64)]
    L.fdetd_server_poll.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.fdetd_server_wait.argtypes = [vp, u64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.fdetd_server_ticket_times.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_double)]
    L.fdetd_server_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    L.fdetd_server_cancel_queued.argtypes = [vp, ctypes.POINTER(u64)]
    L.fdetd_server_destroy.argtypes = [vp]
    L._server_bound = True
    return L


@dataclass
class FieldRequest:
    Nz: int
    Nr: int
    modes: List[int]
    order: int
    dz: float
    dr: float
    dt: float
    steps: int
    F: np.ndarray                 # [nmodes][6][Nz][Nr] complex
    J: Optional[np.ndarray] = None
    precision: str = "bf16x6"
    kind: str = "field"


@dataclass
class EnvelopeRequest:
    Nz: int
    Nr: int
    order: int
    taylor_order: int
    dz: float
    dr: float
    dt: float
    steps: int
    a: np.ndarray                 # [2][Nz][Nr] complex (a, a~)
    chi: np.ndarray               # [Nz][Nr] real
    k0: float = 2 * np.pi
    kind: str = "envelope"


class Ticket:
    """A submitted request: its id, the host buffers the library reads and writes, and its result."""

    def __init__(self, server, request, c_req, keep):
        self.server, self.request, self._c_req, self._keep = server, request, c_req, keep
        self.id = None
        self.arrival = None
        self._final = None      # (state, latency) once done or failed: kept after the server is closed

    def _poll(self):
        if self._final is not None:
            return self._final
        if not self.server.handle:
            return (QUEUED, None)
        lat = ctypes.c_double(-1.0)
        st = ctypes.c_int(0)
        _bind().fdetd_server_poll(self.server.handle, self.id, ctypes.byref(st), ctypes.byref(lat))
        if st.value in (DONE, FAILED):
            self._final = (st.value, lat.value if st.value == DONE else None)
            return self._final
        return (st.value, None)

    @property
    def state(self):
        return self._poll()[0]

    @property
    def latency(self):
        """Completion minus submission time in seconds, None until done."""
        return self._poll()[1]

    def times(self):
        t = (ctypes.c_double * 3)()
        nat._check(_bind().fdetd_server_ticket_times(self.server.handle, self.id, t))
        return tuple(t)

    @property
    def result(self):
        return self._keep["out"] if self.state == DONE else None

    def wait(self, timeout=600.0):
        lat = ctypes.c_double(-1.0)
        nat._check(_bind().fdetd_server_wait(self.server.handle, self.id, timeout, ctypes.byref(lat)))
        return lat.value


def _c_request(req, keep_result=True):
    """The C request and the host arrays it points into (kept alive by the ticket); without keep_result the
    library copies no result back."""
    keep = {}
    r = _Request()
    r.Nz, r.Nr, r.order, r.steps = req.Nz, req.Nr, req.order, req.steps
    r.dz, r.dr, r.dt = req.dz, req.dr, req.dt
    if req.kind == "envelope":
        r.kind = REQUEST_ENVELOPE
        r.taylor_order, r.k0 = req.taylor_order, req.k0
        keep["fields"] = np.ascontiguousarray(req.a, dtype=np.complex64)
        keep["chi"] = np.ascontiguousarray(req.chi, dtype=np.float32)
        r.chi = keep["chi"].ctypes.data
    else:
        r.kind = REQUEST_FIELD
        r.precision = _PREC[req.precision]
        cdt = np.complex128 if req.precision == "fp64" else np.complex64
        keep["modes"] = (ctypes.c_int * len(req.modes))(*req.modes)
        r.nmodes = len(req.modes)
        r.modes = keep["modes"]
        keep["fields"] = np.ascontiguousarray(req.F, dtype=cdt)
        if req.J is not None:
            keep["J"] = np.ascontiguousarray(req.J, dtype=cdt)
            r.J = keep["J"].ctypes.data
    keep["out"] = np.empty_like(keep["fields"]) if keep_result else None
    r.fields = keep["fields"].ctypes.data
    r.out = keep["out"].ctypes.data if keep_result else None
    return r, keep


def estimate_bytes(req):
    """Device bytes the server reserves for a request while it is admitted (fdetd_request_device_bytes)."""
    r, _ = _c_request(req)
    return int(_bind().fdetd_request_device_bytes(ctypes.byref(r)))


class Server:
    def __init__(self, hbm_budget, chunk_steps=16, plan_workers=4, dry_run=False):
        L = _bind()
        h = ctypes.c_void_p()
        nat._check(L.fdetd_server_create(ctypes.byref(h), int(hbm_budget), int(chunk_steps), int(plan_workers),
                                         DRY_RUN if dry_run else 0))
        self.handle = h
        self.budget = int(hbm_budget)
        self.tickets = []

    def submit(self, req, arrival=None, keep_result=True):
        r, keep = _c_request(req, keep_result)
        t = Ticket(self, req, r, keep)
        tid = ctypes.c_uint64(0)
        nat._check(_bind().fdetd_server_submit(self.handle, ctypes.byref(r), ctypes.byref(tid)))
        t.id = tid.value
        t.arrival = time.perf_counter() if arrival is None else arrival
        self.tickets.append(t)
        return t

    def prewarm(self, requests, workers=8):
        """Compute the radial tables of the field requests' grids into the library's plan cache before they
        arrive (distinct (Nr, order, dr, mode) only, on `workers` threads; the calls release the GIL).
        Returns the number of distinct mode tables."""
        import concurrent.futures as cf
        keys = sorted({(r.Nr, r.order, float(r.dr), m) for r in requests if r.kind == "field" for m in r.modes},
                      key=lambda k: -k[0])
        with cf.ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
            list(ex.map(lambda k: nat.fdetd_plan_cache_warm(k[0], k[1], k[2], [k[3]]), keys))
        return len(keys)

    def stats(self):
        s = _Stats()
        nat._check(_bind().fdetd_server_stats(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    @property
    def used(self):
        return self.stats()["used_bytes"]

    @property
    def peak_used(self):
        return self.stats()["peak_bytes"]

    def pending(self):
        s = self.stats()
        return s["queued"] + s["building"] + s["running"]

    def drain(self, timeout=600.0):
        t0 = time.perf_counter()
        for t in self.tickets:
            left = max(0.0, timeout - (time.perf_counter() - t0))
            lat = ctypes.c_double(-1.0)
            rc = _bind().fdetd_server_wait(self.handle, t.id, left, ctypes.byref(lat))
            if rc == 6:
                raise TimeoutError("server did not drain in time")

    def cancel_queued(self):
        """End every request still waiting for admission (failed, 'cancelled before admission')."""
        n = ctypes.c_uint64(0)
        nat._check(_bind().fdetd_server_cancel_queued(self.handle, ctypes.byref(n)))
        return n.value

    def close(self):
        """Finish every submitted request, record each ticket's final state, then stop the server."""
        if self.handle:
            self.drain(timeout=3600.0)
            for t in self.tickets:
                t._poll()
            _bind().fdetd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_poisson(server, make_request, rate_hz, duration_s, seed=0, max_requests=None, keep_result=True):
    """Submit requests with Poisson arrivals (rate_hz over duration_s), each built when it arrives; returns the
    tickets (not waited for)."""
    rng = np.random.default_rng(seed)
    times = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s or (max_requests and len(times) >= max_requests):
            break
        times.append(t)
    t0 = time.perf_counter()
    tickets = []
    for k, at in enumerate(times):
        req = make_request(k, rng)
        delay = t0 + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(server.submit(req, arrival=t0 + at, keep_result=keep_result))
    return tickets


def latency_stats(tickets):
    lat = np.array([x for x in (t.latency for t in tickets) if x is not None])
    if lat.size == 0:
        return {"count": 0}
    return {"count": int(lat.size), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
