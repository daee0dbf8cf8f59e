"""Continuous-batching server for field-advance and envelope-advance requests.

Requests of different sizes arrive over time; each is admitted when its device footprint
(plan tables + scratch + resident state) fits the HBM budget, gets its own CUDA stream and
stays resident on the device until it completes.  Work advances in chunks of a few steps per
request per scheduling round, so requests that arrive while others run are admitted as soon as
memory frees up and their chunks interleave with the running ones on the device.  Plans are
built on worker threads (the host eigen-solve runs in C++ and releases the GIL).  All device
work is done by the C-ABI library; this module only schedules it.
"""
import concurrent.futures as cf
import itertools
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import _native as nat


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
    precision: str = "bf16x3"
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


@dataclass
class Ticket:
    id: int
    request: object
    arrival: float
    admitted: Optional[float] = None
    completed: Optional[float] = None
    result: Optional[np.ndarray] = None
    bytes: int = 0
    # device-side state while active
    _plan: object = None
    _state: object = None
    _aux: object = None
    _stream: object = None
    _done_steps: int = 0
    _event: object = None
    _host: object = None
    _future: object = None

    @property
    def latency(self):
        return None if self.completed is None else self.completed - self.arrival


def _pad(x, m):
    return (x + m - 1) // m * m


def estimate_bytes(req):
    """Device bytes a request holds while admitted (plan tables, scratch, resident state)."""
    if req.kind == "envelope":
        cells = req.Nz * req.Nr
        return cells * (2 * 8 + 4 + 6 * 8) + req.Nr * (req.order + 2) * 4
    n, Nz, nm = req.Nr, req.Nz, len(req.modes)
    cells = nm * Nz * n
    elt = 16 if req.precision == "fp64" else 8
    state = cells * 6 * elt + (cells * 3 * elt if req.J is not None else 0)
    coef = cells * 9 * elt
    phase = nm * 2 * n * Nz * (32 if req.precision == "fp64" else 16)
    tables = phase + Nz * 16 * 2 + nm * 2 * n * 16 + 64
    if req.precision in ("bf16x3", "bf16x6"):
        npc = 2 if req.precision == "bf16x3" else 3
        kp = _pad(n, 64)
        mats = nm * 2 * npc * (3 * _pad(n, 256) + 3 * _pad(n, 128)) * 3 * kp * 2
        split = nm * npc * 6 * kp * 2 * Nz * 2
        tables += mats + split
    else:
        tables += 2 * nm * 2 * (3 * n) ** 2 * (8 if req.precision == "fp64" else 4)
    return state + coef + tables


class Server:
    def __init__(self, hbm_budget, chunk_steps=16, plan_workers=4):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget)
        self.used = 0
        self.peak_used = 0
        self.chunk = chunk_steps
        self.queue: List[Ticket] = []      # arrived, not admitted
        self.building: List[Ticket] = []   # admitted, plan under construction
        self.active: List[Ticket] = []     # on the device
        self.finishing: List[Ticket] = []  # last chunk launched, waiting for its event
        self.done: List[Ticket] = []
        self.ids = itertools.count()
        self.pool = cf.ThreadPoolExecutor(max_workers=plan_workers)
        self.streams = []

    # ------------------------------------------------------------- API
    def submit(self, req, arrival=None):
        t = Ticket(next(self.ids), req, time.perf_counter() if arrival is None else arrival)
        t.bytes = estimate_bytes(req)
        if t.bytes > self.budget:
            raise nat.FdetdError(f"request {t.id} needs {t.bytes} bytes, more than the whole budget {self.budget}")
        self.queue.append(t)
        return t

    def pending(self):
        return len(self.queue) + len(self.building) + len(self.active) + len(self.finishing)

    def pump(self):
        """One scheduling round: admit, start plans, launch chunks, reap completions."""
        self._admit()
        self._start_ready()
        self._launch_chunks()
        self._reap()

    def drain(self, timeout=600.0):
        t0 = time.perf_counter()
        while self.pending():
            self.pump()
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError("server did not drain in time")
            time.sleep(0)

    def close(self):
        self.pool.shutdown(wait=True)

    # ------------------------------------------------------------- internals
    def _admit(self):
        # first-come first-served; a request that does not fit waits (no overtaking, no starvation)
        while self.queue and self.used + self.queue[0].bytes <= self.budget:
            t = self.queue.pop(0)
            self.used += t.bytes
            self.peak_used = max(self.peak_used, self.used)
            t.admitted = time.perf_counter()
            t._future = self.pool.submit(self._build_plan, t.request)
            self.building.append(t)

    @staticmethod
    def _build_plan(req):
        if req.kind == "envelope":
            return nat.envelope_plan(req.Nz, req.Nr, req.order, req.taylor_order, req.dz, req.dr, req.dt, req.k0)
        return nat.fdetd_plan_modes(req.Nz, req.Nr, req.modes, req.order, req.dz, req.dr, req.dt,
                                    precision=req.precision)

    def _stream(self):
        if self.streams:
            return self.streams.pop()
        return self.torch.cuda.Stream()

    def _start_ready(self):
        torch = self.torch
        still = []
        for t in self.building:
            if not t._future.done():
                still.append(t)
                continue
            t._plan = t._future.result()
            t._stream = self._stream()
            req = t.request
            with torch.cuda.stream(t._stream):
                if req.kind == "envelope":
                    t._state = torch.from_numpy(req.a).to(torch.complex64).to("cuda", non_blocking=True)
                    t._aux = torch.from_numpy(np.ascontiguousarray(req.chi, dtype=np.float32)).to("cuda", non_blocking=True)
                else:
                    cdt = t._plan.complex_dtype
                    t._state = torch.from_numpy(req.F).to(cdt).to("cuda", non_blocking=True)
                    t._aux = (torch.from_numpy(req.J).to(cdt).to("cuda", non_blocking=True)
                              if req.J is not None else None)
            self.active.append(t)
        self.building = still

    def _launch_chunks(self):
        torch = self.torch
        still = []
        for t in self.active:
            req = t.request
            n = min(self.chunk, req.steps - t._done_steps)
            if req.kind == "envelope":
                nat.envelope_step(t._plan, t._state, t._aux, n, stream=t._stream)
            else:
                nat.fdetd_step(t._plan, t._state, t._aux, n, stream=t._stream)
            t._done_steps += n
            if t._done_steps >= req.steps:
                with torch.cuda.stream(t._stream):
                    t._host = t._state.to("cpu", non_blocking=True)
                    t._event = torch.cuda.Event()
                    t._event.record(t._stream)
                self.finishing.append(t)
            else:
                still.append(t)
        self.active = still

    def _reap(self):
        still = []
        for t in self.finishing:
            if t._event.query():
                t.completed = time.perf_counter()
                t.result = t._host.numpy().copy()
                if t.request.kind == "field":
                    t._plan.status(t._stream)
                t._plan.close()
                self.streams.append(t._stream)
                t._plan = t._state = t._aux = t._host = t._event = None
                self.used -= t.bytes
                self.done.append(t)
            else:
                still.append(t)
        self.finishing = still


def run_poisson(server, make_request, rate_hz, duration_s, seed=0, max_requests=None):
    """Feed requests with Poisson arrivals (rate_hz over duration_s) and serve them; returns tickets."""
    rng = np.random.default_rng(seed)
    times = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s or (max_requests and len(times) >= max_requests):
            break
        times.append(t)
    reqs = [make_request(i, rng) for i in range(len(times))]
    t0 = time.perf_counter()
    tickets = []
    k = 0
    while k < len(times) or server.pending():
        now = time.perf_counter() - t0
        while k < len(times) and times[k] <= now:
            tickets.append(server.submit(reqs[k], arrival=t0 + times[k]))
            k += 1
        server.pump()
    return tickets


def latency_stats(tickets):
    lat = np.array([t.latency for t in tickets if t.latency is not None])
    if lat.size == 0:
        return {}
    return {"count": int(lat.size), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
