"""ctypes binding of libfdetd.so (same names as the C-ABI; marshalling only)."""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

PRECISIONS = {"fp64": 0, "fp32": 1, "bf16x3": 2, "bf16x6": 3}


class FdetdError(RuntimeError):
    """A library call failed; `code` is its FDETD_ERR_* value."""

    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


def lib_path():
    return os.path.join(_HERE, "lib", "libfdetd.so")


def lib():
    """Load libfdetd.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise FdetdError(f"{path} is missing; build it with `python {_HERE}/build.py` "
                         "(or __graft_entry__.build())")
    L = ctypes.CDLL(path)
    c_int, c_dbl, c_vp, c_u64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_uint64
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    L.fdetd_plan.argtypes = [ctypes.POINTER(c_vp), c_int, c_int, c_int, c_int, c_dbl, c_dbl, c_dbl, c_int, c_u64]
    L.fdetd_plan_modes.argtypes = [ctypes.POINTER(c_vp), c_int, c_int, ctypes.POINTER(c_int), c_int, c_int,
                                   c_dbl, c_dbl, c_dbl, c_int, c_u64]
    L.fdetd_step.argtypes = [c_vp, c_vp, c_vp, c_int, c_vp]
    L.fdetd_step_host.argtypes = [c_vp, c_vp, c_vp, c_int, c_vp]
    L.fdetd_destagger.argtypes = [c_vp, c_vp, c_vp, c_vp]
    L.fdetd_current_correct.argtypes = [c_vp, c_vp, c_vp, c_vp, c_vp]
    L.fdetd_current_host_bands.argtypes = [c_int, c_int, c_dbl, c_int, dp, dp, dp, dp]
    L.fdetd_plan_device_bytes.argtypes = [c_vp]
    L.fdetd_plan_device_bytes.restype = ctypes.c_size_t
    L.fdetd_plan_launches_per_step.argtypes = [c_vp]
    L.fdetd_plan_destroy.argtypes = [c_vp]
    L.fdetd_plan_set_profiling.argtypes = [c_vp, c_int]
    L.fdetd_plan_status.argtypes = [c_vp, c_vp]
    L.fdetd_stream_status.argtypes = [c_vp, c_vp]
    L.fdetd_plan_set_wait_limit.argtypes = [c_vp, ctypes.c_longlong]
    L.fdetd_plan_kernel_times.argtypes = [c_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long)]
    L.fdetd_host_tables.argtypes = [c_int, c_int, c_int, c_int, c_dbl, c_dbl, c_dbl, dp, dp, dp, dp, dp, dp,
                                    u8p, u8p, dp, dp, dp]
    L.fdetd_host_coeffs.argtypes = [c_int, c_int, dp]
    L.fdetd_host_spectral_order.argtypes = [c_int, c_int, c_vp]
    L.fdetd_host_spectral_radices.argtypes = [c_int, c_int, ctypes.POINTER(c_int)]
    L.fdetd_plan_cache_set_limit.argtypes = [ctypes.c_size_t]
    L.fdetd_plan_cache_warm.argtypes = [c_int, c_int, c_dbl, ctypes.POINTER(c_int), c_int]
    L.fdetd_plan_cache_stats.argtypes = [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                         ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64)]
    L.envelope_plan.argtypes = [ctypes.POINTER(c_vp), c_int, c_int, c_int, c_int, c_dbl, c_dbl, c_dbl, c_dbl]
    L.envelope_step.argtypes = [c_vp, c_vp, c_vp, c_int, c_vp]
    L.envelope_step_absorbing.argtypes = [c_vp, c_vp, c_vp, c_vp, c_int, c_vp]
    L.envelope_step_fused.argtypes = [c_vp, c_vp, c_vp, c_int, c_vp]
    L.envelope_plan_launches_per_step.argtypes = [c_vp]
    L.envelope_plan_device_bytes.argtypes = [c_vp]
    L.envelope_plan_device_bytes.restype = ctypes.c_size_t
    L.fdetd_batch_create.argtypes = [ctypes.POINTER(c_vp)]
    L.fdetd_batch_add.argtypes = [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(c_int)]
    L.fdetd_batch_capture.argtypes = [c_vp, c_int, c_vp]
    L.fdetd_batch_set_autotune.argtypes = [c_vp, c_int]
    L.fdetd_batch_group_info.argtypes = [c_vp, c_int, ctypes.POINTER(c_int), dp]
    L.fdetd_plan_autotune.argtypes = [c_vp, c_vp, c_vp, c_vp, dp]
    L.fdetd_plan_tile_config.argtypes = [c_vp, ctypes.POINTER(c_int)]
    L.fdetd_plan_set_tile_config.argtypes = [c_vp, ctypes.POINTER(c_int)]
    L.fdetd_probe_mma_rounding.argtypes = [ctypes.POINTER(ctypes.c_float), c_int, c_vp]
    L.fdetd_taylor_plan.argtypes = [ctypes.POINTER(c_vp), c_int, c_int, ctypes.POINTER(c_int), c_int, c_int, c_dbl,
                                    c_dbl, c_dbl, c_int, c_int]
    L.fdetd_taylor_step.argtypes = [c_vp, c_vp, c_vp, c_int, c_vp]
    L.fdetd_taylor_launches_per_step.argtypes = [c_vp]
    L.fdetd_taylor_destroy.argtypes = [c_vp]
    L.fdetd_taylor_host_bands.argtypes = [c_int, c_int, c_dbl, c_int, dp, dp]
    L.fdetd_batch_launch.argtypes = [c_vp, c_vp]
    L.fdetd_batch_set_profiling.argtypes = [c_vp, c_int]
    L.fdetd_batch_collect_stage_times.argtypes = [c_vp]
    L.fdetd_batch_stage_times.argtypes = [c_vp, dp, ctypes.POINTER(ctypes.c_long)]
    L.fdetd_batch_pipeline_waits.argtypes = [c_vp, ctypes.POINTER(ctypes.c_uint64)]
    L.fdetd_batch_set_host_pipeline.argtypes = [c_vp, c_int]
    L.fdetd_host_split_parts.argtypes = [ctypes.POINTER(ctypes.c_size_t), c_int, c_int, ctypes.POINTER(c_int)]
    L.fdetd_host_plan_digest.argtypes = [c_int, c_int, ctypes.POINTER(c_int), c_int, c_int, c_dbl, c_dbl, c_dbl, dp]
    L.fdetd_plan_pipeline_waits.argtypes = [c_vp, ctypes.POINTER(ctypes.c_uint64)]
    L.fdetd_batch_step_host.argtypes = [c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_int, c_vp]
    L.fdetd_batch_destroy.argtypes = [c_vp]
    L.envelope_step_static.argtypes = [c_vp, c_vp, c_int, c_int, c_int, c_int, c_dbl, c_dbl, c_dbl, c_dbl, c_int,
                                       c_vp]
    L.envelope_plan_destroy.argtypes = [c_vp]
    L.fdetd_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    _LIB = L
    return L


def _check(rc):
    if rc != 0:
        buf = ctypes.create_string_buffer(512)
        lib().fdetd_last_error(buf, 512)
        raise FdetdError(f"fdetd error {rc}: {buf.value.decode(errors='replace')}", rc)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if arr is not None else None


PIPELINE_SLOTS = ("cta", "mma_wait_a", "mma_wait_b", "mma_wait_tmem", "producer_wait_stage",
                  "converter_wait_staged", "converter_busy", "epilogue_busy")


SPECTRAL_PHASES = ("cycles", "load_and_first_stage", "forward_stages", "middle_fused", "inverse_stages",
                   "output_stage", "blocks")


def pipeline_report(counters):
    """The 24 raw counters as {kernel: {slot: share of the residency}} with the raw cycle sums: the two
    tensor-core kernels' role waits, and the phases of the spectral kernel specialised on Nz (per block)."""
    rep = {}
    for k, name in enumerate(("projection", "backprojection")):
        c = counters[8 * k: 8 * k + 8]
        tot = c[0]
        rep[name] = {"cycles": tot}
        if tot:
            rep[name].update({slot: c[i] / tot for i, slot in enumerate(PIPELINE_SLOTS) if i})
    c = counters[16:24]
    rep["spectral"] = {"cycles": c[0], "blocks": c[6]}
    if c[0]:
        rep["spectral"].update({ph: c[i] / c[0] for i, ph in enumerate(SPECTRAL_PHASES) if 1 <= i <= 5})
        rep["spectral"]["cycles_per_block"] = c[0] / max(c[6], 1)
    return rep


class FdetdPlan:
    def __init__(self, handle, Nz, Nr, modes, order, dz, dr, dt, precision):
        self.handle = handle
        self.Nz, self.Nr, self.modes, self.order = Nz, Nr, list(modes), order
        self.dz, self.dr, self.dt, self.precision = dz, dr, dt, precision

    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == "fp64" else torch.complex64

    @property
    def device_bytes(self):
        return lib().fdetd_plan_device_bytes(self.handle)

    @property
    def launches_per_step(self):
        return lib().fdetd_plan_launches_per_step(self.handle)

    def status(self, stream=None):
        """Synchronise and raise FdetdError if an earlier step failed on the device."""
        _check(lib().fdetd_plan_status(self.handle, _stream_handle(stream)))

    def set_wait_limit(self, polls=-1):
        """Polls before a tensor-core pipeline wait gives up (< 0: default; 0: at once, drives the timeout path)."""
        _check(lib().fdetd_plan_set_wait_limit(self.handle, int(polls)))

    def set_profiling(self, on=True):
        _check(lib().fdetd_plan_set_profiling(self.handle, int(on)))

    def kernel_times(self):
        """{stage: (total_ms, launches)} for stages projection / spectral / backprojection."""
        ms = (ctypes.c_double * 3)()
        calls = (ctypes.c_long * 3)()
        _check(lib().fdetd_plan_kernel_times(self.handle, ms, calls))
        return {name: (ms[i], calls[i]) for i, name in enumerate(("projection", "spectral", "backprojection"))}

    def pipeline_waits(self):
        """Pipeline cycle counters of the tensor-core kernels while profiling is on (see pipeline_report)."""
        out = (ctypes.c_uint64 * 24)()
        _check(lib().fdetd_plan_pipeline_waits(self.handle, out))
        return pipeline_report(list(out))

    @property
    def tile_config(self):
        """Tensor-core tile configuration (tn_proj, tn_back, sched_proj, sched_back)."""
        cfg = (ctypes.c_int * 4)()
        _check(lib().fdetd_plan_tile_config(self.handle, cfg))
        return tuple(cfg)

    @tile_config.setter
    def tile_config(self, cfg):
        arr = (ctypes.c_int * 4)(*cfg)
        _check(lib().fdetd_plan_set_tile_config(self.handle, arr))

    def autotune(self, fields, J=None, stream=None):
        """Time the tensor-core tile configurations on these device arrays (read only) and keep the
        fastest; returns (best projection ms, best back-projection ms).  No-op for fp64 / fp32."""
        _check_tensor(fields, self, 6, "fields")
        jp = None
        if J is not None:
            _check_tensor(J, self, 3, "J")
            jp = J.data_ptr()
        ms = (ctypes.c_double * 2)()
        _check(lib().fdetd_plan_autotune(self.handle, fields.data_ptr(), jp, _stream_handle(stream), ms))
        return ms[0], ms[1]

    def close(self):
        if self.handle:
            lib().fdetd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SPECTRAL_COLUMNS = 1   # plan flag: the z transform in its column-split form (FDETD_FLAG_SPECTRAL_COLUMNS)
J_ON_PRIMARY = 2       # plan flag: J_rho given on the primary radial grid, downstaggered by the step


def fdetd_plan_modes(Nz, Nr, modes, order, dz, dr, dt, precision="fp64", flags=0):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * len(modes))(*modes)
    _check(lib().fdetd_plan_modes(ctypes.byref(h), Nz, Nr, arr, len(modes), order, dz, dr, dt,
                                  PRECISIONS[precision], flags))
    return FdetdPlan(h, Nz, Nr, modes, order, dz, dr, dt, precision)


def fdetd_plan(Nz, Nr, M, order, dz, dr, dt, precision="fp64", flags=0):
    return fdetd_plan_modes(Nz, Nr, list(range(M + 1)), order, dz, dr, dt, precision, flags)


def _check_tensor(t, plan, ncomp, name):
    shape = (len(plan.modes), ncomp, plan.Nz, plan.Nr)
    if tuple(t.shape) != shape:
        raise FdetdError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
    if t.dtype != plan.complex_dtype:
        raise FdetdError(f"{name} must be {plan.complex_dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise FdetdError(f"{name} must be contiguous")


def fdetd_step(plan, fields, J=None, nsteps=1, stream=None):
    """Advance device `fields` in place by nsteps exact midpoint steps (see include/fdetd.h)."""
    if not fields.is_cuda:
        raise FdetdError("fields must be a CUDA tensor (use fdetd_step_host for host arrays)")
    _check_tensor(fields, plan, 6, "fields")
    jp = None
    if J is not None:
        _check_tensor(J, plan, 3, "J")
        jp = J.data_ptr()
    _check(lib().fdetd_step(plan.handle, fields.data_ptr(), jp, nsteps, _stream_handle(stream)))
    return fields


def fdetd_destagger(plan, fields, out=None, stream=None):
    """Fields of `plan` on the Yee grid -> all six on the primary grids (new tensor unless `out` given)."""
    import torch
    _check_tensor(fields, plan, 6, "fields")
    if not fields.is_cuda:
        raise FdetdError("fields must be a CUDA tensor")
    if out is None:
        out = torch.empty_like(fields)
    _check_tensor(out, plan, 6, "out")
    _check(lib().fdetd_destagger(plan.handle, fields.data_ptr(), out.data_ptr(), _stream_handle(stream)))
    return out


def fdetd_current_correct(plan, J, rho_xy, out=None, stream=None):
    """Deposited J [modes][3][Nz][Nr] and rho_xy [modes][Nz][Nr] -> corrected J on the field step's Yee grid."""
    import torch
    _check_tensor(J, plan, 3, "J")
    shape = (len(plan.modes), plan.Nz, plan.Nr)
    if tuple(rho_xy.shape) != shape or rho_xy.dtype != plan.complex_dtype or not rho_xy.is_contiguous():
        raise FdetdError(f"rho_xy must be a contiguous {plan.complex_dtype} tensor of shape {shape}")
    if out is None:
        out = torch.empty_like(J)
    _check_tensor(out, plan, 3, "out")
    _check(lib().fdetd_current_correct(plan.handle, J.data_ptr(), rho_xy.data_ptr(), out.data_ptr(),
                                       _stream_handle(stream)))
    return out


def fdetd_current_host_bands(Nr, order, dr, m):
    """Host-only: Div+ and D- bands [Nr][order+1] and the LU factors of the radial Laplacian of mode m."""
    N = order // 2
    divp, dm = np.zeros((Nr, order + 1)), np.zeros((Nr, order + 1))
    lo, up = np.zeros((Nr, N)), np.zeros((Nr, N + 1))
    _check(lib().fdetd_current_host_bands(Nr, order, dr, m, _dptr(divp), _dptr(dm), _dptr(lo), _dptr(up)))
    return divp, dm, lo, up


def fdetd_step_host(plan, host_fields, host_J=None, nsteps=1, stream=None):
    """End-to-end step on HOST tensors (pinned recommended): h2d, step, d2h inside the call."""
    _check_tensor(host_fields, plan, 6, "fields")
    jp = None
    if host_J is not None:
        _check_tensor(host_J, plan, 3, "J")
        jp = host_J.data_ptr()
    _check(lib().fdetd_step_host(plan.handle, host_fields.data_ptr(), jp, nsteps, _stream_handle(stream)))
    return host_fields


def fdetd_host_tables(Nz, Nr, m, order, dz, dr, dt):
    """Host-only FP64 plan tables of one mode (no GPU needed)."""
    N3 = 3 * Nr
    out = {k: np.zeros((N3, N3)) for k in ("PE", "PB", "QE", "QB")}
    out["lam"], out["mu"] = np.zeros(Nr), np.zeros(Nr)
    out["tm_live"], out["te_live"] = np.zeros(Nr, np.uint8), np.zeros(Nr, np.uint8)
    out["kappa2"] = np.zeros(Nz)
    sp, sm = np.zeros(2 * Nz), np.zeros(2 * Nz)
    u8 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    _check(lib().fdetd_host_tables(Nz, Nr, m, order, dz, dr, dt, _dptr(out["PE"]), _dptr(out["PB"]),
                                   _dptr(out["QE"]), _dptr(out["QB"]), _dptr(out["lam"]), _dptr(out["mu"]),
                                   u8(out["tm_live"]), u8(out["te_live"]), _dptr(out["kappa2"]), _dptr(sp),
                                   _dptr(sm)))
    out["sp"] = sp[0::2] + 1j * sp[1::2]
    out["sm"] = sm[0::2] + 1j * sm[1::2]
    return out


class TaylorPlan:
    """The paper's Taylor-polynomial time stepper on the GPU (see include/fdetd.h)."""

    def __init__(self, handle, Nz, Nr, modes, order, dz, dr, dt, taylor_order, substeps):
        self.handle = handle
        self.Nz, self.Nr, self.modes, self.order = Nz, Nr, list(modes), order
        self.dz, self.dr, self.dt = dz, dr, dt
        self.taylor_order, self.substeps = taylor_order, substeps
        self.precision = "fp32"

    @property
    def complex_dtype(self):
        import torch
        return torch.complex64

    @property
    def launches_per_step(self):
        return lib().fdetd_taylor_launches_per_step(self.handle)

    def close(self):
        if self.handle:
            lib().fdetd_taylor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fdetd_taylor_plan(Nz, Nr, modes, order, dz, dr, dt, taylor_order=4, substeps=1):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * len(modes))(*modes)
    _check(lib().fdetd_taylor_plan(ctypes.byref(h), Nz, Nr, arr, len(modes), order, dz, dr, dt, taylor_order,
                                   substeps))
    return TaylorPlan(h, Nz, Nr, modes, order, dz, dr, dt, taylor_order, substeps)


def fdetd_taylor_step(plan, fields, J=None, nsteps=1, stream=None):
    """Advance cuda complex64 `fields` [modes][6][Nz][Nr] in place by nsteps Taylor steps."""
    if not fields.is_cuda:
        raise FdetdError("fields must be a CUDA tensor")
    _check_tensor(fields, plan, 6, "fields")
    jp = None
    if J is not None:
        _check_tensor(J, plan, 3, "J")
        jp = J.data_ptr()
    _check(lib().fdetd_taylor_step(plan.handle, fields.data_ptr(), jp, nsteps, _stream_handle(stream)))
    return fields


def fdetd_taylor_host_bands(Nr, order, dr, m):
    """Host-only: the four banded radial operators [4][Nr][order+1] and axis weights [2][order/2]."""
    bands = np.zeros((4, Nr, order + 1))
    axis = np.zeros((2, order // 2))
    _check(lib().fdetd_taylor_host_bands(Nr, order, dr, m, _dptr(bands), _dptr(axis)))
    return bands, axis


def fdetd_probe_mma_rounding(reps=1, stream=None):
    """Diagnostic tcgen05 accumulation test (see include/fdetd.h): a (12, 2) float32 array."""
    out = (ctypes.c_float * 24)()
    _check(lib().fdetd_probe_mma_rounding(out, reps, _stream_handle(stream)))
    return np.array(out, dtype=np.float32).reshape(12, 2)


def fdetd_host_spectral_order(Nz, precision="bf16x6"):
    """kz index of each entry of the spectral kernel's per-kz tables (see include/fdetd.h)."""
    out = np.zeros(Nz, dtype=np.int32)
    _check(lib().fdetd_host_spectral_order(Nz, PRECISIONS[precision], out.ctypes.data_as(ctypes.c_void_p)))
    return out


def fdetd_host_spectral_radices(Nz, precision="bf16x6"):
    """Host-only: the stage radices of the z transform, first to last (empty when Nz is not 7-smooth)."""
    rad = (ctypes.c_int * 16)()
    n = lib().fdetd_host_spectral_radices(Nz, PRECISIONS[precision], rad)
    if n < 0:
        _check(-n)
    return [rad[k] for k in range(n)]


def fdetd_plan_cache_set_limit(nbytes):
    """Byte limit of the process-wide cache of per-mode radial tables (0 empties and disables it)."""
    _check(lib().fdetd_plan_cache_set_limit(int(nbytes)))


def fdetd_plan_cache_warm(Nr, order, dr, modes):
    """Compute the radial tables of `modes` on the grid (Nr, order, dr) into the cache (host only)."""
    m = (ctypes.c_int * len(modes))(*modes)
    _check(lib().fdetd_plan_cache_warm(int(Nr), int(order), float(dr), m, len(modes)))


def fdetd_plan_cache_stats():
    """The radial-table cache: bytes held, limit, entries, hits and misses since the process started."""
    b, lim = ctypes.c_size_t(0), ctypes.c_size_t(0)
    n = ctypes.c_int(0)
    h, m = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().fdetd_plan_cache_stats(ctypes.byref(b), ctypes.byref(lim), ctypes.byref(n), ctypes.byref(h),
                                        ctypes.byref(m)))
    return {"bytes": b.value, "limit": lim.value, "entries": n.value, "hits": h.value, "misses": m.value}


def fdetd_host_plan_digest(Nz, Nr, modes, order, dz, dr, dt):
    """Host only: per-mode left-to-right sums (PE, PB, QE, QB, lambda, mu) of a multi-mode plan's host tables."""
    m = (ctypes.c_int * len(modes))(*modes)
    out = np.zeros(6 * len(modes))
    _check(lib().fdetd_host_plan_digest(Nz, Nr, m, len(modes), order, dz, dr, dt, _dptr(out)))
    return out.reshape(len(modes), 6)


def fdetd_host_split_parts(sizes, parts):
    """Host only: the part of each item in the host-buffer batch step's split of `sizes` into `parts`."""
    n = len(sizes)
    b = (ctypes.c_size_t * max(n, 1))(*[int(x) for x in sizes])
    out = (ctypes.c_int * max(n, 1))()
    r = lib().fdetd_host_split_parts(b, n, int(parts), out)
    if r < 0:
        _check(-r)
    return [out[k] for k in range(n)], r


def fdetd_host_coeffs(kind, order):
    buf = np.zeros(64)
    n = lib().fdetd_host_coeffs(kind, order, _dptr(buf))
    if n < 0:
        _check(n)
    return buf[:n].copy()


class EnvelopePlan:
    def __init__(self, handle, Nz, Nr, order, taylor_order, dz, dr, dt, k0):
        self.handle = handle
        self.Nz, self.Nr, self.order, self.taylor_order = Nz, Nr, order, taylor_order
        self.dz, self.dr, self.dt, self.k0 = dz, dr, dt, k0

    @property
    def launches_per_step(self):
        return lib().envelope_plan_launches_per_step(self.handle)

    @property
    def device_bytes(self):
        return lib().envelope_plan_device_bytes(self.handle)

    def close(self):
        if self.handle:
            lib().envelope_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def envelope_plan(Nz, Nr, order, taylor_order, dz, dr, dt, k0=2 * np.pi):
    h = ctypes.c_void_p()
    _check(lib().envelope_plan(ctypes.byref(h), Nz, Nr, order, taylor_order, dz, dr, dt, k0))
    return EnvelopePlan(h, Nz, Nr, order, taylor_order, dz, dr, dt, k0)


def envelope_step(plan, a, chi, nsteps=1, stream=None):
    """Advance psi_a = a[0] (a), a[1] (a~) in place: a cuda complex64 [2][Nz][Nr], chi float32 [Nz][Nr]."""
    import torch
    if not a.is_cuda or a.dtype != torch.complex64 or tuple(a.shape) != (2, plan.Nz, plan.Nr) or not a.is_contiguous():
        raise FdetdError("a must be a contiguous cuda complex64 tensor of shape (2, Nz, Nr)")
    if not chi.is_cuda or chi.dtype != torch.float32 or tuple(chi.shape) != (plan.Nz, plan.Nr) or not chi.is_contiguous():
        raise FdetdError("chi must be a contiguous cuda float32 tensor of shape (Nz, Nr)")
    _check(lib().envelope_step(plan.handle, a.data_ptr(), chi.data_ptr(), nsteps, _stream_handle(stream)))
    return a


def envelope_step_fused(plan, a, chi, nsteps=1, stream=None):
    """envelope_step with every Taylor term in one launch (order 8, N_T = 4, Nz a multiple of 32)."""
    import torch
    if not a.is_cuda or a.dtype != torch.complex64 or tuple(a.shape) != (2, plan.Nz, plan.Nr) or not a.is_contiguous():
        raise FdetdError("a must be a contiguous cuda complex64 tensor of shape (2, Nz, Nr)")
    if not chi.is_cuda or chi.dtype != torch.float32 or tuple(chi.shape) != (plan.Nz, plan.Nr) or not chi.is_contiguous():
        raise FdetdError("chi must be a contiguous cuda float32 tensor of shape (Nz, Nr)")
    _check(lib().envelope_step_fused(plan.handle, a.data_ptr(), chi.data_ptr(), nsteps, _stream_handle(stream)))
    return a


def envelope_step_absorbing(plan, a, chi, sigma, nsteps=1, stream=None):
    """Envelope step with the split-operator absorbing layer (see include/fdetd.h); sigma float32 [Nz][Nr]."""
    import torch
    if not a.is_cuda or a.dtype != torch.complex64 or tuple(a.shape) != (2, plan.Nz, plan.Nr) or not a.is_contiguous():
        raise FdetdError("a must be a contiguous cuda complex64 tensor of shape (2, Nz, Nr)")
    for name, t in (("chi", chi), ("sigma", sigma)):
        if not t.is_cuda or t.dtype != torch.float32 or tuple(t.shape) != (plan.Nz, plan.Nr) or not t.is_contiguous():
            raise FdetdError(f"{name} must be a contiguous cuda float32 tensor of shape (Nz, Nr)")
    _check(lib().envelope_step_absorbing(plan.handle, a.data_ptr(), chi.data_ptr(), sigma.data_ptr(), nsteps,
                                         _stream_handle(stream)))
    return a


def envelope_step_static(a, chi, order, taylor_order, dz, dr, dt, k0=2 * np.pi, nsteps=1, stream=None):
    """Allocation-free envelope step (see include/fdetd.h): same arguments as a plan plus step."""
    import torch
    if not a.is_cuda or a.dtype != torch.complex64 or a.dim() != 3 or a.shape[0] != 2 or not a.is_contiguous():
        raise FdetdError("a must be a contiguous cuda complex64 tensor of shape (2, Nz, Nr)")
    Nz, Nr = a.shape[1], a.shape[2]
    if not chi.is_cuda or chi.dtype != torch.float32 or tuple(chi.shape) != (Nz, Nr) or not chi.is_contiguous():
        raise FdetdError("chi must be a contiguous cuda float32 tensor of shape (Nz, Nr)")
    rc = lib().envelope_step_static(a.data_ptr(), chi.data_ptr(), Nz, Nr, order, taylor_order, dz, dr, dt, k0,
                                    nsteps, _stream_handle(stream))
    if rc != 0:
        raise FdetdError(f"envelope_step_static error {rc}")
    return a


class FdetdBatch:
    """Uneven instances advanced together by one captured CUDA graph (see include/fdetd.h)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().fdetd_batch_create(ctypes.byref(h)))
        self.handle = h
        self._keep = []

    def add(self, plan, fields, J=None):
        _check_tensor(fields, plan, 6, "fields")
        jp = None
        if J is not None:
            _check_tensor(J, plan, 3, "J")
            jp = J.data_ptr()
        idx = ctypes.c_int(-1)
        _check(lib().fdetd_batch_add(self.handle, plan.handle, fields.data_ptr(), jp, ctypes.byref(idx)))
        self._keep.append((plan, fields, J))
        return idx.value

    def set_autotune(self, on=True):
        _check(lib().fdetd_batch_set_autotune(self.handle, int(on)))

    def capture(self, nsteps=1, stream=None):
        _check(lib().fdetd_batch_capture(self.handle, nsteps, _stream_handle(stream)))

    def groups(self):
        """Per tensor-core group after capture: the chosen tiles, sizes and tuned times."""
        out = []
        gi = 0
        while True:
            info = (ctypes.c_int * 7)()
            ms = (ctypes.c_double * 2)()
            ng = lib().fdetd_batch_group_info(self.handle, gi, info, ms)
            if ng < 0:
                _check(-ng)
            if gi >= ng:
                return out
            out.append({"tn_proj": info[0], "tn_back": info[1], "sched_proj": info[2], "sched_back": info[3],
                        "instances": info[4], "proj_tiles": info[5], "back_tiles": info[6],
                        "tuned_ms": (ms[0], ms[1])})
            gi += 1

    def launch(self, stream=None):
        _check(lib().fdetd_batch_launch(self.handle, _stream_handle(stream)))

    def set_wait_limit(self, polls=-1):
        """Polls before a tensor-core pipeline wait gives up (< 0: default; 0: at once, drives the timeout path)."""
        _check(lib().fdetd_plan_set_wait_limit(self.handle, int(polls)))

    def set_profiling(self, on=True):
        """Record stage-timing events into the graph at the next capture (drops the captured graph)."""
        _check(lib().fdetd_batch_set_profiling(self.handle, int(on)))

    def collect_stage_times(self):
        """Add the last completed replay's stage times to the running sums (caller synchronizes first)."""
        _check(lib().fdetd_batch_collect_stage_times(self.handle))

    def stage_times(self):
        """{'projection', 'spectral', 'backprojection'}: (summed ms, steps summed)."""
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_long(0)
        _check(lib().fdetd_batch_stage_times(self.handle, ms, ctypes.byref(n)))
        return {k: (ms[i], n.value) for i, k in enumerate(("projection", "spectral", "backprojection"))}

    def pipeline_waits(self):
        """Pipeline cycle counters of the grouped tensor-core kernels of a batch captured with profiling on."""
        out = (ctypes.c_uint64 * 24)()
        _check(lib().fdetd_batch_pipeline_waits(self.handle, out))
        return pipeline_report(list(out))

    def set_host_pipeline(self, parts):
        """Parts of the host-buffer step whose copies overlap each other's compute (1: serial form)."""
        _check(lib().fdetd_batch_set_host_pipeline(self.handle, int(parts)))

    def step_host(self, host_fields, host_J=None, nlaunch=1, stream=None):
        """Host-buffer form: copy every instance's fields (and J) in, replay the graph nlaunch times, copy the
        fields back into host_fields; host tensors in instance order (pinned for asynchronous copies)."""
        n = len(host_fields)
        hf = (ctypes.c_void_p * n)(*[t.data_ptr() for t in host_fields])
        hj = None
        if host_J is not None:
            hj = (ctypes.c_void_p * n)(*[None if t is None else t.data_ptr() for t in host_J])
        _check(lib().fdetd_batch_step_host(self.handle, hf, hj, nlaunch, _stream_handle(stream)))

    def close(self):
        if self.handle:
            lib().fdetd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
