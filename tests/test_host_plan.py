"""Host-side checks of the C-ABI library (no GPU): symbol exports, stencil coefficients and the
FP64 plan tables (radial eigenbases folded into projection matrices) against the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import maxwell as mx
from oracle import stencils as st

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

native = pytest.importorskip("paper_2605_12132_gb300._native")


def _lib_or_skip():
    try:
        return native.lib()
    except native.FdetdError as e:
        pytest.skip(str(e))


def test_library_exports_every_declared_symbol():
    L = _lib_or_skip()
    hdr = open(os.path.join(ROOT, "include", "fdetd.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"^\s*(?:int|size_t)\s+(\w+)\s*\(", hdr, flags=re.M))
    assert {"fdetd_plan", "fdetd_step", "envelope_step", "envelope_plan"} <= names
    for nm in sorted(names):
        assert hasattr(L, nm), nm
        assert ctypes.cast(getattr(L, nm), ctypes.c_void_p).value


@pytest.mark.parametrize("order", [2, 4, 8, 16, 24, 32])
def test_host_coefficients_match_oracle(order):
    _lib_or_skip()
    np.testing.assert_allclose(native.fdetd_host_coeffs(0, order), st.staggered_coeffs(order), rtol=2e-16, atol=0)
    np.testing.assert_allclose(native.fdetd_host_coeffs(1, order), st.centred_d1_coeffs(order), rtol=2e-16, atol=0)
    e0, e = st.centred_d2_coeffs(order)
    np.testing.assert_allclose(native.fdetd_host_coeffs(2, order), np.concatenate([[e0], e]), rtol=4e-16, atol=0)
    np.testing.assert_allclose(native.fdetd_host_coeffs(3, order), st.axis_coeffs(order // 2), rtol=2e-16, atol=0)


TAU = -1j


def _phase(w, t):
    with np.errstate(divide="ignore", invalid="ignore"):
        A1 = np.where(w * t > 1e-3, np.sin(w * t) / w, t * (1 - (w * t) ** 2 / 6))
        A2 = np.where(w * t > 1e-3, 2 * np.sin(w * t / 2) ** 2 / w ** 2, t * t / 2 * (1 - (w * t) ** 2 / 12))
    return A1, A2


def factorised_step(F, J, T, dt, nsteps):
    """The factorised exact step, written with the exported host tables (what the kernels compute)."""
    n = F.shape[2]
    G = F.copy()
    for f in (1, 3, 5):
        G[f] = TAU * G[f]
    JJ = J.copy()
    JJ[1] = TAU * JJ[1]
    sp, sm, k2 = T["sp"][:, None], T["sm"][:, None], T["kappa2"][:, None]
    for _ in range(nsteps):
        cE = np.concatenate([G[0], G[1], G[2]], axis=1) @ T["PE"].T
        cB = np.concatenate([G[4], G[3], G[5]], axis=1) @ T["PB"].T
        cJ = np.concatenate([JJ[0], JJ[1], JJ[2]], axis=1) @ T["PE"].T
        cE, cB, cJ = (np.fft.fft(c, axis=0) for c in (cE, cB, cJ))
        e, a, c = cE[:, :n], cE[:, n:2 * n], cE[:, 2 * n:]
        b, d, f = cB[:, :n], cB[:, n:2 * n], cB[:, 2 * n:]
        eJ, aJ, cJ_ = cJ[:, :n], cJ[:, n:2 * n], cJ[:, 2 * n:]
        lam = T["lam"][None, :]
        w = np.sqrt(k2 + lam)
        A1, A2 = _phase(w, dt)
        B1, B2 = _phase(w, dt / 2)
        live = T["tm_live"][None, :] > 0
        A1, A2, B1, B2 = (np.where(live, x, 0) for x in (A1, A2, B1, B2))
        Mtm = lambda x: (-lam * x[2], -sp * x[2], x[0] - sm * x[1])

        def upd(x, xJ, M):
            y, z, yJ, zJ = M(x), M(M(x)), M(xJ), M(M(xJ))
            return tuple(x[i] + A1 * y[i] + A2 * z[i] - dt * (xJ[i] + B1 * yJ[i] + B2 * zJ[i]) for i in range(3))

        e, a, b = upd((e, a, b), (eJ, aJ, 0 * eJ), Mtm)
        mu = T["mu"][None, :]
        w = np.sqrt(k2 + mu)
        A1, A2 = _phase(w, dt)
        B1, B2 = _phase(w, dt / 2)
        live = T["te_live"][None, :] > 0
        A1, A2, B1, B2 = (np.where(live, x, 0) for x in (A1, A2, B1, B2))
        Mte = lambda x: (-sp * x[1] + x[2], -sm * x[0], -mu * x[0])
        c, d, f = upd((c, d, f), (cJ_, 0 * cJ_, 0 * cJ_), Mte)
        XE = np.fft.ifft(np.concatenate([e, a, c], axis=1), axis=0) @ T["QE"].T
        XB = np.fft.ifft(np.concatenate([b, d, f], axis=1), axis=0) @ T["QB"].T
        G = np.zeros_like(G)
        G[0], G[1], G[2] = XE[:, :n], XE[:, n:2 * n], XE[:, 2 * n:]
        G[4], G[3], G[5] = XB[:, :n], XB[:, n:2 * n], XB[:, 2 * n:]
    for f in (1, 3, 5):
        G[f] = G[f] / TAU
    return G


@pytest.mark.parametrize("m", [0, 1, 2, 3])
@pytest.mark.parametrize("order", [4, 8])
def test_host_tables_reproduce_oracle_step(m, order):
    _lib_or_skip()
    rng = np.random.default_rng(20 + m + order)
    Nz, Nr, dz, dr, dt = 16, 13, 1 / 16, 1 / 4, 1 / 16
    F = rng.standard_normal((6, Nz, Nr)) + 1j * rng.standard_normal((6, Nz, Nr))
    J = rng.standard_normal((3, Nz, Nr)) + 1j * rng.standard_normal((3, Nz, Nr))
    T = native.fdetd_host_tables(Nz, Nr, m, order, dz, dr, dt)
    got = factorised_step(F, J, T, dt, 3)
    ref = mx.step_spectral(F, J, Nz, Nr, m, order, dz, dr, dt, nsteps=3)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_host_tables_full_size_structure():
    # order 16, Nr = 256 (the 2048 x 256 workload): real spectra, bounded tables
    _lib_or_skip()
    for m in (0, 1):
        T = native.fdetd_host_tables(64, 256, m, 16, 1 / 16, 1 / 4, 1 / 16)
        assert (T["lam"] >= 0).all() and (T["mu"] >= 0).all()
        assert T["tm_live"].sum() == 256 - (m == 0)
        assert T["te_live"].sum() == 255 + (m == 0)
        for k in ("PE", "PB", "QE", "QB"):
            assert np.isfinite(T[k]).all() and np.abs(T[k]).max() < 100


def test_plan_errors_are_reported():
    _lib_or_skip()
    with pytest.raises(native.FdetdError, match="order"):
        native.fdetd_host_tables(16, 8, 0, 7, 0.1, 0.1, 0.1)
    with pytest.raises(native.FdetdError):
        native.fdetd_host_tables(16, 3, 0, 8, 0.1, 0.1, 0.1)


def _dense_from_bands(band, order):
    n = band.shape[0]
    ND = order // 2
    A = np.zeros((n, n))
    for k in range(n):
        for t in range(2 * ND + 1):
            j = k - ND + t
            if 0 <= j < n:
                A[k, j] = band[k, t]
    return A


@pytest.mark.parametrize("m", [0, 1, 2, 3])
@pytest.mark.parametrize("order", [4, 8, 16])
def test_taylor_bands_reproduce_oracle_radial_operators(m, order):
    """The banded operators of the Taylor stepper are the oracle's radial blocks of H (Sec. 2.5)."""
    _lib_or_skip()
    Nr, dr = 23, 0.25
    rad = mx.Radial(Nr, order, dr, m)
    bands, axis = native.fdetd_taylor_host_bands(Nr, order, dr, m)
    dense = [_dense_from_bands(bands[b], order) for b in range(4)]
    # band 0 acts on B_z slots 1.. with the axis value folded in: D^+ X0
    A0 = rad.Dp @ rad.X0
    assert np.allclose(dense[0][:, 1:], A0, atol=1e-12 * np.abs(A0).max()) and np.all(dense[0][:, 0] == 0)
    A1 = rad.Dp * rad.rhom[None, :] / rad.rho[:, None]
    assert np.allclose(dense[1], A1, atol=1e-12 * np.abs(A1).max())
    A2 = rad.Dm.copy()
    A2[0] = 0
    assert np.allclose(dense[2], A2, atol=1e-12 * np.abs(A2).max())
    A3 = np.zeros_like(rad.Dm)
    A3[1:] = rad.Dm[1:] * rad.rho[None, :] / rad.rhom[1:, None]
    assert np.allclose(dense[3], A3, atol=1e-12 * np.abs(A3).max())
    ND = order // 2
    assert np.allclose(axis[0], rad.axis_polar[:ND]) and np.all(rad.axis_polar[ND:] == 0)
    assert np.allclose(axis[1], rad.axis_scalar[:ND]) and np.all(rad.axis_scalar[ND:] == 0)


def _dif_model(x, rad):
    """In-place decimation-in-frequency FFT with the given stage radices (numpy model of the spectral kernels'
    stage structure): returns the array of output positions and the last stage's radix."""
    N = len(x)
    assert int(np.prod(rad)) == N
    y = x.astype(complex).copy()
    M = N
    for R in rad:
        L = M // R
        for blk in range(N // M):
            for n1 in range(L):
                idx = blk * M + n1 + L * np.arange(R)
                v = np.fft.fft(y[idx])
                v[1:] *= np.exp(-2j * np.pi * n1 * np.arange(1, R) / M)
                y[idx] = v
        M = L
    return y, rad[-1]


@pytest.mark.parametrize("Nz", [2, 4, 8, 16, 64, 128, 512, 1024, 2048, 4096, 96, 576, 640, 960, 1344, 3136, 4032])
@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_spectral_table_order_is_the_transform_output_order(Nz, prec):
    # the per-kz tables must list, entry by entry, the kz the in-place forward transform leaves at the
    # position that reads the entry: position b RL + r reads entry r (Nz / RL) + b
    _lib_or_skip()
    kz = native.fdetd_host_spectral_order(Nz, prec)
    assert sorted(kz.tolist()) == list(range(Nz))
    rad = native.fdetd_host_spectral_radices(Nz, prec)
    assert int(np.prod(rad)) == Nz and all(r in (2, 3, 4, 5, 7, 8) for r in rad)
    x = np.random.default_rng(Nz).standard_normal(Nz) + 1j * np.random.default_rng(Nz + 1).standard_normal(Nz)
    y, RL = _dif_model(x, rad)
    X = np.fft.fft(x)
    nb = Nz // RL
    for i in range(Nz):
        p = (i % nb) * RL + i // nb
        assert abs(y[p] - X[kz[i]]) < 1e-9 * np.abs(X).max(), (i, p, kz[i])


def test_spectral_radices_reject_large_prime_factors():
    _lib_or_skip()
    assert native.fdetd_host_spectral_radices(4093, "bf16x6") == []
    assert native.fdetd_host_spectral_radices(64 * 11, "fp32") == []
    assert native.fdetd_host_spectral_radices(4096, "fp32") == [8, 8, 8, 8]
    assert native.fdetd_host_spectral_radices(4096, "fp64") == [4] * 6


def test_radial_table_cache_returns_the_same_tables_and_honours_its_limit():
    # the radial tables depend on (Nr, order, dr, m) only: a second plan with another Nz and dt is a hit and its
    # tables are bitwise those of a fresh build; limit 0 empties and disables the cache
    _lib_or_skip()
    native.fdetd_plan_cache_set_limit(0)
    native.fdetd_plan_cache_set_limit(1 << 30)
    s0 = native.fdetd_plan_cache_stats()
    assert s0["bytes"] == 0 and s0["entries"] == 0 and s0["limit"] == 1 << 30
    a = native.fdetd_host_tables(16, 40, 1, 8, 1 / 16, 1 / 4, 1 / 16)
    s1 = native.fdetd_plan_cache_stats()
    assert s1["misses"] == s0["misses"] + 1 and s1["entries"] == 1
    assert s1["bytes"] >= 4 * (3 * 40) ** 2 * 8
    b = native.fdetd_host_tables(32, 40, 1, 8, 1 / 8, 1 / 4, 1 / 32)
    s2 = native.fdetd_plan_cache_stats()
    assert s2["hits"] == s1["hits"] + 1 and s2["misses"] == s1["misses"]
    for k in ("PE", "PB", "QE", "QB", "lam", "mu", "tm_live", "te_live"):
        assert np.array_equal(a[k], b[k]), k
    # a different dr, m or order is a different key
    native.fdetd_host_tables(16, 40, 1, 8, 1 / 16, 1 / 5, 1 / 16)
    native.fdetd_host_tables(16, 40, 2, 8, 1 / 16, 1 / 4, 1 / 16)
    native.fdetd_host_tables(16, 40, 1, 4, 1 / 16, 1 / 4, 1 / 16)
    s3 = native.fdetd_plan_cache_stats()
    assert s3["misses"] == s2["misses"] + 3 and s3["entries"] == 4
    # a limit that holds about two entries evicts the least recently used ones
    one = s1["bytes"]
    native.fdetd_plan_cache_set_limit(2 * one + one // 2)
    s4 = native.fdetd_plan_cache_stats()
    assert s4["entries"] == 2 and s4["bytes"] <= 2 * one + one // 2
    native.fdetd_plan_cache_set_limit(0)
    c = native.fdetd_host_tables(16, 40, 1, 8, 1 / 16, 1 / 4, 1 / 16)
    s5 = native.fdetd_plan_cache_stats()
    assert s5["entries"] == 0 and s5["misses"] == s4["misses"] + 1
    for k in ("PE", "PB", "QE", "QB", "lam", "mu"):
        assert np.array_equal(a[k], c[k]), k
    native.fdetd_plan_cache_set_limit(4 << 30)


def test_host_step_split_is_contiguous_ordered_and_balanced():
    # the split of the host-buffer batch step: contiguous parts in instance order, none empty, at most
    # min(parts, n), each closing at the first item that reaches its share of the total bytes
    _lib_or_skip()
    rng = np.random.default_rng(5)
    cases = [[1000] * 64, list(rng.integers(1, 10 ** 6, 37)), [5, 10 ** 9, 3, 4, 7], [42], list(rng.integers(1, 100, 8))]
    for sizes in cases:
        for parts in (1, 2, 3, 8, 16, 100):
            part_of, nparts = native.fdetd_host_split_parts(sizes, parts)
            n = len(sizes)
            P = min(parts, n)
            assert 1 <= nparts <= P
            assert part_of[0] == 0 and part_of[-1] == nparts - 1
            assert all(b - a in (0, 1) for a, b in zip(part_of, part_of[1:]))      # contiguous, ordered
            total = sum(sizes)
            csum = np.cumsum(sizes)
            for p in range(nparts - 1):
                last = max(k for k in range(n) if part_of[k] == p)
                assert csum[last] * P >= total * (p + 1)                          # reached its share
                first = min(k for k in range(n) if part_of[k] == p)
                if first > 0 and last > first:
                    assert csum[last - 1] * P < total * (p + 1)                   # and closed at the first such item
    part_of, nparts = native.fdetd_host_split_parts([1000] * 64, 16)
    assert nparts == 16 and all(part_of.count(p) == 4 for p in range(16))
    assert native.fdetd_host_split_parts([], 4) == ([], 0)
    with pytest.raises(native.FdetdError):
        native.fdetd_host_split_parts([1, 2], 0)


def test_python_flag_and_precision_constants_match_the_header():
    hdr = open(os.path.join(ROOT, "include", "fdetd.h")).read()
    flags = dict((k, int(v)) for k, v in re.findall(r"#define (FDETD_FLAG_\w+) (\d+)ull", hdr))
    assert flags == {"FDETD_FLAG_SPECTRAL_COLUMNS": native.SPECTRAL_COLUMNS, "FDETD_FLAG_J_ON_PRIMARY": native.J_ON_PRIMARY}
    prec = dict((k.lower(), int(v)) for k, v in re.findall(r"FDETD_PREC_(\w+) = (\d+)", hdr))
    assert prec == native.PRECISIONS


def test_parallel_multi_mode_build_equals_single_mode_builds():
    # a plan builds its modes' radial eigenbases on parallel threads (and each mode's TM and TE bases on two):
    # every mode's tables must be bitwise those of a single-mode build, with the radial-table cache off (every
    # table built in the threads) and on
    _lib_or_skip()
    Nz, Nr, order, dz, dr, dt = 32, 40, 8, 1 / 16, 1 / 4, 1 / 16
    modes = [0, 1, 2, 3, 5]

    def seq_sum(x):
        return float(np.cumsum(np.asarray(x, dtype=np.float64).ravel())[-1])
    native.fdetd_plan_cache_set_limit(0)
    ref = []
    for m in modes:
        T = native.fdetd_host_tables(Nz, Nr, m, order, dz, dr, dt)
        ref.append([seq_sum(T[k]) for k in ("PE", "PB", "QE", "QB", "lam", "mu")])
    ref = np.array(ref)
    for limit in (0, 1 << 30):
        native.fdetd_plan_cache_set_limit(limit)
        for _ in range(2):
            got = native.fdetd_host_plan_digest(Nz, Nr, modes, order, dz, dr, dt)
            assert np.array_equal(got, ref), (limit, np.abs(got - ref).max())
    native.fdetd_plan_cache_set_limit(4 << 30)
    with pytest.raises(native.FdetdError):
        native.fdetd_host_plan_digest(Nz, Nr, [0, 70], order, dz, dr, dt)
