"""GPU parity of the envelope Taylor propagator against the FP64 oracle (through the C-ABI)."""
import numpy as np
import pytest

from oracle import envelope as ev
from paper_2605_12132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402


def _gpu(a, at, chi, order, NT, dz, dr, dt, nsteps):
    Nz, Nr = a.shape
    plan = fd.envelope_plan(Nz, Nr, order, NT, dz, dr, dt)
    psi = torch.from_numpy(np.stack([a, at])).to(torch.complex64).cuda()
    c = torch.from_numpy(chi).to(torch.float32).cuda()
    fd.envelope_step(plan, psi, c, nsteps)
    torch.cuda.synchronize()
    out = psi.cpu().numpy().astype(np.complex128)
    return out[0], out[1]


def _rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


@pytest.mark.parametrize("NT", [1, 2, 4])
def test_envelope_small_random(NT):
    rng = np.random.default_rng(5)
    Nz, Nr, order, dz, dr, dt = 64, 40, 8, 0.2, 0.25, 0.05
    a = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    at = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    chi = 0.5 * rng.random((Nz, Nr))
    ga, gt = _gpu(a, at, chi, order, NT, dz, dr, dt, 3)
    ra, rt = ev.envelope_step(a, at, chi, order, NT, dz, dr, dt, nsteps=3)
    assert _rel(ga, ra) < 2e-6 and _rel(gt, rt) < 2e-6


def test_envelope_full_size():
    # The FP32 state a carries a rounding error of ~2^-24 |a| each step; the Laplacian (infinity
    # norm ||L|| = (|e0| + 2 sum|e_n|)(dr^-2 + dz^-2)) maps it into da~/dt, so after n steps the
    # a~ error is bounded by ~n dt ||L|| 2^-24 ||a|| (relative to ||a~||).
    from oracle.stencils import centred_d2_coeffs
    w = inputs.envelope_workload("envelope_4096x256")
    a, at, chi = inputs.envelope_inputs(w)
    nsteps = 3
    ga, gt = _gpu(a, at, chi, w.order, w.taylor_order, w.dz, w.dr, w.dt, nsteps)
    ra, rt = ev.envelope_step(a, at, chi, w.order, w.taylor_order, w.dz, w.dr, w.dt, nsteps=nsteps)
    e0, e = centred_d2_coeffs(w.order)
    Lnorm = (abs(e0) + 2 * np.abs(e).sum()) * (w.dr ** -2 + w.dz ** -2)
    tol_t = max(2e-6, nsteps * w.dt * Lnorm * 2.0 ** -24 * np.linalg.norm(ra) / np.linalg.norm(rt))
    assert _rel(ga, ra) < 2e-6
    assert _rel(gt, rt) < tol_t, (_rel(gt, rt), tol_t)


def test_envelope_argument_errors():
    with pytest.raises(fd.FdetdError):
        fd.envelope_plan(64, 40, 7, 4, 0.2, 0.25, 0.05)
    with pytest.raises(fd.FdetdError):
        fd.envelope_plan(64, 40, 8, 0, 0.2, 0.25, 0.05)
    plan = fd.envelope_plan(64, 40, 8, 4, 0.2, 0.25, 0.05)
    with pytest.raises(fd.FdetdError):
        fd.envelope_step(plan, torch.zeros((2, 64, 41), dtype=torch.complex64, device="cuda"),
                         torch.zeros((64, 41), device="cuda"))


def test_envelope_absorbing_layer_matches_oracle():
    rng = np.random.default_rng(9)
    Nz, Nr, order, NT, dz, dr, dt = 64, 40, 8, 4, 0.2, 0.25, 0.05
    a = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    at = rng.standard_normal((Nz, Nr)) + 1j * rng.standard_normal((Nz, Nr))
    chi = 0.5 * rng.random((Nz, Nr))
    z = np.arange(Nz) * dz
    sigma = np.repeat((3.0 * np.clip((z - 8.0) / 4.0, 0, None) ** 2)[:, None], Nr, axis=1)
    plan = fd.envelope_plan(Nz, Nr, order, NT, dz, dr, dt)
    psi = torch.from_numpy(np.stack([a, at])).to(torch.complex64).cuda()
    c = torch.from_numpy(chi).to(torch.float32).cuda()
    s = torch.from_numpy(sigma).to(torch.float32).cuda()
    fd.envelope_step_absorbing(plan, psi, c, s, 3)
    torch.cuda.synchronize()
    out = psi.cpu().numpy().astype(np.complex128)
    ra, rt = ev.envelope_step_absorbing(a, at, chi, sigma.astype(np.float32).astype(np.float64), order, NT, dz, dr,
                                        dt, nsteps=3)
    assert _rel(out[0], ra) < 2e-6 and _rel(out[1], rt) < 2e-6


@pytest.mark.parametrize("nsteps", [1, 2, 5])
def test_fused_envelope_equals_term_by_term_launches(nsteps):
    # the all-terms-in-one-launch step (order 8, N_T = 4) does the term-by-term arithmetic cell for cell, so
    # the two agree bit for bit; odd and even step counts (the state alternates with a plan buffer), a ragged
    # radial tile (Nr = 200) and the periodic z halo
    rng = np.random.default_rng(40 + nsteps)
    Nz, Nr = 256, 200
    a = rng.standard_normal((2, Nz, Nr)) + 1j * rng.standard_normal((2, Nz, Nr))
    chi = 0.3 * rng.random((Nz, Nr))
    plan = fd.envelope_plan(Nz, Nr, 8, 4, 0.2, 0.25, 0.05)
    c = torch.from_numpy(chi).float().cuda()
    x = torch.from_numpy(a).to(torch.complex64).cuda()
    y = x.clone()
    fd.envelope_step_fused(plan, x, c, nsteps)
    fd.envelope_step(plan, y, c, nsteps)
    torch.cuda.synchronize()
    assert torch.equal(x, y)
