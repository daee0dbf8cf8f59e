"""The current pipeline on the GPU against the oracle (Sec. 2.5 stagger, Sec. 3 planar current correction)."""
import numpy as np
import pytest

from oracle import current as cur

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

# FP32 inputs and outputs (divergence, solve and gradient in double-float arithmetic): a few e-7 relative;
# FP64 end to end
TOL = {"fp64": 1e-11, "fp32": 2e-6}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [4, 8, 16])
def test_current_pipeline_matches_oracle(prec, order):
    rng = np.random.default_rng(order)
    Nz, Nr, modes, dr = 64, 45, [0, 1, 2, 3], 0.25
    J = rng.standard_normal((4, 3, Nz, Nr)) + 1j * rng.standard_normal((4, 3, Nz, Nr))
    rho = rng.standard_normal((4, Nz, Nr)) + 1j * rng.standard_normal((4, Nz, Nr))
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, order, 1 / 16, dr, 1 / 16, precision=prec)
    dt = plan.complex_dtype
    j = torch.from_numpy(J).to(dt).cuda()
    r = torch.from_numpy(rho).to(dt).cuda()
    for call in range(2):        # the first call builds the operators, the second reuses them
        out = fd.fdetd_current_correct(plan, j, r).cpu().numpy().astype(np.complex128)
        Jin, rin = j.cpu().numpy().astype(np.complex128), r.cpu().numpy().astype(np.complex128)
        for i, m in enumerate(modes):
            ref, _ = cur.current_pipeline(Jin[i], rin[i], m, order, dr)
            for c in range(3):
                err = np.linalg.norm(out[i, c] - ref[c]) / np.linalg.norm(ref[c])
                assert err < TOL[prec], (call, m, c, err)


def test_current_pipeline_feeds_the_field_step():
    # a corrected current is a valid J for fdetd_step (layout, type) and the step runs on it
    Nz, Nr = 64, 32
    rng = np.random.default_rng(4)
    plan = fd.fdetd_plan(Nz, Nr, 1, 8, 1 / 16, 1 / 4, 1 / 16, precision="bf16x6")
    J = torch.from_numpy(rng.standard_normal((2, 3, Nz, Nr)) + 0j).to(torch.complex64).cuda()
    rho = torch.zeros((2, Nz, Nr), dtype=torch.complex64, device="cuda")
    Jc = fd.fdetd_current_correct(plan, J, rho)
    f = torch.zeros((2, 6, Nz, Nr), dtype=torch.complex64, device="cuda")
    fd.fdetd_step(plan, f, Jc, 2)
    plan.status()
    assert torch.isfinite(torch.view_as_real(f)).all()


def test_current_pipeline_rejects_aliasing():
    plan = fd.fdetd_plan(64, 16, 0, 4, 1 / 16, 1 / 4, 1 / 16, precision="fp32")
    J = torch.zeros((1, 3, 64, 16), dtype=torch.complex64, device="cuda")
    rho = torch.zeros((1, 64, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(fd.FdetdError):
        fd.fdetd_current_correct(plan, J, rho, J)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x6", 2e-6)])
def test_j_on_primary_flag_downstaggers_j_rho(prec, tol):
    # a plan with J_ON_PRIMARY stepping a current whose J_rho sits on the primary grid equals a plain plan
    # stepping the oracle's downstaggered current (S_rho^(-, mA) of Eq. spatialAM_staggerS); J is left as given
    from paper_2605_12132_gb300 import _native as nat
    from tests.gpu_util import zero_axis
    rng = np.random.default_rng(12)
    Nz, Nr, modes, order = 64, 40, [0, 1, 2], 8
    F = zero_axis(rng.standard_normal((3, 6, Nz, Nr)) + 1j * rng.standard_normal((3, 6, Nz, Nr)))
    J = rng.standard_normal((3, 3, Nz, Nr)) + 1j * rng.standard_normal((3, 3, Nz, Nr))
    Js = np.stack([np.stack([cur.s_rho_minus(J[i, 0], order, abs(m - 1) % 2 == 0), J[i, 1], J[i, 2]])
                   for i, m in enumerate(modes)])
    flagged = fd.fdetd_plan_modes(Nz, Nr, modes, order, 1 / 16, 1 / 4, 1 / 16, precision=prec,
                                  flags=nat.J_ON_PRIMARY)
    plain = fd.fdetd_plan_modes(Nz, Nr, modes, order, 1 / 16, 1 / 4, 1 / 16, precision=prec)
    dt = plain.complex_dtype
    j = torch.from_numpy(J).to(dt).cuda()
    j0 = j.clone()
    a = torch.from_numpy(F).to(dt).cuda()
    fd.fdetd_step(flagged, a, j, 2)
    flagged.status()
    assert torch.equal(j, j0)
    b = torch.from_numpy(F).to(dt).cuda()
    fd.fdetd_step(plain, b, torch.from_numpy(Js).to(dt).cuda(), 2)
    plain.status()
    err = (torch.linalg.vector_norm(a.to(torch.complex128) - b) / torch.linalg.vector_norm(b.to(torch.complex128)))
    assert float(err) < tol, float(err)
    # a batch takes J on the Yee locations: the flagged plan with a current is refused there
    batch = fd.FdetdBatch()
    with pytest.raises(fd.FdetdError):
        batch.add(flagged, a, j)
    batch.close()
