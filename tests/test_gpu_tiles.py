"""Tile shapes, schedules, the autotuner and grouped launches of the tensor-core radial transforms.

Every tile configuration sums each output over K in the same order, so results must be bitwise
identical across configurations, across grouped and single-instance launches, and after autotuning
(which must leave the caller's fields untouched)."""
import itertools

import numpy as np
import pytest

from oracle import maxwell as mx
from paper_2605_12132_gb300 import inputs
from tests.gpu_util import check_report, field_report, zero_axis

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

TOL = {"bf16x6": 1e-6, "bf16x3": 2.5e-5}


def _configs(prec, Nz):
    for tp, tb, sp, sb in itertools.product((128, 256), (128, 256), (0, 1), (0, 1)):
        if prec == "bf16x6" and tb != 128:
            continue
        if Nz % (tb // 2):
            continue
        yield (tp, tb, sp, sb)


def _case(seed, Nz, Nr, nm):
    rng = np.random.default_rng(seed)
    F = zero_axis(rng.standard_normal((nm, 6, Nz, Nr)) + 1j * rng.standard_normal((nm, 6, Nz, Nr)))
    J = 0.3 * (rng.standard_normal((nm, 3, Nz, Nr)) + 1j * rng.standard_normal((nm, 3, Nz, Nr)))
    return F, J


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_every_tile_config_gives_identical_bits(prec):
    # ragged everywhere: 100 radial points = 3 x 32 + 4 (projection K), 64 + 36 (back-projection K),
    # one partial 128-row tile; 3 modes, current on
    Nz, Nr, modes, order, dz, dr, dt = 256, 100, [0, 1, 2], 8, 1 / 16, 1 / 4, 1 / 16
    F, J = _case(3, Nz, Nr, len(modes))
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, order, dz, dr, dt, precision=prec)
    j = torch.from_numpy(J).to(torch.complex64).cuda()
    results = {}
    for cfg in _configs(prec, Nz):
        plan.tile_config = cfg
        assert plan.tile_config == cfg
        f = torch.from_numpy(F).to(torch.complex64).cuda()
        fd.fdetd_step(plan, f, j, 2)
        plan.status()
        results[cfg] = f.cpu()
    base = next(iter(results.values()))
    for cfg, r in results.items():
        assert torch.equal(r, base), cfg
    ref = np.stack([mx.step_spectral(F[i], J[i], Nz, Nr, m, order, dz, dr, dt, nsteps=2) for i, m in enumerate(modes)])
    got = base.numpy().astype(np.complex128)
    for i in range(len(modes)):
        rows = field_report(got[i], ref[i], nd=order // 2)
        check_report(rows, TOL[prec] * 2, TOL[prec] * 2, label=f"{prec} m={modes[i]}")


def test_invalid_tile_config_is_rejected():
    plan = fd.fdetd_plan(64, 32, 0, 4, 1 / 16, 1 / 4, 1 / 16, precision="bf16x6")
    with pytest.raises(fd.FdetdError):
        plan.tile_config = (256, 256, 0, 0)   # 3 pieces of a 256-wide back-projection tile
    with pytest.raises(fd.FdetdError):
        plan.tile_config = (192, 128, 0, 0)
    p3 = fd.fdetd_plan(64, 32, 0, 4, 1 / 16, 1 / 4, 1 / 16, precision="bf16x3")
    with pytest.raises(fd.FdetdError):
        p3.tile_config = (256, 256, 0, 0)     # Nz = 64 is not a multiple of 128 z per tile
    fp = fd.fdetd_plan(64, 32, 0, 4, 1 / 16, 1 / 4, 1 / 16, precision="fp32")
    with pytest.raises(fd.FdetdError):
        fp.tile_config


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_autotune_reads_only_and_keeps_results(prec):
    Nz, Nr, modes, order, dz, dr, dt = 512, 128, [0, 1], 16, 1 / 16, 1 / 4, 1 / 16
    F, J = _case(5, Nz, Nr, len(modes))
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, order, dz, dr, dt, precision=prec)
    f = torch.from_numpy(F).to(torch.complex64).cuda()
    j = torch.from_numpy(J).to(torch.complex64).cuda()
    f0, j0 = f.clone(), j.clone()
    ref = f.clone()
    fd.fdetd_step(plan, ref, j, 1)
    tp, tb = plan.autotune(f, j)
    torch.cuda.synchronize()
    assert tp > 0 and tb > 0
    assert torch.equal(f, f0) and torch.equal(j, j0)
    assert plan.tile_config in set(_configs(prec, Nz))
    fd.fdetd_step(plan, f, j, 1)
    plan.status()
    assert torch.equal(f, ref)


def test_autotune_is_a_noop_on_cuda_core_plans():
    plan = fd.fdetd_plan(64, 32, 0, 4, 1 / 16, 1 / 4, 1 / 16, precision="fp32")
    f = torch.zeros((1, 6, 64, 32), dtype=torch.complex64, device="cuda")
    assert plan.autotune(f) == (0.0, 0.0)


def _instances(seed, count, precs):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        prec = precs[k % len(precs)]
        Nz = int(rng.choice([64, 128, 256, 512]))
        Nr = int(rng.integers(8, 100)) * 2
        M = int(rng.integers(1, 4))
        order = int(rng.choice([8, 16]))
        F = np.zeros((M + 1, 6, Nz, Nr), complex)
        F[1] = inputs.pulse_fields(Nz, Nr, 1 / 16, 1 / 4, float(rng.uniform(10, 40)) * 0.25, 2.0)
        for f in (0, 4, 5):
            F[:, f, :, 0] = 0
        J = None
        if k % 3 != 2:
            J = np.stack([inputs.random_current(Nz, Nr, m, 4.0, 1e-2, seed + k) for m in range(M + 1)])
        out.append((fd.fdetd_plan(Nz, Nr, M, order, 1 / 16, 1 / 4, 1 / 16, precision=prec), F, J))
    return out


@pytest.mark.parametrize("autotune", [True, False])
def test_grouped_batch_mixed_precisions_matches_single_steps(autotune):
    inst = _instances(11, 9, ["bf16x3", "bf16x6", "fp32"])
    batch = fd.FdetdBatch()
    batch.set_autotune(autotune)
    tensors = []
    for plan, F, J in inst:
        f = torch.from_numpy(F).to(torch.complex64).cuda()
        j = torch.from_numpy(J).to(torch.complex64).cuda() if J is not None else None
        tensors.append((f, j))
        batch.add(plan, f, j)
    batch.capture(2)
    groups = batch.groups()
    assert len(groups) == 2 and sorted(g["instances"] for g in groups) == [3, 3]
    for g in groups:
        assert g["proj_tiles"] > 0 and g["back_tiles"] > 0
        assert (min(g["tuned_ms"]) > 0) == autotune
    batch.launch()
    batch.launch()
    torch.cuda.synchronize()
    for (plan, F, J), (f, j) in zip(inst, tensors):
        ref = torch.from_numpy(F).to(torch.complex64).cuda()
        jr = torch.from_numpy(J).to(torch.complex64).cuda() if J is not None else None
        fd.fdetd_step(plan, ref, jr, 4)
        plan.status()
        torch.cuda.synchronize()
        assert torch.equal(ref, f)


def test_more_instances_than_one_group_holds():
    # 70 tiny tensor-core instances: two groups (64 + 6) of one precision
    inst = []
    batch = fd.FdetdBatch()
    batch.set_autotune(False)
    rng = np.random.default_rng(2)
    for _ in range(70):
        plan = fd.fdetd_plan(64, 8, 0, 4, 1 / 16, 1 / 4, 1 / 16, precision="bf16x3")
        F = zero_axis(rng.standard_normal((1, 6, 64, 8)) + 1j * rng.standard_normal((1, 6, 64, 8)))
        f = torch.from_numpy(F).to(torch.complex64).cuda()
        batch.add(plan, f)
        inst.append((plan, F, f))
    batch.capture(1)
    assert [g["instances"] for g in batch.groups()] == [64, 6]
    batch.launch()
    torch.cuda.synchronize()
    for plan, F, f in inst[::7]:
        ref = torch.from_numpy(F).to(torch.complex64).cuda()
        fd.fdetd_step(plan, ref, None, 1)
        torch.cuda.synchronize()
        assert torch.equal(ref, f)
