"""Long z columns against the oracle on sampled kz columns, with and without a current: the two-kernel spectral
paths (the current's source term transformed first, then the field columns alone) of the power-of-two transform
(Nz = 8192; FP64 at 4096) and of the mixed-radix transform (FP64 at 3136 = 7^2 64 and 4032 = 7 3^2 64), and the
fused mixed-radix kernel at long non-power-of-two lengths (3840, 2880)."""
import numpy as np
import pytest

from oracle import maxwell as mx
from paper_2605_12132_gb300 import inputs
from tests.gpu_util import check_report, column_report, format_report, kz_columns, zero_axis

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

# per-step tolerance of the fields with >= 10% of the state, and the bound of the weak fields (relative L2
# per field, floor 1e-12 of the state's norm)
TOL = {"fp64": 1e-12, "fp32": 1e-6, "bf16x6": 4e-6, "bf16x3": 2.5e-5}
TOL_WEAK = {"fp64": 1e-11, "fp32": 3e-5, "bf16x6": 3e-5, "bf16x3": 1e-3}


@pytest.mark.parametrize("prec,Nz", [("fp32", 8192), ("bf16x3", 8192), ("bf16x6", 8192), ("fp64", 4096),
                                     ("fp64", 4032), ("fp64", 3136), ("bf16x6", 3840), ("fp32", 2880)])
@pytest.mark.parametrize("with_J", [True, False])
def test_long_z_sampled_kz(prec, Nz, with_J):
    rng = np.random.default_rng(Nz + with_J)
    Nr, modes, order, dz, dr, dt = 48, [0, 1], 16, 1 / 16, 1 / 4, 1 / 16
    F = np.zeros((2, 6, Nz, Nr), complex)
    F[1] = inputs.pulse_fields(Nz, Nr, dz, dr, 3.0, 8.0)
    F += 1e-3 * (rng.standard_normal(F.shape) + 1j * rng.standard_normal(F.shape))
    F = zero_axis(F)
    J = np.stack([inputs.random_current(Nz, Nr, m, 8.0, 1e-2, 3) for m in modes]) if with_J else None
    plan = fd.fdetd_plan_modes(Nz, Nr, modes, order, dz, dr, dt, precision=prec)
    f = torch.from_numpy(F).to(plan.complex_dtype).cuda()
    j = torch.from_numpy(J).to(plan.complex_dtype).cuda() if with_J else None
    nsteps = 2
    fd.fdetd_step(plan, f, j, nsteps)
    plan.status()
    G = f.cpu().numpy().astype(np.complex128)
    qs = [0, 1, Nz // 16, Nz // 2, int(rng.integers(2, Nz // 2))]
    for i, m in enumerate(modes):
        ref = mx.step_spectral(F[i], None if J is None else J[i], Nz, Nr, m, order, dz, dr, dt, nsteps=nsteps,
                               kz_subset=qs, method="expm")
        Gq = kz_columns(G[i], qs)
        rows = column_report([Gq[:, k, :] for k in range(len(qs))], [ref[q] for q in qs])
        label = f"{prec} Nz={Nz} J={with_J} m={m}"
        print("\n" + format_report(rows, label))
        check_report(rows, TOL[prec] * nsteps, TOL_WEAK[prec] * nsteps, label=label)
