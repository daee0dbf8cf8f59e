"""Writes tests/golden/batch_instances_ref.npz: the FP64 oracle's sampled kz columns of the three parity
instances of the uneven mix (inputs.PARITY_INSTANCES) after 1 and 100 exact midpoint steps
(Eq. maxwellAM_solution2), for the parity of the batched launch (tests/test_gpu_batch.py).  Calls only the
oracle and the seeded input generator.

    python tests/golden/make_batch_instances.py      # a few minutes (dense (6 Nr - 3)^2 expm per column)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import maxwell as mx  # noqa: E402
from paper_2605_12132_gb300 import inputs  # noqa: E402

COUNTS = [1, 100]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_instances_ref.npz")


def sample_kz(Nz, seed):
    """kz = 0, the carrier kz = 2 pi (q = Nz dz) and one seeded column outside the pulse band."""
    rng = np.random.default_rng(seed)
    return [0, Nz // 16, int(rng.integers(Nz // 8, Nz // 2))]


def main():
    out = {}
    for k, c in enumerate(inputs.PARITY_INSTANCES):
        F, J = inputs.instance_inputs(c)
        qs = sample_kz(c["Nz"], c["seed"])
        ref = np.zeros((len(COUNTS), c["M"] + 1, len(qs), 6, c["Nr"]), complex)
        t0 = time.time()
        for m in range(c["M"] + 1):
            cols = mx.step_spectral(F[m], J[m], c["Nz"], c["Nr"], m, c["order"], 1 / 16, 1 / 4, 1 / 16,
                                    nsteps=COUNTS, kz_subset=qs, method="expm")
            for ci in range(len(COUNTS)):
                for kq, q in enumerate(qs):
                    ref[ci, m, kq] = cols[ci][q]
        out[f"ref{k}"] = ref
        out[f"qs{k}"] = np.array(qs)
        print(f"instance {k} {c}: {time.time() - t0:.0f} s", flush=True)
    np.savez(OUT, counts=np.array(COUNTS), **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
