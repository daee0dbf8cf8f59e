"""Writes tests/golden/sweep_8192x512_ref.npz: the FP64 oracle's sampled kz columns of the 8192 x 512 three-mode
current-driven workload after 1, 100 and 1000 exact midpoint steps (Eq. maxwellAM_solution2), for the long
precision sweep (tests/test_gpu_sweep_8192x512.py).  Calls only the oracle and the seeded input generator.

    python tests/golden/make_sweep_8192x512.py      # ~30 min on 16 cores (one dense 3069^2 expm per column)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import maxwell as mx  # noqa: E402
from paper_2605_12132_gb300 import inputs  # noqa: E402

COUNTS = [1, 100, 1000]
# q = Nz dz = 512 is the carrier kz = 2 pi; 480 lies inside the pulse band, 1 and 2800 outside it
QS = [512, 480, 1, 2800]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_8192x512_ref.npz")


def main():
    w = inputs.workload("sweep_m012_8192x512")
    F, J = inputs.workload_inputs(w)
    ref = np.zeros((len(COUNTS), len(w.modes), len(QS), 6, w.Nr), dtype=np.complex128)
    for i, m in enumerate(w.modes):
        t0 = time.time()
        cols = mx.step_spectral(F[i], J[i], w.Nz, w.Nr, m, w.order, w.dz, w.dr, w.dt, nsteps=COUNTS, kz_subset=QS,
                                method="expm")
        for c in range(len(COUNTS)):
            for k, q in enumerate(QS):
                ref[c, i, k] = cols[c][q]
        print(f"mode {m}: {time.time() - t0:.0f} s", flush=True)
    np.savez(OUT, ref=ref, counts=np.array(COUNTS), qs=np.array(QS), modes=np.array(w.modes))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
