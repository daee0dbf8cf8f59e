"""FP64 CPU oracle for the cylindrical FDETD field update and the laser-envelope propagator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library, the
Python binding, the kernels) imports, links or executes anything in this
package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.

The oracle is a plain, slow, obviously-correct restatement of the method of
"High-order exponential solver method for particle-in-cell simulations in
cylindrical geometry" (Majorosi, Hafz, Lecz):

* ``stencils``   - exact rational finite-difference and axis coefficients
                   (Sec. 2.3 Eq. spatial_derivativeSt, Sec. 2.4 axis rule).
* ``maxwell``    - the discrete azimuthal-mode Maxwell operator of Sec. 2.5
                   (Eqs. spatialAM_maxwell_Er ... _Bz) assembled explicitly, and
                   three independent evaluators of the midpoint exponential step
                   of Sec. 2.1 (Eq. maxwellAM_solution2):
                   (i) per-kz dense eigendecomposition / dense expm,
                   (ii) brute-force expm of the whole real-space operator,
                   (iii) the paper's own truncated-Taylor FDETD (Sec. 2.5 summary).
* ``envelope``   - the discrete envelope operator H_a of Sec. 4.2
                   (Eq. spatialAM_envelope_H) and its Taylor propagator.
* ``diagnostics``- discrete energy, divergence (Eqs. spatialAM_divE) and the
                   pulse-energy / centroid diagnostics of Sec. 5.1.

Every function is FP64 (complex128) and cites the passage it follows.
"""
