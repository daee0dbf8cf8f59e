"""Helpers shared by the GPU tests (error metric of the parity checks)."""
import numpy as np


def field_errors(got, ref, floor=1e-12):
    """Per-field relative L2 error ||X - X_ref|| / max(||X_ref||, floor ||Psi_ref||) of one mode.

    got, ref: [6][Nz][Nr].  floor = 1e-12 for the FP64 path (a field below 1e-12 of the
    state's norm, e.g. Ez, Bz early in a vacuum run, is measured against the state).  The
    reduced-precision paths use floor = 0.1: every output component mixes all components of
    its group through the radial transforms, so its absolute error scales with the state's
    norm, and a field carrying under 10% of that norm is measured against 10% of it.
    """
    tot = np.linalg.norm(ref)
    out = []
    for f in range(ref.shape[0]):
        den = max(np.linalg.norm(ref[f]), floor * tot)
        out.append(np.linalg.norm(got[f] - ref[f]) / den)
    return np.array(out)


def floor_for(prec):
    return 1e-12 if prec == "fp64" else 0.1


def zero_axis(F):
    """Zero the axis slot of the staggered-grid fields (not part of the state on input)."""
    F = F.copy()
    for f in (0, 4, 5):
        F[..., f, :, 0] = 0
    return F
