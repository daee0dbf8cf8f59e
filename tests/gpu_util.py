"""Helpers shared by the GPU tests (error metric of the parity checks)."""
import numpy as np


def field_errors(got, ref):
    """Per-field relative L2 error ||X - X_ref|| / ||X_ref|| of one mode ([6][Nz][Nr]).

    A field whose reference norm is below 1e-12 of the whole state's norm (e.g. Ez, Bz
    early in a vacuum run) is measured against the whole state's norm instead.
    """
    tot = np.linalg.norm(ref)
    out = []
    for f in range(ref.shape[0]):
        nr = np.linalg.norm(ref[f])
        den = nr if nr >= 1e-12 * tot else tot
        out.append(np.linalg.norm(got[f] - ref[f]) / den)
    return np.array(out)


def zero_axis(F):
    """Zero the axis slot of the staggered-grid fields (not part of the state on input)."""
    F = F.copy()
    for f in (0, 4, 5):
        F[..., f, :, 0] = 0
    return F
