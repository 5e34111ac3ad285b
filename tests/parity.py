"""The parity rule between the CUDA library and the FP64 oracle.

Assignments: the GPU must equal the oracle except at points whose FP64 top-2
squared-distance gap is below 1e-6 * (||x||^2 + ||c||^2) (near-ties, where the
FP32 scan may legitimately pick the other centroid); those are counted and
reported.  Centroids: within 1e-5 relative (per coordinate, against the
larger of |c| and 1e-6 of the centroid set's largest coordinate).
"""
import numpy as np

import oracle

ASSIGN_GAP_REL = 1e-6
CENTROID_REL = 1e-5


def check_assignments(X, C64, a_gpu, label=""):
    """Oracle assignment from the GPU's centroids (teacher forcing) vs the
    GPU's assignment.  Returns the number of exempt near-tie mismatches."""
    a_or, d1, d2, sc = oracle.assign(X, C64)
    mism = np.asarray(a_gpu) != a_or
    tie = oracle.near_tie_mask(d1, d2, sc, ASSIGN_GAP_REL)
    bad = mism & ~tie
    assert not bad.any(), (f"{label}: {int(bad.sum())} non-near-tie assignment mismatches, first at "
                           f"{np.flatnonzero(bad)[:5]} (gpu {np.asarray(a_gpu)[bad][:5]}, oracle {a_or[bad][:5]})")
    return int((mism & tie).sum())


def check_centroids(C_gpu, C_ref, label=""):
    C_gpu = np.asarray(C_gpu, np.float64)
    C_ref = np.asarray(C_ref, np.float64)
    scale = max(float(np.abs(C_ref).max()), 1e-30)
    tol = CENTROID_REL * np.maximum(np.abs(C_ref), 1e-6 * scale)
    err = np.abs(C_gpu - C_ref)
    assert np.all(err <= tol), f"{label}: centroid error {float((err / tol).max()):.3g} x tolerance"
    return float((err / np.maximum(np.abs(C_ref), 1e-6 * scale)).max())
