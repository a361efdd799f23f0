"""Helpers shared by the GPU tests (no method arithmetic)."""
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def smooth_density(P):
    """A smooth surface density: the oracle's own normal field of the charges."""
    return P.bq()
