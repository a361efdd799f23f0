"""Helpers shared by the GPU tests (no method arithmetic).

Every parity check compares two vectors twice:
* norm-wise, |y - ref|_2 / |ref|_2 < l2, the benchmark spec's matvec and energy
  gates (1e-5 against the oracle);
* element-wise, max_i |y_i - ref_i| / max_i |ref_i| < inf, by default
  3 x l2.  The FMM truncation at p = 10 leaves at most 2e-5 of the largest
  entry on any single row of the product (4e-6 at p >= 12), while a wrong
  leaf, interaction-list entry or near-singular table entry moves a row by
  1e-3 of the largest entry or more, far above the bound.
"""
import numpy as np

INF_FACTOR = 3.0


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def relmax(a, b):
    """max_i |a_i - b_i| / max_i |b_i|"""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.abs(a - b).max() / np.abs(b).max())


def close(a, b, l2, inf=None, what=""):
    """Assert both the norm-wise and the element-wise relative error bounds;
    returns (l2 error, max error)."""
    if inf is None:
        inf = INF_FACTOR * l2
    e2, ei = rel(a, b), relmax(a, b)
    assert e2 < l2, f"{what} relative L2 error {e2:.3e} >= {l2:.1e} (max error {ei:.3e})"
    assert ei < inf, f"{what} relative max error {ei:.3e} >= {inf:.1e} (L2 error {e2:.3e})"
    return e2, ei


def smooth_density(P):
    """A smooth surface density: the oracle's own normal field of the charges."""
    return P.bq()
