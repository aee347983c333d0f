"""Element-wise comparison of a GPU result with the oracle's, right-hand side
by right-hand side (shared by the GPU parity tests).

For every right-hand side r two figures are checked:
  * the relative L2 error  |u_r - ref_r| / |ref_r|;
  * the relative max error max_k |u_r[k] - ref_r[k]| / max_k |ref_r[k]|, which
    a wrong value at a few nodes (a transfer strip, a corner, one subdomain's
    seam) cannot hide under, as it could under a norm over the whole output.
"""
import numpy as np


def per_rhs_errors(u, ref):
    u = np.asarray(u).reshape(np.shape(u)[0], -1)
    ref = np.asarray(ref).reshape(np.shape(ref)[0], -1)
    l2 = [float(np.linalg.norm(u[r] - ref[r]) / np.linalg.norm(ref[r])) for r in range(ref.shape[0])]
    mx = [float(np.abs(u[r] - ref[r]).max() / np.abs(ref[r]).max()) for r in range(ref.shape[0])]
    return l2, mx


def assert_close(u, ref, tol_l2, tol_max, what=""):
    """Every right-hand side within tol_l2 (relative L2) and tol_max (relative
    max); returns the worst pair for reporting."""
    l2, mx = per_rhs_errors(u, ref)
    assert max(l2) <= tol_l2, (what, "rel L2 per RHS", l2, tol_l2)
    assert max(mx) <= tol_max, (what, "rel max per RHS", mx, tol_max)
    return max(l2), max(mx)
