"""Adjoint solve and receiver-misfit gradient w.r.t. m = 1/c^2 (oracle; test infrastructure only).

The discrete operator A(m) of ``helmholtz`` (J-multiplied PML form) is complex
symmetric, A^T = A, so A^H = conj(A) and  A^H lam = g  is solved as
lam = conj(A^{-1} conj(g))  -- the same solver (direct or DDM-preconditioned)
applied to conjugated data.

Loss for sources s and receivers r (full-grid node indices):
    L(m) = 1/2 sum_s sum_r |u_s(x_r) - d_{s,r}|^2,   A(m) u_s = J f_s.
With dA/dm_k = omega^2 J_k e_k e_k^T (only the mass term depends on m):
    dL/dm_k = -omega^2 sum_s Re( conj(lam_{s,k}) J_k u_{s,k} ),
    lam_s = A^{-H} P^T (P u_s - d_s).
The paper mentions this use (full waveform inversion, Remark 2) without
formulas; the gradient above is the definition of dL/dm, and tests pin it
with central finite differences.
"""
from __future__ import annotations

import numpy as np

from .helmholtz import global_operator


def receiver_values(u, receivers):
    """P u: (nsrc, nrec) samples of u (nsrc, *grid) at receiver index tuples (x, y[, z])."""
    idx = tuple(np.asarray(receivers)[:, a] for a in reversed(range(receivers.shape[1])))
    return u[(slice(None),) + idx]


def misfit(u, receivers, d):
    r = receiver_values(u, receivers) - d
    return 0.5 * float(np.sum(np.abs(r) ** 2))


def adjoint_source(u, receivers, d):
    """P^T (P u - d) on the full grid."""
    g = np.zeros_like(u)
    idx = tuple(np.asarray(receivers)[:, a] for a in reversed(range(receivers.shape[1])))
    g[(slice(None),) + idx] = receiver_values(u, receivers) - d
    return g


def adjoint_solve(solve, g):
    """lam = A^{-H} g = conj(A^{-1} conj(g)) given a solver u = solve(b) of A u = b."""
    return np.conj(solve(np.conj(g)))


def gradient(wl, u, lam, form="literal"):
    """dL/dm on the full grid from forward fields u and adjoint fields lam."""
    _, J = global_operator(wl, form)
    J = J.reshape(u.shape[1:])
    return -wl.omega ** 2 * np.sum(np.real(np.conj(lam) * J[None] * u), axis=0)
