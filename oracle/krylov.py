"""Right-preconditioned restarted GMRES in float64 (oracle; test infrastructure only).

Remark 1 (Section 4): the diagonal sweeping DDM is used as a preconditioner of
GMRES for the global discrete system; the paper stops at a relative residual of
1e-6 (Section 5.2).  The paper does not say left or right preconditioning or
whether GMRES restarts; we read it as right preconditioning (so the residual
monitored is the true residual of A u = J f) with restart length ``restart``.

This is the flexible form (the preconditioned directions z_k = M v_k are kept,
x = x0 + Z y), which equals plain right-preconditioned GMRES for a linear M.
Arnoldi uses modified Gram-Schmidt; the small least-squares problems are
solved with numpy.linalg.lstsq.  Every right-hand side has its own Krylov
space; the loop is vectorised over right-hand sides only.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    """Per-RHS <a, b> = sum conj(a) b over the grid axes."""
    return np.sum(np.conj(a) * b, axis=tuple(range(1, a.ndim)))


def _norm(a):
    return np.sqrt(np.real(_dot(a, a)))


def gmres(apply_A, b, apply_M, rtol=1e-6, restart=30, maxit=200, x0=None):
    """Solve A x = b for every right-hand side (leading axis of b).

    Returns (x, info) with info = {"iters": per-RHS inner iterations,
    "resid": per-RHS final true relative residual, "history": list}."""
    nr = b.shape[0]
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bn = _norm(b)
    bn[bn == 0] = 1.0
    iters = np.zeros(nr, dtype=int)
    history = []
    total = 0
    while True:
        r = b - apply_A(x)
        rel = _norm(r) / bn
        history.append(rel.copy())
        active = rel > rtol
        if not active.any() or total >= maxit:
            break
        beta = _norm(r)
        V = [r / np.where(beta > 0, beta, 1.0).reshape((nr,) + (1,) * (b.ndim - 1))]
        Z = []
        H = np.zeros((nr, restart + 1, restart), dtype=np.complex128)
        y = None
        for k in range(restart):
            z = apply_M(V[k])
            w = apply_A(z)
            Z.append(z)
            for i in range(k + 1):
                H[:, i, k] = _dot(V[i], w)
                w = w - H[:, i, k].reshape((nr,) + (1,) * (b.ndim - 1)) * V[i]
            H[:, k + 1, k] = _norm(w)
            V.append(w / np.where(H[:, k + 1, k] > 0, H[:, k + 1, k], 1.0).real.reshape(
                (nr,) + (1,) * (b.ndim - 1)))
            total += 1
            iters += active
            # least squares min || beta e1 - H_k y || per RHS
            y = np.zeros((nr, k + 1), dtype=np.complex128)
            est = np.zeros(nr)
            for s in range(nr):
                e1 = np.zeros(k + 2, dtype=np.complex128)
                e1[0] = beta[s]
                ys, *_ = np.linalg.lstsq(H[s, :k + 2, :k + 1], e1, rcond=None)
                y[s] = ys
                est[s] = np.linalg.norm(e1 - H[s, :k + 2, :k + 1] @ ys) / bn[s]
            if np.all((est <= rtol) | ~active) or total >= maxit:
                break
        for i in range(len(Z)):
            coef = np.where(active, y[:, i], 0.0).reshape((nr,) + (1,) * (b.ndim - 1))
            x = x + coef * Z[i]
    return x, {"iters": iters, "resid": history[-1], "history": history}
