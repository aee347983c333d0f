"""Helmholtz PML problem on a window of the global grid (oracle; test infrastructure only).

Section 2.1: uniaxial PML with alpha_j = 1 + i sigma_j(x_j) (Eq. 2.1) and the
PML equation  J^{-1} div(A grad u) + kappa^2 u = f  (Eq. 2.2) with
A = diag(alpha_2/alpha_1, alpha_1/alpha_2), J = alpha_1 alpha_2 in 2D and
A = diag(a2 a3/a1, a1 a3/a2, a1 a2/a3), J = a1 a2 a3 in 3D.

Discretisation (Section 5: second-order central differences, 5/7-point
stencil).  We discretise the J-multiplied form  div(A grad u) + J kappa^2 u = J f,
which has the same solution and a complex-symmetric matrix:

  (A u)_k = sum_a  P_a(k) / h^2 * [ (u_{k+e_a} - u_k) / alpha_a(k_a + 1/2)
                                   - (u_k - u_{k-e_a}) / alpha_a(k_a - 1/2) ]
            + omega^2 m_k J_k u_k,          P_a(k) = prod_{b != a} alpha_b(k_b)

with homogeneous Dirichlet values one node beyond the window.  Nodes are cell
centred (node k at cell position k + 1/2), faces at integer positions.

PML profile (Eq. 2.1 with sigma_hat(t) = sigma0 (t/L)^power; Eq. 2.3 shifted):
on a side whose PML starts at face ``face`` after a zero-sigma gap of ``gap``
cells and is ``width`` cells thick,  sigma(p) = sigma0 ((t - gap)/width)^power
for t = distance of position p beyond ``face`` when t > gap, else 0.
The global problem uses gap = 0 at the interior boundary; a subdomain uses
gap = d on its internal sides (the shifted profile of Eq. 2.3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass(frozen=True)
class Side:
    """PML on one side of one axis: starts ``gap`` cells beyond ``face``."""
    face: float
    gap: float
    width: float


@dataclass(frozen=True)
class AxisWindow:
    lo: int          # first global node index of the window on this axis
    hi: int          # one past the last
    left: Side
    right: Side


def sigma(p: np.ndarray, ax: AxisWindow, sigma0: float, power: int) -> np.ndarray:
    """sigma(p) for cell positions p (Eq. 2.1 and the shifted profile Eq. 2.3)."""
    p = np.asarray(p, dtype=np.float64)
    s = np.zeros_like(p)
    tl = ax.left.face - p
    ml = tl > ax.left.gap
    s[ml] = sigma0 * ((tl[ml] - ax.left.gap) / ax.left.width) ** power
    tr = p - ax.right.face
    mr = tr > ax.right.gap
    s[mr] = sigma0 * ((tr[mr] - ax.right.gap) / ax.right.width) ** power
    return s


def alpha(p, ax, sigma0, power, omega, form="literal"):
    """alpha(p) = 1 + i sigma(p) (Eq. 2.1, literal) or 1 + i sigma/omega."""
    s = sigma(p, ax, sigma0, power)
    if form == "omega":
        s = s / omega
    return 1.0 + 1j * s


def global_axes(n, pml):
    """The global PML box: interior faces pml .. pml+n, PML of ``pml`` cells."""
    return [AxisWindow(0, k + 2 * pml, Side(pml, 0.0, pml), Side(pml + k, 0.0, pml)) for k in n]


def assemble(axes, m_window: np.ndarray, h: float, omega: float, sigma0: float,
             power: int, form: str = "literal"):
    """Sparse matrix of the J-multiplied PML operator on a window, and J there.

    ``axes`` lists the AxisWindow of x, y[, z]; ``m_window`` is the squared
    slowness on the window nodes (grid shape, x fastest).  Returns (A, J) with
    A a CSR complex128 matrix over the window nodes in C order and J the
    flattened alpha_1 alpha_2 (alpha_3)."""
    ndim = len(axes)
    sizes = [ax.hi - ax.lo for ax in axes]
    shape = tuple(reversed(sizes))
    nn = int(np.prod(sizes))
    a_node = [alpha(np.arange(ax.lo, ax.hi) + 0.5, ax, sigma0, power, omega, form) for ax in axes]
    a_face = [alpha(np.arange(ax.lo, ax.hi + 1).astype(np.float64), ax, sigma0, power, omega, form)
              for ax in axes]

    def along(vec, a):  # broadcast a 1-D array on axis a to the grid shape
        s = [1] * ndim
        s[ndim - 1 - a] = vec.shape[0]
        return vec.reshape(s)

    J = np.ones(shape, dtype=np.complex128)
    for a in range(ndim):
        J = J * along(a_node[a], a)
    idx = np.arange(nn).reshape(shape)
    diag = omega ** 2 * m_window.reshape(shape) * J
    rows, cols, vals = [], [], []
    for a in range(ndim):
        P = np.ones(shape, dtype=np.complex128)
        for b in range(ndim):
            if b != a:
                P = P * along(a_node[b], b)
        ga = ndim - 1 - a
        # coupling to the + neighbour uses alpha_a at the face k+1/2 (face index k+1)
        cp = P / (h * h) / along(a_face[a][1:], a)
        cm = P / (h * h) / along(a_face[a][:-1], a)
        diag = diag - cp - cm
        sl_lo = [slice(None)] * ndim
        sl_hi = [slice(None)] * ndim
        sl_lo[ga] = slice(0, sizes[a] - 1)
        sl_hi[ga] = slice(1, sizes[a])
        sl_lo, sl_hi = tuple(sl_lo), tuple(sl_hi)
        rows += [idx[sl_lo].ravel(), idx[sl_hi].ravel()]
        cols += [idx[sl_hi].ravel(), idx[sl_lo].ravel()]
        vals += [cp[sl_lo].ravel(), cm[sl_hi].ravel()]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nn, nn))
    return A, J.ravel()


def global_operator(wl, form="literal"):
    """(A, J) of the global PML problem P_B on the full grid of workload ``wl``."""
    axes = global_axes(wl.n, wl.pml)
    return assemble(axes, wl.m, wl.h, wl.omega, wl.sigma0, wl.power, form)


def solve_global(wl, f=None, form="literal", dense=False):
    """Direct solve of the global discrete PML system  A u = J f  (complex128).

    ``dense=True`` uses numpy.linalg.solve (tiny grids only); otherwise SuperLU.
    Returns u with the shape of f."""
    f = wl.f if f is None else f
    A, J = global_operator(wl, form)
    b = (f.reshape(f.shape[0], -1) * J[None, :]).T
    if dense:
        u = np.linalg.solve(A.toarray(), b)
    else:
        u = spla.splu(A.tocsc(), permc_spec="COLAMD").solve(np.ascontiguousarray(b))
    return u.T.reshape(f.shape)
