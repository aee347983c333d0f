"""Diagonal sweeping DDM with source transfer (oracle; test infrastructure only).

Restates, in plain sequential NumPy/SciPy:
  * the checkerboard partition and overlapping subdomains (Section 2.1),
  * the 1-D cutoffs beta^{(a)}_{box,i}, the directional cutoffs beta_{dir;i,j}
    and the box cutoff beta_{0,0;i,j}, the truncations chi_{dir;i,j} and the
    transfer operator Psi_{dir;i,j}(v) = -L_{(i,j)+dir}(beta_{dir;i,j} v) chi_{dir;i,j}
    (Section 2.2),
  * Rules 3.1/3.2 (2D) and 4.1/4.2 (3D) and the routing "smallest usable sweep
    l' >= l" (Algorithm 3.1 / 4.1),
  * Algorithm 3.1 (2D) and Algorithm 4.1 (3D), and for cross-checking the
    additive Algorithm 2.1 / 2.2.

Discrete readings (the paper states the method for the continuous problem):
  * Subdomain boxes are unions of cells; faces sit between nodes.  An edge box
    runs to the end of the global grid (xi_1 = -inf, xi_{Nx+1} = +inf).
  * A subdomain window is its box plus, on each internal side, d overlap cells
    with zero sigma followed by ``sub_pml`` PML cells (shifted profile, Eq. 2.3);
    on an outer side it is the global PML.  Dirichlet one node beyond.
  * Cutoff at the m-th node outside a box face (m = 0 is the first outside
    node): beta_hat(m/d), beta_hat(t) = 1 - (10t^3 - 15t^4 + 6t^5) on [0,1].
    beta = 1 on the box and on the first outside node (one stencil layer), so
    the discrete form of Lemma 2.1 holds exactly: the residual of beta*u is
    supported strictly beyond the face.
  * beta_{0,0;i,j} is the product of the four 1-D cutoffs of box (i,j)
    (the subscripts i+1, j+1 printed in Section 2.2 contradict the 2x2 example
    beta_{Omega_11} = beta_-> beta_^; we read them as i, j).
  * I^{(3)}_{+1,k} is read as (zeta_{k+1}, +inf), as for x and y.
All computations are in the J-multiplied form A = J L (see ``helmholtz``):
the transferred source -A_recv(beta v) chi equals J_recv Psi(v).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from .helmholtz import AxisWindow, Side, assemble, global_axes, global_operator


# ----------------------------------------------------------------------------- cutoff
def beta_hat(t):
    """Monotone C^2 step: 1 for t <= 0, 0 for t >= 1 (Section 2.2)."""
    t = np.clip(np.asarray(t, dtype=np.float64), 0.0, 1.0)
    return 1.0 - t ** 3 * (10.0 - 15.0 * t + 6.0 * t * t)


# ----------------------------------------------------------------------------- sweeps and rules
# the other 3D order Section 4.1 mentions: the L1 distance of each direction
# to the first one never decreases along it
ALT_ORDER_3D = [(1, 1, 1), (-1, 1, 1), (1, -1, 1), (1, 1, -1),
                (-1, -1, 1), (-1, 1, -1), (1, -1, -1), (-1, -1, -1)]


def sweep_dirs(ndim, order=0):
    """Sweep order: (+,+),(-,+),(+,-),(-,-) in 2D (Algorithm 3.1); list
    (Sorder3D) in 3D (Section 4.1): x flips fastest, then y, then z.  With
    order=1 in 3D, the alternative order of Section 4.1 (ALT_ORDER_3D)."""
    if ndim == 3 and order == 1:
        return list(ALT_ORDER_3D)
    return [tuple(-1 if (l >> a) & 1 else 1 for a in range(ndim)) for l in range(2 ** ndim)]


def transfer_dirs(ndim):
    """The 3^n - 1 transfer directions (box, triangle[, circle]) != 0."""
    return [d for d in itertools.product((-1, 0, 1), repeat=ndim) if any(d)][::-1]


def similar(d1, d2):
    """Rule 3.1 (2D): d1.d2 > 0.  Rule 4.1 (3D): d1.d2 > 0 and d1(k) d2(k) >= 0."""
    dot = sum(a * b for a, b in zip(d1, d2))
    if len(d1) == 2:
        return dot > 0
    return dot > 0 and all(a * b >= 0 for a, b in zip(d1, d2))


def opposite_block(d_src, d_gen, d_use):
    """Rule 3.2 / 4.2: a transferred source generated in the sweep of direction
    d_gen is not used in a later sweep d_use if, in some coordinate plane
    (the plane itself in 2D; xy, xz, yz in 3D), the projection of d_src has
    exactly one zero component and the projections of d_gen and d_use are
    opposite."""
    ndim = len(d_src)
    planes = [(0, 1)] if ndim == 2 else [(0, 1), (0, 2), (1, 2)]
    for a, b in planes:
        zeros = (d_src[a] == 0) + (d_src[b] == 0)
        if zeros == 1 and d_gen[a] == -d_use[a] and d_gen[b] == -d_use[b]:
            return True
    return False


def route(ndim, order=0):
    """Routing table {(l, d_src): l'} -- the smallest sweep l' >= l that may
    use a source of direction d_src generated in sweep l (Algorithm 3.1 / 4.1),
    or None if no later sweep may use it; ``order`` as in sweep_dirs."""
    S = sweep_dirs(ndim, order)
    table = {}
    for l in range(len(S)):
        for d in transfer_dirs(ndim):
            table[(l, d)] = None
            for l2 in range(l, len(S)):
                if similar(d, S[l2]) and not opposite_block(d, S[l], S[l2]):
                    table[(l, d)] = l2
                    break
    return table


def front_index(I, nb, D):
    """0-based step of box I in the sweep of direction D: sum of I_a when
    D_a = +1 and of nb_a - 1 - I_a when D_a = -1."""
    return sum(i if s > 0 else nb_a - 1 - i for i, s, nb_a in zip(I, D, nb))


# ----------------------------------------------------------------------------- partition
@dataclass
class Sub:
    I: tuple            # box index per axis (0-based)
    box: list           # per axis (lo, hi) global node range of the box
    axes: list          # per axis AxisWindow of the window
    A: object = None    # local operator (CSR)
    lu: object = None   # SuperLU factorisation

    @property
    def lo(self):
        return [ax.lo for ax in self.axes]

    @property
    def hi(self):
        return [ax.hi for ax in self.axes]

    @property
    def shape(self):
        return tuple(reversed([ax.hi - ax.lo for ax in self.axes]))


class Partition:
    """Checkerboard partition with overlapping PML subdomains (Section 2.1)."""

    def __init__(self, wl, form="literal", factor=True, ideal=False):
        self.wl, self.form = wl, form
        # ideal=True: every subdomain "window" is the whole grid and every local
        # PML problem is the global one (a subdomain PML without truncation).
        # The discrete Lemma 2.1 is then exact for any medium, so Algorithm 3.1/4.1
        # must return the global solution to rounding: a pin of the cutoffs,
        # truncations, transfers, routing and assembly independent of the PML.
        self.ideal = ideal
        self.ndim = wl.ndim
        self.nb = tuple(wl.nb)
        self.N = wl.N
        self.d = wl.overlap
        P, W = wl.pml, wl.sub_pml
        gax = global_axes(wl.n, P)
        self.boxes = []
        for a in range(self.ndim):
            c = np.asarray(wl.cuts[a])
            bl = []
            for i in range(self.nb[a]):
                lo = 0 if i == 0 else P + int(c[i])
                hi = self.N[a] if i == self.nb[a] - 1 else P + int(c[i + 1])
                bl.append((lo, hi))
            self.boxes.append(bl)
        self.subs = {}
        for I in itertools.product(*[range(k) for k in self.nb]):
            axes, box = [], []
            for a, i in enumerate(I):
                blo, bhi = self.boxes[a][i]
                box.append((blo, bhi))
                if i == 0:
                    left, lo = gax[a].left, 0
                else:
                    left, lo = Side(blo, self.d, W), blo - self.d - W
                if i == self.nb[a] - 1:
                    right, hi = gax[a].right, self.N[a]
                else:
                    right, hi = Side(bhi, self.d, W), bhi + self.d + W
                if lo < 0 or hi > self.N[a]:
                    raise ValueError("subdomain window leaves the global grid")
                if bhi - blo < self.d + 2:
                    raise ValueError("box narrower than overlap + 2")
                axes.append(AxisWindow(lo, hi, left, right))
            if ideal:
                axes = list(gax)
            s = Sub(I, box, axes)
            if ideal:
                if not self.subs:
                    A, _ = global_operator(wl, form)
                    glu = spla.splu(A.tocsc(), permc_spec="COLAMD")
                s.A, s.lu = A, glu
            else:
                msl = tuple(slice(ax.lo, ax.hi) for ax in reversed(axes))
                s.A, _ = assemble(axes, wl.m[msl], wl.h, wl.omega, wl.sigma0, wl.power, form)
                if factor:
                    s.lu = spla.splu(s.A.tocsc(), permc_spec="COLAMD")
            self.subs[I] = s

    # -- 1-D cutoffs and truncations over a range of global node indices
    def beta1(self, a, i, box_sign, k):
        """beta^{(a)}_{box_sign, i}(k) at global nodes k (Section 2.2)."""
        k = np.asarray(k)
        lo, hi = self.boxes[a][i]
        out = np.ones(k.shape)
        if box_sign == 1 and i != self.nb[a] - 1:
            out = np.where(k >= hi, beta_hat((k - hi) / self.d), 1.0)
        elif box_sign == -1 and i != 0:
            out = np.where(k < lo, beta_hat((lo - 1 - k) / self.d), 1.0)
        return out

    def chi1(self, a, i, box_sign, k):
        """Indicator of I^{(a)}_{box_sign, i}: beyond the upper face (+1), below
        the lower face (-1), everything (0)."""
        k = np.asarray(k)
        lo, hi = self.boxes[a][i]
        if box_sign == 1:
            return (k >= hi).astype(np.float64)
        if box_sign == -1:
            return (k < lo).astype(np.float64)
        return np.ones(k.shape)

    def _grid(self, vecs):
        """Outer product of per-axis 1-D arrays, in grid (x fastest) order."""
        out = np.ones(())
        for v in reversed(vecs):
            out = np.multiply.outer(out, v)
        return out

    def beta_dir(self, I, d, s):
        """beta_{d;I} on the window of sub s."""
        return self._grid([self.beta1(a, I[a], d[a], np.arange(s.lo[a], s.hi[a]))
                           for a in range(self.ndim)])

    def beta_box(self, I, s):
        """beta_{0,0;I} = product over axes of beta_{-1} beta_{+1} of box I."""
        return self._grid([self.beta1(a, I[a], -1, np.arange(s.lo[a], s.hi[a])) *
                           self.beta1(a, I[a], 1, np.arange(s.lo[a], s.hi[a]))
                           for a in range(self.ndim)])

    def chi_dir(self, I, d, s):
        return self._grid([self.chi1(a, I[a], d[a], np.arange(s.lo[a], s.hi[a]))
                           for a in range(self.ndim)])

    def chi_box(self, I, s):
        return self._grid([((np.arange(s.lo[a], s.hi[a]) >= self.boxes[a][I[a]][0]) &
                            (np.arange(s.lo[a], s.hi[a]) < self.boxes[a][I[a]][1])).astype(float)
                           for a in range(self.ndim)])

    # -- moving window data
    def restrict(self, full, s):
        """Full-grid (nrhs, *grid) -> window (nrhs, *window)."""
        sl = (slice(None),) + tuple(slice(ax.lo, ax.hi) for ax in reversed(s.axes))
        return full[sl]

    def embed_into(self, full, s, val):
        sl = (slice(None),) + tuple(slice(ax.lo, ax.hi) for ax in reversed(s.axes))
        full[sl] += val

    def move(self, v, s_from, s_to):
        """Window data of s_from re-indexed onto the window of s_to (zero where
        s_from does not reach)."""
        out = np.zeros((v.shape[0],) + s_to.shape, dtype=v.dtype)
        src, dst = [slice(None)], [slice(None)]
        for a in reversed(range(self.ndim)):
            lo = max(s_from.lo[a], s_to.lo[a])
            hi = min(s_from.hi[a], s_to.hi[a])
            if hi <= lo:
                return out
            src.append(slice(lo - s_from.lo[a], hi - s_from.lo[a]))
            dst.append(slice(lo - s_to.lo[a], hi - s_to.lo[a]))
        out[tuple(dst)] = v[tuple(src)]
        return out

    def local_solve(self, s, r):
        """u = A_s^{-1} r for window data r of shape (nrhs, *window)."""
        nr = r.shape[0]
        rhs = np.ascontiguousarray(r.reshape(nr, -1).T)
        return s.lu.solve(rhs).T.reshape(r.shape)

    def psi(self, I, d, u):
        """Transferred source J_recv Psi_{d;I}(u) = -A_recv(beta_{d;I} u) chi_{d;I}
        on the window of the receiver I + d (Section 2.2)."""
        s = self.subs[I]
        J2 = tuple(i + k for i, k in zip(I, d))
        s2 = self.subs[J2]
        bu = self.move(u, s, s2) * self.beta_dir(I, d, s2)[None]
        nr = u.shape[0]
        Abu = (s2.A @ bu.reshape(nr, -1).T).T.reshape(bu.shape)
        return -Abu * self.chi_dir(I, d, s2)[None]

    def neighbour(self, I, d):
        J2 = tuple(i + k for i, k in zip(I, d))
        return J2 if all(0 <= j < nb for j, nb in zip(J2, self.nb)) else None

    def assemble_solution(self, parts, nrhs):
        """u_DDM = sum over (l, I) of beta_{0,0;I} u^l_I  (Eq. 3.x / 4.x)."""
        U = np.zeros((nrhs,) + tuple(reversed(self.N)), dtype=np.complex128)
        for (l, I), u in parts.items():
            s = self.subs[I]
            self.embed_into(U, s, u * self.beta_box(I, s)[None])
        return U


def diagonal_sweep(part: Partition, b, trace=None, nsweeps=None, order=0):
    """Algorithm 3.1 (2D) / 4.1 (3D) applied to the J-scaled source b = J f
    (shape (nrhs, *grid)).  Returns u_DDM on the full grid.

    ``trace``, if a dict, receives per (l, I) the local source and solution and
    per (l, I, d) the routed sweep, for invariant tests; ``nsweeps`` stops after
    the first sweeps (tests of the first sweep only); ``order`` selects the 3D
    sweep order (sweep_dirs)."""
    ndim, nb = part.ndim, part.nb
    S = sweep_dirs(ndim, order)
    table = route(ndim, order)
    nrhs = b.shape[0]
    r = {}
    for I, s in part.subs.items():
        r[(0, I)] = part.restrict(b, s) * part.chi_box(I, s)[None]
    parts = {}
    nsteps = sum(k - 1 for k in nb) + 1
    for l, D in enumerate(S[:nsweeps]):
        for step in range(nsteps):
            for I in sorted(part.subs):
                if front_index(I, nb, D) != step:
                    continue
                s = part.subs[I]
                rl = r.get((l, I))
                if rl is None:
                    rl = np.zeros((nrhs,) + s.shape, dtype=np.complex128)
                u = part.local_solve(s, rl)
                parts[(l, I)] = u
                if trace is not None:
                    trace[(l, I)] = (rl, u)
                for d in transfer_dirs(ndim):
                    J2 = part.neighbour(I, d)
                    if J2 is None:
                        continue
                    l2 = table[(l, d)]
                    if trace is not None:
                        trace[(l, I, d)] = l2
                    if l2 is None:
                        continue
                    p = part.psi(I, d, u)
                    key = (l2, J2)
                    r[key] = p if key not in r else r[key] + p
    return part.assemble_solution(parts, nrhs)


def additive(part: Partition, b):
    """Algorithm 2.1 (2D) / 2.2 (3D): every subdomain solves at every step with
    the sum of transfers from step s - |d|_1 (cross-check of the sweeps)."""
    ndim, nb = part.ndim, part.nb
    nrhs = b.shape[0]
    nsteps = sum(k - 1 for k in nb) + 1
    hist = {}
    parts = {}
    for step in range(nsteps):
        for I, s in part.subs.items():
            if step == 0:
                rl = part.restrict(b, s) * part.chi_box(I, s)[None]
            else:
                rl = np.zeros((nrhs,) + s.shape, dtype=np.complex128)
                for d in transfer_dirs(ndim):
                    I0 = tuple(i - k for i, k in zip(I, d))
                    src_step = step - sum(abs(k) for k in d)
                    if src_step < 0 or (src_step, I0) not in hist:
                        continue
                    rl = rl + part.psi(I0, d, hist[(src_step, I0)])
            u = part.local_solve(s, rl)
            hist[(step, I)] = u
            parts[(step, I)] = u
    return part.assemble_solution(parts, nrhs)


def stationary(part: Partition, A, b, iters, order=0):
    """The DDM as an iterative solver, the way Section 5.2.2 runs it (rather
    than as a preconditioner): u_0 = 0, u_{k+1} = u_k + M (b - A u_k), with M
    one application of Algorithm 3.1/4.1 and b = J f.  Returns the iterates
    u_1 .. u_iters and the relative residuals |b - A u_k| / |b| for
    k = 0 .. iters (max over right-hand sides)."""
    nrhs = b.shape[0]
    bn = np.linalg.norm(b.reshape(nrhs, -1), axis=1)
    bn[bn == 0] = 1.0
    u = np.zeros_like(b)
    us, res = [], []
    for k in range(iters + 1):
        r = b - (A @ u.reshape(nrhs, -1).T).T.reshape(b.shape)
        res.append(float(np.max(np.linalg.norm(r.reshape(nrhs, -1), axis=1) / bn)))
        if k == iters:
            break
        u = u + diagonal_sweep(part, r, order=order)
        us.append(u)
    return us, res


class DDMPreconditioner:
    """M: J-scaled residual -> correction, one application of Algorithm 3.1/4.1."""

    def __init__(self, wl, form="literal"):
        self.part = Partition(wl, form)

    def __call__(self, b):
        return diagonal_sweep(self.part, b)


def ddm_solution(wl, f=None, form="literal", order=0):
    """u_DDM for source f: Algorithm 3.1/4.1 applied to J f (3D sweep order
    ``order``, as in sweep_dirs)."""
    f = wl.f if f is None else f
    _, J = global_operator(wl, form)
    part = Partition(wl, form)
    b = f * J.reshape((1,) + f.shape[1:])
    return diagonal_sweep(part, b, order=order)
