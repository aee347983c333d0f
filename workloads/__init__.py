"""Seeded synthetic inputs for the diagonal sweeping DDM (media, sources, partitions).

This module is shared by the CPU oracle and by the CUDA path's tests and bench.
It holds problem *inputs* only -- grid sizes, squared slowness fields, source
vectors, subdomain cut positions -- and none of the method's arithmetic (no PML
stretching, no operator, no cutoff, no sweep).

Conventions (shared by both sides):
  * The full grid is the interior (``n[a]`` cells per axis) plus ``pml`` cells
    on each side, ``N[a] = n[a] + 2*pml``.  Arrays over it are C-ordered with x
    fastest: shape ``(Ny, Nx)`` in 2D and ``(Nz, Ny, Nx)`` in 3D.
  * Nodes are cell centred.  Global node ``k`` along an axis sits at interior
    coordinate ``x = (k - pml + 0.5) * h``; the interior spans ``[0, n*h]``.
  * ``cuts[a]`` are the subdomain box faces in interior cells, ``cuts[a][0]=0``
    and ``cuts[a][-1]=n[a]`` (Section 2.1 partition xi_i, eta_j, zeta_k).
  * ``m`` is the squared slowness 1/c^2 on the full grid (float64); the PML
    rows copy the nearest interior value.
  * ``f`` holds the right-hand sides of  Delta u + kappa^2 u = f  (Eq. 1.1),
    complex128, shape ``(nrhs, *grid)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "Workload", "uniform_cuts", "random_cuts", "gaussian_sources", "point_sources",
    "constant_medium", "layered_medium", "smooth_random_medium", "config", "small_2d",
    "small_3d", "two_layer_2d", "iter_r3_3d", "CONFIG_NAMES",
]


@dataclass
class Workload:
    name: str
    ndim: int
    n: tuple                    # interior cells per axis (x, y[, z])
    h: float
    omega: float
    pml: int                    # global PML cells per side
    sigma0: float               # PML strength: sigma(t) = sigma0 (t/L)^power
    power: int
    nb: tuple                   # subdomains per axis
    cuts: tuple                 # per-axis int arrays of box faces (interior cells)
    overlap: int                # d, in cells
    sub_pml: int                # PML cells on internal subdomain sides
    m: np.ndarray               # full-grid squared slowness
    f: Optional[np.ndarray]     # (nrhs, *grid) complex128 sources
    receivers: Optional[np.ndarray] = None   # (nrec, ndim) global node indices
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> tuple:
        return tuple(int(k) + 2 * self.pml for k in self.n)

    @property
    def grid_shape(self) -> tuple:
        return tuple(reversed(self.N))

    @property
    def nrhs(self) -> int:
        return 0 if self.f is None else int(self.f.shape[0])


# ----------------------------------------------------------------------------- partitions
def uniform_cuts(n: int, nb: int) -> np.ndarray:
    """Uniform box faces 0 = c_0 < c_1 < ... < c_nb = n (rounded to cells)."""
    return np.array([(i * n) // nb for i in range(nb + 1)], dtype=np.int64)


def random_cuts(n: int, nb: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Box widths drawn from U{lo..hi}, then moved one cell at a time (round
    robin, staying inside [lo, hi]) until they sum to n."""
    rng = np.random.default_rng(seed)
    w = rng.integers(lo, hi + 1, size=nb).astype(np.int64)
    if not (nb * lo <= n <= nb * hi):
        raise ValueError("widths cannot sum to n within bounds")
    i = 0
    while w.sum() != n:
        step = 1 if w.sum() < n else -1
        if lo <= w[i % nb] + step <= hi:
            w[i % nb] += step
        i += 1
    return np.concatenate([[0], np.cumsum(w)]).astype(np.int64)


# ----------------------------------------------------------------------------- coordinates
def node_coords(n: Sequence[int], pml: int, h: float):
    """Interior coordinates of every full-grid node, one 1-D array per axis."""
    return [((np.arange(k + 2 * pml) - pml) + 0.5) * h for k in n]


def _mesh(n, pml, h):
    xs = node_coords(n, pml, h)
    return np.meshgrid(*reversed(xs), indexing="ij")[::-1]  # x, y[, z] arrays in grid shape


# ----------------------------------------------------------------------------- media
def constant_medium(n, pml, c: float = 1.0) -> np.ndarray:
    shape = tuple(reversed([k + 2 * pml for k in n]))
    return np.full(shape, 1.0 / (c * c), dtype=np.float64)


def _filtered_noise(shape, sigma_cells: float, seed: int) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    g = gaussian_filter(rng.standard_normal(shape), sigma=sigma_cells, mode="nearest")
    return g / np.max(np.abs(g))


def layered_medium(n, pml, h, speeds=(1500.0, 2250.0, 3000.0, 3750.0, 4500.0),
                   perturb: float = 0.1, corr_cells: float = 10.0, seed: int = 2,
                   depth_axis: int = 1) -> np.ndarray:
    """Equal-depth layers (speed grows with depth) times (1 + perturb*g), g a
    Gaussian-filtered white field normalised to max|g| = 1.  PML cells copy the
    nearest interior layer."""
    N = [k + 2 * pml for k in n]
    shape = tuple(reversed(N))
    nd = n[depth_axis]
    k = np.clip(np.arange(N[depth_axis]) - pml, 0, nd - 1)
    layer = np.minimum((k * len(speeds)) // nd, len(speeds) - 1)
    c1 = np.asarray(speeds, dtype=np.float64)[layer]
    bshape = [1] * len(n)
    bshape[len(n) - 1 - depth_axis] = N[depth_axis]
    c = np.broadcast_to(c1.reshape(bshape), shape).copy()
    if perturb:
        c *= 1.0 + perturb * _filtered_noise(shape, corr_cells, seed)
    return 1.0 / (c * c)


def smooth_random_medium(n, pml, cmin: float, cmax: float, corr_cells: float,
                         seed: int) -> np.ndarray:
    """White noise filtered with a Gaussian of std ``corr_cells`` cells, mapped
    affinely onto [cmin, cmax]."""
    shape = tuple(reversed([k + 2 * pml for k in n]))
    g = _filtered_noise(shape, corr_cells, seed)
    g = (g - g.min()) / (g.max() - g.min())
    c = cmin + (cmax - cmin) * g
    return 1.0 / (c * c)


# ----------------------------------------------------------------------------- sources
def gaussian_sources(n, pml, h, centres, width: float) -> np.ndarray:
    """exp(-|x-x0|^2 / (2 width^2)) for each centre x0 (interior coordinates)."""
    X = _mesh(n, pml, h)
    out = np.zeros((len(centres),) + X[0].shape, dtype=np.complex128)
    for s, x0 in enumerate(centres):
        r2 = sum((X[a] - x0[a]) ** 2 for a in range(len(n)))
        out[s] = np.exp(-r2 / (2.0 * width * width))
    return out


def point_sources(n, pml, h, nodes) -> np.ndarray:
    """Discrete delta 1/h^ndim at the given global node index tuples (x, y[, z])."""
    shape = tuple(reversed([k + 2 * pml for k in n]))
    out = np.zeros((len(nodes),) + shape, dtype=np.complex128)
    for s, idx in enumerate(nodes):
        out[(s,) + tuple(reversed(tuple(int(i) for i in idx)))] = 1.0 / h ** len(n)
    return out


# ----------------------------------------------------------------------------- configs
CONFIG_NAMES = {
    1: "2d-const-160sq-2x2-1rhs",
    2: "2d-layered-1064sq-8x8-64rhs",
    3: "3d-const-80cube-4x4x4-16rhs",
    4: "2d-smooth-2088x1576-12x9-256rhs",
    5: "2d-adjoint-544sq-4x4-32src-256rec",
}


def config(k: int, with_sources: bool = True, src: Sequence[int] = None) -> Workload:
    """The five seismic-shaped synthetic workloads, with the sizes of the
    paper's experiments (Section 5) scaled to one GPU.  ``src`` keeps only the
    sources with these indices (same positions as in the full set)."""
    pick = (lambda xs: [xs[i] for i in src]) if src is not None else (lambda xs: list(xs))
    if k == 1:
        n, pml, h = (128, 128), 16, 1.0 / 128
        m = constant_medium(n, pml)
        f = gaussian_sources(n, pml, h, pick([(0.3, 0.6)]), 2 * h) if with_sources else None
        return Workload(CONFIG_NAMES[1], 2, n, h, 2 * np.pi * 8, pml, 50.0, 2, (2, 2),
                        (uniform_cuts(128, 2), uniform_cuts(128, 2)), 8, 16, m, f)
    if k == 2:
        n, pml, h = (1024, 1024), 20, 10.0
        m = layered_medium(n, pml, h, seed=2)
        nodes = [(pml + 16 * s + 8, pml + 2) for s in range(64)]
        f = point_sources(n, pml, h, pick(nodes)) if with_sources else None
        return Workload(CONFIG_NAMES[2], 2, n, h, 2 * np.pi * 15, pml, 50.0, 2, (8, 8),
                        (uniform_cuts(1024, 8), uniform_cuts(1024, 8)), 8, 20, m, f)
    if k == 3:
        n, pml, h = (64, 64, 64), 8, 1.0 / 64
        m = constant_medium(n, pml)
        rng = np.random.default_rng(3)
        centres = rng.uniform(0.125, 0.875, size=(16, 3))
        f = gaussian_sources(n, pml, h, pick(list(centres)), 2 * h) if with_sources else None
        cuts = tuple(uniform_cuts(64, 4) for _ in range(3))
        return Workload(CONFIG_NAMES[3], 3, n, h, 2 * np.pi * 8, pml, 50.0, 2, (4, 4, 4),
                        cuts, 2, 6, m, f)
    if k == 4:
        n, pml, h = (2048, 1536), 20, 7.5
        m = smooth_random_medium(n, pml, 1500.0, 4500.0, 40.0, seed=4)
        rng = np.random.default_rng(41)
        xs = np.sort(rng.integers(0, n[0], size=256))
        nodes = [(pml + int(x), pml + 2) for x in xs]
        f = point_sources(n, pml, h, pick(nodes)) if with_sources else None
        cuts = (random_cuts(2048, 12, 96, 224, seed=40), random_cuts(1536, 9, 96, 224, seed=40))
        return Workload(CONFIG_NAMES[4], 2, n, h, 2 * np.pi * 20, pml, 50.0, 2, (12, 9),
                        cuts, 8, 20, m, f)
    if k == 5:
        n, pml, h = (512, 512), 16, 10.0
        m0 = layered_medium(n, pml, h, seed=5)
        X = _mesh(n, pml, h)
        xc = (n[0] * h / 2, n[1] * h / 2)
        bump = np.exp(-((X[0] - xc[0]) ** 2 + (X[1] - xc[1]) ** 2) / (2 * 50.0 ** 2))
        m_true = m0 * (1.0 + 0.05 * bump)
        shots = [(pml + int((s + 0.5) * n[0] / 32), pml + 2) for s in range(32)]
        rec = np.array([(pml + int((r + 0.5) * n[0] / 256), pml + 2) for r in range(256)])
        f = point_sources(n, pml, h, pick(shots)) if with_sources else None
        return Workload(CONFIG_NAMES[5], 2, n, h, 2 * np.pi * 10, pml, 50.0, 2, (4, 4),
                        (uniform_cuts(512, 4), uniform_cuts(512, 4)), 8, 16, m0, f,
                        receivers=rec, meta={"m_true": m_true})
    raise ValueError(f"unknown config {k}")


def iter_const_2d(cells: int, nb: int, freq: float, pml: int = 30, overlap: int = 8) -> Workload:
    """The constant-medium scaling problems of Section 5.2.1: the unit square
    (c = 1) with ``cells`` x ``cells`` cells in ``nb`` x ``nb`` equal subdomains,
    omega = 2 pi freq, a PML of ``pml`` cells (global and subdomain) and one
    right-hand side made of four discrete deltas at the quarter points
    (1/4, 1/4), (1/4, 3/4), (3/4, 1/4), (3/4, 3/4), each at its nearest node.
    The overlap d is not stated there (8 cells, as for the other workloads)."""
    n = (cells, cells)
    h = 1.0 / cells
    m = constant_medium(n, pml)
    idx = [int(round(q / h - 0.5)) + pml for q in (0.25, 0.75)]
    f = point_sources(n, pml, h, [(ix, iy) for ix in idx for iy in idx]).sum(axis=0, keepdims=True)
    return Workload(f"2d-const-{cells}sq-{nb}x{nb}-iter", 2, n, h, 2 * np.pi * freq, pml, 50.0, 2,
                    (nb, nb), (uniform_cuts(cells, nb), uniform_cuts(cells, nb)), overlap, pml, m, f)


def iter_r3_3d(nb: int, box: int = 16, pml: int = 6, overlap: int = 2, sub_pml: int = 6,
               seed: int = 53) -> Workload:
    """A scaled stand-in of the 3D five-layer experiment of Section 5.2
    (Table tab:iter_R3): the unit cube in nb^3 equal subdomains of box^3 cells
    (box = 16 and a 6-cell PML where the paper has 30 and 12, so that a plane
    block of a window stays within 32 x 32 nodes), five equal-depth layers of
    speed 1.0 .. 2.0 along z (the paper's speeds are given only in a figure), a
    frequency of 8 points per wavelength at the slowest speed, and
    N_RHS = 2 (3 nb - 2) point sources on the plane z = 0.85 at seeded (x, y)
    positions."""
    cells = box * nb
    n, h = (cells, cells, cells), 1.0 / cells
    m = layered_medium(n, pml, h, speeds=(1.0, 1.25, 1.5, 1.75, 2.0), perturb=0.0, depth_axis=2)
    omega = 2 * np.pi * 1.0 / (8 * h)
    rng = np.random.default_rng(seed)
    nrhs = 2 * (3 * nb - 2)
    xy = rng.uniform(0.1, 0.9, size=(nrhs, 2))
    iz = int(round(0.85 / h - 0.5)) + pml
    nodes = [(int(round(x / h - 0.5)) + pml, int(round(y / h - 0.5)) + pml, iz) for x, y in xy]
    f = point_sources(n, pml, h, nodes)
    cuts = tuple(uniform_cuts(cells, nb) for _ in range(3))
    return Workload(f"3d-5layer-{cells + 2 * pml}cube-{nb}x{nb}x{nb}-{nrhs}rhs", 3, n, h, omega, pml, 50.0, 2,
                    (nb, nb, nb), cuts, overlap, sub_pml, m, f)


def small_2d(nx=48, ny=40, nbx=3, nby=2, pml=8, overlap=4, sub_pml=8, nrhs=2,
             medium="layered", omega=None, seed=7, sigma0=50.0) -> Workload:
    """A small 2D case (oracle runs in well under a second) spanning several
    kernel tiles and a ragged tail: odd sizes, unequal boxes."""
    n, h = (nx, ny), 1.0 / max(nx, ny)
    if medium == "const":
        m = constant_medium(n, pml)
    else:
        m = layered_medium(n, pml, h, speeds=(1.0, 1.3, 1.7), perturb=0.1,
                           corr_cells=3.0, seed=seed)
    omega = omega if omega is not None else 2 * np.pi * max(nx, ny) / 12.0
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.15, 0.85, size=(nrhs, 2)) * np.array([nx * h, ny * h])
    f = gaussian_sources(n, pml, h, centres, 1.5 * h)
    return Workload(f"small2d-{nx}x{ny}-{nbx}x{nby}", 2, n, h, omega, pml, sigma0, 2,
                    (nbx, nby), (uniform_cuts(nx, nbx), uniform_cuts(ny, nby)), overlap,
                    sub_pml, m, f)


def small_3d(n=(20, 18, 16), nb=(2, 2, 2), pml=5, overlap=2, sub_pml=4, nrhs=2,
             medium="const", seed=11) -> Workload:
    h = 1.0 / max(n)
    m = constant_medium(n, pml) if medium == "const" else layered_medium(
        n, pml, h, speeds=(1.0, 1.4), perturb=0.05, corr_cells=2.0, seed=seed, depth_axis=2)
    omega = 2 * np.pi * max(n) / 10.0
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(nrhs, 3)) * np.array([k * h for k in n])
    f = gaussian_sources(n, pml, h, centres, 1.5 * h)
    cuts = tuple(uniform_cuts(n[a], nb[a]) for a in range(3))
    return Workload(f"small3d-{n[0]}x{n[1]}x{n[2]}", 3, tuple(n), h, omega, pml, 50.0, 2,
                    tuple(nb), cuts, overlap, sub_pml, m, f)


def two_layer_2d(n=64, nb=(2, 2), pml=12, overlap=6, sub_pml=12, interface_frac=0.75,
                 speeds=(1.0, 1.5), source_box=(1, 0)) -> Workload:
    """Two-layer medium with the interface in the upper half (Section 5.2.2); one
    Gaussian source centred in box ``source_box`` (0-based box indices)."""
    N = n + 2 * pml
    h = 1.0 / n
    k = np.arange(N) - pml
    c1 = np.where(k < int(interface_frac * n), speeds[0], speeds[1]).astype(np.float64)
    m = np.broadcast_to((1.0 / c1 ** 2)[:, None], (N, N)).copy()
    cuts = (uniform_cuts(n, nb[0]), uniform_cuts(n, nb[1]))
    cx = 0.5 * (cuts[0][source_box[0]] + cuts[0][source_box[0] + 1]) * h
    cy = 0.5 * (cuts[1][source_box[1]] + cuts[1][source_box[1] + 1]) * h
    f = gaussian_sources((n, n), pml, h, [(cx, cy)], 1.5 * h)
    return Workload(f"twolayer-{n}-{nb[0]}x{nb[1]}", 2, (n, n), h, 2 * np.pi * n / 12.0, pml,
                    50.0, 2, tuple(nb), cuts, overlap, sub_pml, m, f)
