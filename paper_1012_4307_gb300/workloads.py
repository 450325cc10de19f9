"""Seeded synthetic inputs: grids, k^2 fields and sources shaped like the paper's model
problems (Section 5: potential wells, a wavenumber that grows toward the boundary, ECS
layers, localised sources).

This module holds no arithmetic of the solver itself.  It only draws inputs, so the GPU
path and the CPU oracle are fed identical arrays.  Random numbers come from splitmix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators", 2014) and
Box-Muller, written out here, so the arrays are the same on every machine and numpy version.

Arrays are numpy, C-ordered with x fastest, including the Dirichlet boundary nodes.
Node coordinates: x_j = lo + j (hi - lo) / (n - 1) on every axis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of splitmix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.arange(1, count + 1, dtype=np.uint64) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal doubles by Box-Muller on pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    r = np.sqrt(-2.0 * np.log(1.0 - u[0::2]))
    t = 2.0 * math.pi * u[1::2]
    return np.concatenate([r * np.cos(t), r * np.sin(t)])[:count]


def coords(dim: int, n: int, lo: float = -1.0, hi: float = 1.0):
    """Real node coordinates as a list of broadcastable arrays (x fastest)."""
    x = lo + (hi - lo) * np.arange(n, dtype=np.float64) / (n - 1)
    out = []
    for a in range(dim):
        shape = [1] * dim
        shape[dim - 1 - a] = n
        out.append(x.reshape(shape))
    return out


def k2_constant(dim: int, n: int, k: float) -> np.ndarray:
    return np.full((n,) * dim, k * k, dtype=np.float64)


def k2_well_growth(dim: int, n: int, E: float = 2.0, V0: float = 5.0, sigma: float = 0.2,
                   kh_max: float = 0.6, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """k^2 = 2 (E - V) with V = -V0 exp(-r^2/sigma^2) - c r^4, evaluated at the real nodes.

    A Gaussian well at the centre plus a term that grows toward the boundary; c is fixed so
    that k h reaches ``kh_max`` exactly at the corners (r^2 = dim) and stays below elsewhere.
    """
    h = (hi - lo) / (n - 1)
    X = coords(dim, n, lo, hi)
    r2 = sum(x * x for x in X)
    d = float(dim)
    c = ((kh_max / h) ** 2 / 2.0 - E - V0 * math.exp(-d / sigma ** 2)) / (d * d)
    V = -V0 * np.exp(-r2 / sigma ** 2) - c * r2 * r2
    return np.ascontiguousarray(np.broadcast_to(2.0 * (E - V), (n,) * dim)).astype(np.float64)


def gaussian_source(dim: int, n: int, sigma: float, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """f = exp(-|x - c|^2 / (2 sigma^2)) with centre c uniform in [-0.5, 0.5]^dim; zero boundary."""
    c = uniform(seed, dim) - 0.5
    X = coords(dim, n, lo, hi)
    r2 = sum((x - c[a]) ** 2 for a, x in enumerate(X))
    f = np.exp(-r2 / (2.0 * sigma * sigma)).astype(np.complex128)
    f = np.ascontiguousarray(np.broadcast_to(f, (n,) * dim)).copy()
    _zero_ring(f)
    return f


def random_box_source(dim: int, n: int, seed: int, half_width: float = 0.5,
                      lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """i.i.d. complex N(0, 1) node values where |x|_inf < half_width, zero elsewhere."""
    g = normal(seed, 2 * n ** dim)
    f = (g[0::2] + 1j * g[1::2]).reshape((n,) * dim)
    X = coords(dim, n, lo, hi)
    inside = np.ones((n,) * dim, dtype=bool)
    for x in X:
        inside &= np.abs(x) < half_width
    f = np.where(inside, f, 0).astype(np.complex128)
    _zero_ring(f)
    return f


def random_field(shape, seed: int) -> np.ndarray:
    """i.i.d. complex N(0,1) values on every node of ``shape`` with a zero boundary ring."""
    n = int(np.prod(shape))
    g = normal(seed, 2 * n)
    x = (g[0::2] + 1j * g[1::2]).reshape(shape).astype(np.complex128)
    _zero_ring(x)
    return x


def _zero_ring(x: np.ndarray) -> None:
    for ax in range(x.ndim):
        idx = [slice(None)] * x.ndim
        idx[ax] = 0
        x[tuple(idx)] = 0
        idx[ax] = -1
        x[tuple(idx)] = 0


@dataclass
class Problem:
    """One synthetic model problem (geometry, ECS, k^2, source, preconditioner, solver)."""
    name: str
    dim: int
    n: int
    k2: np.ndarray
    f: np.ndarray
    theta: float = math.pi / 6
    r0: float = 0.75
    lo: float = -1.0
    hi: float = 1.0
    pc: str = "csg"
    theta_a: float = math.pi / 14
    beta: tuple = (-1.0, -0.5)
    nu1: int = 2
    nu2: int = 2
    omega: float = 0.8
    smoother: str = "jacobi"
    coarsest_n: int = 17
    restart: int = 30
    tol: float = 1e-10
    extra: dict = field(default_factory=dict)
    r0_lo: float | None = None  # start of the lower layer (default -r0; outside [lo, hi]: none)
    r0_hi: float | None = None  # start of the upper layer (default r0)

    @property
    def unknowns(self) -> int:
        return (self.n - 2) ** self.dim

    @property
    def layers(self):
        """(r0_lo, r0_hi) of every axis."""
        return (-self.r0 if self.r0_lo is None else self.r0_lo, self.r0 if self.r0_hi is None else self.r0_hi)


def config_small(n: int = 65) -> Problem:
    """2D -Delta u - k^2 u = f on [-1,1]^2, n x n nodes, ECS beyond |x|,|y| = 0.75 at pi/6,
    constant k = 10, Gaussian source (sigma 0.05, seed 0), CSG by one V(2,2) cycle of
    omega-Jacobi (0.8), GMRES(30) to 1e-10."""
    return Problem("2d-const-k10-n%d" % n, 2, n, k2_constant(2, n, 10.0), gaussian_source(2, n, 0.05, 0),
                   coarsest_n=17, restart=30, tol=1e-10)


# CSG angle of the well workloads: the paper hand-tunes theta_a per model problem (Section 6,
# Tables 1-4); for these workloads (V(2,2) cycle, k h up to 0.6) a sweep over pi/17 .. pi/6 puts
# the fewest FGMRES iterations at pi/10 .. pi/9 on every grid.
WELL_THETA_A = math.pi / 10


def config_2d_well(n: int = 1025, seed: int = 1) -> Problem:
    """2D n x n nodes, k^2 = 2(E - V) with a Gaussian well (E=2, V0=5, sigma=0.2) and growth
    toward the boundary so that k h <= 0.6, ECS at pi/6, random source on |x|_inf < 0.5."""
    return Problem("2d-well-n%d" % n, 2, n, k2_well_growth(2, n), random_box_source(2, n, seed),
                   coarsest_n=17, restart=30, tol=1e-8, theta_a=WELL_THETA_A)


def config_3d_well(n: int = 257, seed: int = 2) -> Problem:
    """3D 7-point problem, n^3 nodes, same k^2 profile in r, ECS on all faces, FGMRES(20)."""
    return Problem("3d-well-n%d" % n, 3, n, k2_well_growth(3, n), random_box_source(3, n, seed),
                   coarsest_n=9, restart=20, tol=1e-8, theta_a=WELL_THETA_A)


def config_batch(count: int = 64, seed: int = 3, sizes=(129, 257, 513, 1025)):
    """Independent 2D problems, sizes drawn uniformly from ``sizes``, energies E in [0.5, 4],
    Gaussian sources (sigma 0.05)."""
    u = uniform(seed, 3 * count)
    out = []
    for i in range(count):
        n = sizes[min(int(u[3 * i] * len(sizes)), len(sizes) - 1)]
        E = 0.5 + 3.5 * u[3 * i + 1]
        src_seed = int(splitmix64(seed + 1000 + i, 1)[0] % np.uint64(2 ** 31))
        out.append(Problem("batch%d-n%d" % (i, n), 2, n, k2_well_growth(2, n, E=E),
                           gaussian_source(2, n, 0.05, src_seed), coarsest_n=17, restart=30, tol=1e-8,
                           theta_a=WELL_THETA_A, extra={"E": E}))
    return out


def config_adjoint(n: int = 513):
    """2D n x n, k^2 profile with E = 2, Gaussian source (seed 4) and Gaussian probe g (seed 5)."""
    p = Problem("2d-adjoint-n%d" % n, 2, n, k2_well_growth(2, n, E=2.0), gaussian_source(2, n, 0.05, 4),
                coarsest_n=17, restart=30, tol=1e-10, theta_a=WELL_THETA_A)
    g = gaussian_source(2, n, 0.05, 5).real.copy()
    p.extra["probe"] = g
    return p


# ---------------------------------------------------------------- the paper's model problems
# Section 6 (Tables 1-4): 2D, Bi-CGSTAB with one multigrid cycle per preconditioner call.

def paper_mp1(k: float = 160.0, interior_cells: int = 256, layer_cells: int = 64) -> Problem:
    """MP1 (Table 1): Z = -Delta - k^2 with ECS layers of ``layer_cells`` cells on all four sides
    of an interior of ``interior_cells`` cells of width 1 / interior_cells (coordinates shifted so
    that the interior is [-1/2, 1/2]^2), ECS angle pi/6, and a point source: f = 1 at the centre
    node, 0 elsewhere."""
    h = 1.0 / interior_cells
    n = interior_cells + 2 * layer_cells + 1
    half = 0.5 + layer_cells * h
    k2 = np.full((n, n), k * k)
    f = np.zeros((n, n), complex)
    f[n // 2, n // 2] = 1.0
    # k^2 as a sum of one profile per axis (input for the one-dimensional counterpart of QD's
    # lambda0)
    prof = np.full(n, k * k / 2.0)
    return Problem("mp1-k%g" % k, 2, n, k2, f, theta=math.pi / 6, r0=0.5, lo=-half, hi=half, coarsest_n=17,
                   tol=1e-6, extra={"k2_axis": [prof, prof.copy()]})


def _ne_layer_problem(name, k2fun, size, interior_cells, layer_cells, k2axis=None):
    """Square [0, size] of interior_cells cells per axis, ECS layers of layer_cells cells on the
    east and north sides only (Dirichlet at x = 0 and y = 0), ECS angle pi/6; source
    f = exp(-(x^2 + y^2)) (the printed exp(x^2 + y^2) read as the decaying Gaussian)."""
    h = size / interior_cells
    n = interior_cells + layer_cells + 1
    hi = size + layer_cells * h
    X = coords(2, n, 0.0, hi)
    k2 = np.ascontiguousarray(np.broadcast_to(k2fun(X[0], X[1]), (n, n))).astype(np.float64)
    f = np.exp(-(X[0] ** 2 + X[1] ** 2)).astype(np.complex128)
    f = np.ascontiguousarray(np.broadcast_to(f, (n, n))).copy()
    _zero_ring(f)
    extra = {}
    if k2axis is not None:
        x = X[0].ravel()
        prof = np.asarray(k2axis(x), dtype=np.float64)
        extra["k2_axis"] = [prof, prof.copy()]
    return Problem(name, 2, n, k2, f, theta=math.pi / 6, lo=0.0, hi=hi, r0_lo=-1.0, r0_hi=size, coarsest_n=17,
                   tol=1e-6, extra=extra)


def paper_mp2(k: float = 4.0, nu: float = 7.0, size: float = 50.0, interior_cells: int = 512,
              layer_cells: int = 128) -> Problem:
    """MP2 (Table 2): Z = -Delta - nu (exp(-x^2) + exp(-y^2)) - k^2, i.e. k^2(x, y) = k^2 +
    nu (exp(-x^2) + exp(-y^2)) at the real nodes."""
    return _ne_layer_problem("mp2-k%g-nu%g" % (k, nu), lambda x, y: k * k + nu * (np.exp(-x * x) + np.exp(-y * y)),
                             size, interior_cells, layer_cells, lambda x: k * k / 2.0 + nu * np.exp(-x * x))


def paper_mp3(k: float = 2.0, size: float = 50.0, interior_cells: int = 512, layer_cells: int = 128) -> Problem:
    """MP3 (Tables 3, 4): Z = -Delta - 1/x - 1/y - k^2, i.e. k^2(x, y) = k^2 + 1/x + 1/y at the
    real nodes (the singular boundary nodes x = 0, y = 0 are Dirichlet)."""
    def k2fun(x, y):
        with np.errstate(divide="ignore"):
            v = k * k + 1.0 / x + 1.0 / y
        return np.where(np.isfinite(v), v, 0.0)

    def axis(x):
        with np.errstate(divide="ignore"):
            v = k * k / 2.0 + 1.0 / x
        return np.where(np.isfinite(v), v, 0.0)
    return _ne_layer_problem("mp3-k%g-L%g" % (k, size), k2fun, size, interior_cells, layer_cells, axis)
