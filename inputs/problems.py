"""Synthetic Darcy problems in the shape of the paper's workloads.

Each Problem is a 2D Cartesian grid on [0, Lx] x [0, Ly] with nx x ny cells,
a cell-wise scalar permeability K (isotropic, Section 5.1), an integrated
source q per cell, a boundary-condition type per side and a value per
boundary face, the leaf subdomain shape, the interface segment length (the
intermediate scale H-bar of Section 4, in cells) and the Robin coefficient
alpha of Eq. (robin.beta).

Layouts (all float64, x fastest):
  K, q        : (ny, nx)
  bc_type     : (x-, x+, y-, y+), NEUMANN or DIRICHLET
  bc_val      : concatenation of the x- faces (ny, by j), x+ faces (ny),
                y- faces (nx, by i), y+ faces (nx); a Dirichlet side holds
                g_D, a Neumann side the outward normal flux density g_N.
"""
from dataclasses import dataclass, field
import numpy as np

from .fields import lognormal_permeability

NEUMANN = 0
DIRICHLET = 1


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    Lx: float
    Ly: float
    K: np.ndarray
    q: np.ndarray
    bc_type: tuple
    bc_val: np.ndarray
    sub: tuple = (16, 16)
    seg: tuple = (4, 4)
    alpha: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def hx(self):
        return self.Lx / self.nx

    @property
    def hy(self):
        return self.Ly / self.ny

    @property
    def pure_neumann(self):
        return all(t == NEUMANN for t in self.bc_type)

    def bc_slices(self):
        """Index ranges of the four sides inside bc_val."""
        ny, nx = self.ny, self.nx
        return {0: slice(0, ny), 1: slice(ny, 2 * ny),
                2: slice(2 * ny, 2 * ny + nx), 3: slice(2 * ny + nx, 2 * ny + 2 * nx)}


def _bc_left_right(nx, ny, p_left=1.0, p_right=0.0):
    types = (DIRICHLET, DIRICHLET, NEUMANN, NEUMANN)
    val = np.zeros(2 * nx + 2 * ny)
    val[0:ny] = p_left
    val[ny:2 * ny] = p_right
    return types, val


def darcy_problem(nx, ny, *, sigma2=1.0, corr=0.1, seed=0, bc="left_right",
                  alpha=1.0, sub=(16, 16), seg=(4, 4), Lx=1.0, Ly=None,
                  K=None, name=None):
    """Build a problem.

    bc = "left_right": p=1 on x=0, p=0 on x=Lx, no-flow on y=0 and y=Ly,
         no source (the paper's setup, Section 5.1).
    bc = "quarter_five_spot": no-flow on every side, q=+1 in cell (0,0) and
         q=-1 in cell (nx-1, ny-1) (pure Neumann; pressure mean fixed to 0).
    sigma2 = 0 gives K = 1 (homogeneous case).  K may be passed explicitly.
    """
    if Ly is None:
        Ly = Lx * ny / nx
    hx, hy = Lx / nx, Ly / ny
    if K is None:
        if sigma2 == 0.0:
            K = np.ones((ny, nx))
        else:
            K = lognormal_permeability(nx, ny, hx, hy, sigma2, corr, seed)
    K = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(ny, nx))
    q = np.zeros((ny, nx))
    if bc == "left_right":
        types, val = _bc_left_right(nx, ny)
    elif bc == "quarter_five_spot":
        types = (NEUMANN, NEUMANN, NEUMANN, NEUMANN)
        val = np.zeros(2 * nx + 2 * ny)
        q[0, 0] = 1.0
        q[ny - 1, nx - 1] = -1.0
    else:
        raise ValueError(f"unknown bc preset {bc!r}")
    return Problem(name or f"{nx}x{ny}-{bc}", nx, ny, Lx, Ly, K, q, types, val,
                   tuple(sub), tuple(seg), float(alpha),
                   dict(sigma2=sigma2, corr=corr, seed=seed, bc=bc))


def config_64():
    """64x64 unit square, sigma^2=1, corr 0.1, p=1 left / 0 right, no-flow
    top/bottom, f=0, 4x4 leaves of 16x16, 4-cell segments, alpha=1."""
    return darcy_problem(64, 64, sigma2=1.0, corr=0.1, seed=1000,
                         bc="left_right", alpha=1.0, name="square64-lr")


def config_1024(n=1024):
    """1024x1024 unit square, sigma^2=4, corr 0.05, quarter-five-spot source,
    no-flow boundary, pressure mean 0, 64x64 leaves of 16x16, 4-cell
    segments, alpha=1."""
    return darcy_problem(n, n, sigma2=4.0, corr=0.05, seed=2000,
                         bc="quarter_five_spot", alpha=1.0,
                         name=f"square{n}-qfs")


def config_4096(n=4096):
    """4096x4096 unit square, sigma^2=3, corr 0.02, quarter-five-spot."""
    return darcy_problem(n, n, sigma2=3.0, corr=0.02, seed=5000,
                         bc="quarter_five_spot", alpha=1.0,
                         name=f"square{n}-qfs")


def ensemble_member(r, nmin=250, nmax=1000, seed0=4000):
    """Realisation r of the batched ensemble workload: a unit square with nx,
    ny drawn uniformly from nmin..nmax cells and a log-normal K with sigma^2
    drawn uniformly from [1, 4], correlation length 0.05 (seed seed0 + r for
    both draws); p = 1 on x = 0, p = 0 on x = 1, no-flow on y = 0 and y = 1;
    16 x 16 leaves (truncated at the right and top edges), 4-cell segments,
    alpha = 1."""
    rng = np.random.default_rng(seed0 + r)
    nx, ny = (int(x) for x in rng.integers(nmin, nmax + 1, 2))
    sigma2 = float(rng.uniform(1.0, 4.0))
    return darcy_problem(nx, ny, sigma2=sigma2, corr=0.05, seed=seed0 + r, bc="left_right", alpha=1.0,
                         Lx=1.0, Ly=1.0, name=f"ensemble{r}-{nx}x{ny}")


@dataclass
class Problem3D:
    """A 3D Cartesian grid on [0, Lx] x [0, Ly] x [0, Lz] with nx x ny x nz
    cells.  Layouts (float64, x fastest, then y, then z):
      K, q     : (nz, ny, nx)
      bc_type  : (x-, x+, y-, y+, z-, z+), NEUMANN or DIRICHLET
      bc_val   : the six sides' face values concatenated in that order; the
                 x sides hold (nz, ny) faces, the y sides (nz, nx), the z
                 sides (ny, nx), each flattened with its first listed index
                 slowest.
    sub / seg are the leaf shape and the interface patch shape in cells per
    axis (a patch on an x-normal interface spans seg[1] x seg[2] faces)."""
    name: str
    nx: int
    ny: int
    nz: int
    Lx: float
    Ly: float
    Lz: float
    K: np.ndarray
    q: np.ndarray
    bc_type: tuple
    bc_val: np.ndarray
    sub: tuple = (16, 16, 16)
    seg: tuple = (4, 4, 4)
    alpha: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return (self.nx, self.ny, self.nz)

    @property
    def h(self):
        return (self.Lx / self.nx, self.Ly / self.ny, self.Lz / self.nz)

    @property
    def pure_neumann(self):
        return all(t == NEUMANN for t in self.bc_type)

    def side_shape(self, side):
        """Face array shape of a boundary side (see bc_val)."""
        nx, ny, nz = self.n
        return ((nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx))[side]

    def bc_slices(self):
        out, off = {}, 0
        for s in range(6):
            a, b = self.side_shape(s)
            out[s] = slice(off, off + a * b)
            off += a * b
        return out


def darcy_problem_3d(nx, ny, nz, *, sigma2=2.0, corr=(0.2, 0.2, 0.05), seed=0,
                     bc="left_right", alpha=1.0, sub=(16, 16, 16), seg=(4, 4, 4),
                     L=None, K=None, name=None):
    """bc = "left_right": p = 1 on x = 0, p = 0 on x = Lx, no-flow on the
    other four sides, no source (the paper's 3D setup, Section 5.1).
    bc = "quarter_five_spot": no-flow everywhere, q = +1 in cell (0, 0, 0)
    and -1 in the opposite corner cell.  L defaults to cubic cells with
    Lx = 1.  sigma2 = 0 gives K = 1."""
    from .fields import lognormal_permeability_3d
    if L is None:
        L = (1.0, ny / nx, nz / nx)
    h = (L[0] / nx, L[1] / ny, L[2] / nz)
    if K is None:
        if sigma2 == 0.0:
            K = np.ones((nz, ny, nx))
        else:
            K = lognormal_permeability_3d((nx, ny, nz), h, sigma2, corr, seed)
    K = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(nz, ny, nx))
    q = np.zeros((nz, ny, nx))
    nb = 2 * (ny * nz + nx * nz + nx * ny)
    val = np.zeros(nb)
    if bc == "left_right":
        types = (DIRICHLET, DIRICHLET, NEUMANN, NEUMANN, NEUMANN, NEUMANN)
        val[0:ny * nz] = 1.0
    elif bc == "quarter_five_spot":
        types = (NEUMANN,) * 6
        q[0, 0, 0] = 1.0
        q[nz - 1, ny - 1, nx - 1] = -1.0
    else:
        raise ValueError(f"unknown bc preset {bc!r}")
    return Problem3D(name or f"{nx}x{ny}x{nz}-{bc}", nx, ny, nz, L[0], L[1], L[2], K, q, types,
                     val, tuple(sub), tuple(seg), float(alpha),
                     dict(sigma2=sigma2, corr=tuple(corr), seed=seed, bc=bc))


def config_3d(nx=256, ny=256, nz=64):
    """256 x 256 x 64 cubic cells on [0,1] x [0,1] x [0,0.25], log-normal K
    with sigma^2 = 2 and correlation lengths (0.2, 0.2, 0.05), p = 1 at
    x = 0 / p = 0 at x = 1, no-flow elsewhere; 16^3 leaves, 4 x 4 face
    patches, alpha = 1.  Other sizes keep the cell size h = 1/256."""
    return darcy_problem_3d(nx, ny, nz, sigma2=2.0, corr=(0.2, 0.2, 0.05), seed=3000,
                            bc="left_right", alpha=1.0, L=(nx / 256, ny / 256, nz / 256),
                            name=f"box{nx}x{ny}x{nz}-lr")
