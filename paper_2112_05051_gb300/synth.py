"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds problem *data* only: the soil parameters of the paper's
test soil (Fig. 1 caption and eq. (coefficientspectrum1), Supplementary D),
the boundary and initial conditions of the infiltration workloads, the
time-step schedules and the heterogeneous saturated-conductivity field
generator.  It contains none of the method's arithmetic (no constitutive law,
no residual, no Jacobian, no solver), so both the CPU oracle and the GPU path
may read from it without sharing any computation.

Ks field (heterogeneous workloads): log10 Ks = log10(Ks_mean) + sigma * g,
where g is a unit-variance Gaussian random field with the separable
exponential covariance exp(-|dx|/lx - |dy|/ly - |dz|/lz) (in cells).  It is
realised exactly by a stationary AR(1) filter along each axis in turn
(rho_d = exp(-1/l_d), x_0 = w_0, x_i = rho x_{i-1} + sqrt(1-rho^2) w_i),
driven by numpy PCG64(seed) standard normals.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Face order used everywhere: -x, +x, -y, +y, -z (bottom), +z (top).
FACE_NAMES = ("-x", "+x", "-y", "+y", "-z", "+z")
BC_NOFLUX = 0
BC_DIRICHLET = 1

KMEAN_ARITH = 0
KMEAN_UPSTREAM = 1
KMEAN_HARMONIC = 2
KMEAN_GEOMETRIC = 3
KMEAN_NAMES = {KMEAN_ARITH: "arithmetic", KMEAN_UPSTREAM: "upstream", KMEAN_HARMONIC: "harmonic",
               KMEAN_GEOMETRIC: "geometric"}
KMEAN_SPLIT_FLAG = 0x100


def kmean_split(horizontal: int, vertical: int) -> int:
    """Code of a split face mean (Sec. 2.1): one mean on the x and y faces, another on the z faces."""
    return KMEAN_SPLIT_FLAG | (horizontal << 4) | vertical


def kmean_name(code: int) -> str:
    if code & KMEAN_SPLIT_FLAG:
        return "%s horizontal, %s vertical" % (KMEAN_NAMES[(code >> 4) & 0xF], KMEAN_NAMES[code & 0xF])
    return KMEAN_NAMES[code]


@dataclasses.dataclass(frozen=True)
class Soil:
    """Haverkamp/Celia soil parameters (cm, s).

    Defaults: the paper's test soil, Fig. 1 caption and eq.
    (coefficientspectrum1): alpha=1.611e6, beta=3.96, gamma=4.74,
    a=1.175e6, S_s=0.287, S_r=0.075, K_s=0.00944 cm/s.
    ``rho_phi`` is the rho*phi factor of eq. (dynamic_of_the_problem);
    it is 1 (the 1D forms of Sec. 4.2 carry no such factor).
    """

    alpha: float = 1.611e6
    beta: float = 3.96
    theta_s: float = 0.287
    theta_r: float = 0.075
    a: float = 1.175e6
    gamma: float = 4.74
    ks: float = 9.44e-3
    rho_phi: float = 1.0


@dataclasses.dataclass(frozen=True)
class Grid:
    """n_x x n_y x n_z unknown cells on a box of size l_x x l_y x l_z (cm).

    The paper's grid (Sec. 2.1) has N nodes per direction with the outermost
    nodes on the boundary and unknowns on the interior nodes, so with
    n = N - 2 unknowns the spacing is h = L / (n + 1).  Cell (i, j, k),
    0-based, is unknown number c = i + n_x (j + n_y k) and sits at elevation
    z = (k + 1) h_z (z upward).
    """

    nx: int
    ny: int
    nz: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0
    spacing: Optional[Tuple[float, float, float]] = None  # explicit (h_x, h_y, h_z), e.g. a block of a split grid

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self) -> Tuple[int, int, int]:
        """numpy shape (n_z, n_y, n_x): C order gives c = i + n_x (j + n_y k)."""
        return (self.nz, self.ny, self.nx)

    @property
    def h(self) -> Tuple[float, float, float]:
        if self.spacing is not None:
            return tuple(self.spacing)
        return (self.lx / (self.nx + 1), self.ly / (self.ny + 1), self.lz / (self.nz + 1))


@dataclasses.dataclass(frozen=True)
class BC:
    """Boundary condition per face in FACE_NAMES order.

    ``fields`` optionally gives per-cell Dirichlet values of a face (a float64
    array over the face's cells, flat index i + nx j on z faces, i + nx k on y
    faces, j + ny k on x faces), or None per face for the constant ``value``.
    """

    kind: Tuple[int, int, int, int, int, int]
    value: Tuple[float, float, float, float, float, float]
    fields: Optional[Tuple] = None

    def field(self, f):
        return None if self.fields is None else self.fields[f]


def infiltration_bc(p_top: float = -20.7) -> BC:
    """Dirichlet top face at p_top, no-flux elsewhere (the workloads' BCs)."""
    return BC(kind=(BC_NOFLUX,) * 5 + (BC_DIRICHLET,), value=(0.0,) * 5 + (p_top,))


def all_dirichlet_bc(value: float) -> BC:
    return BC(kind=(BC_DIRICHLET,) * 6, value=(value,) * 6)


def all_noflux_bc() -> BC:
    return BC(kind=(BC_NOFLUX,) * 6, value=(0.0,) * 6)


def paper_infiltration_bc(grid: Grid, h_r: float) -> BC:
    """The paper's infiltration test (Sec. 6): Dirichlet on every face, p = h_r except
    p = 0 on the centred square [a/4, 3a/4] x [b/4, 3b/4] of the top face.

    The paper's formula (1/alpha) ln[exp(alpha h_r) + (1 - exp(alpha h_r)) chi] is 0
    where chi = 1 and h_r elsewhere for any alpha; cell (i, j) of the top face sits
    at ((i+1) h_x, (j+1) h_y)."""
    hx, hy, _ = grid.h
    x = (np.arange(grid.nx) + 1) * hx
    y = (np.arange(grid.ny) + 1) * hy
    inside = ((x[None, :] >= grid.lx / 4) & (x[None, :] <= 3 * grid.lx / 4)
              & (y[:, None] >= grid.ly / 4) & (y[:, None] <= 3 * grid.ly / 4))
    top = np.where(inside, 0.0, h_r).reshape(-1)
    return BC(kind=(BC_DIRICHLET,) * 6, value=(h_r,) * 6, fields=(None, None, None, None, None, top))


P_INITIAL = -61.5
P_TOP = -20.7


def ks_field(grid: Grid, seed: int, sigma: float, corr: Tuple[float, float, float] = (16.0, 16.0, 4.0),
             ks_mean: float = 9.44e-3) -> np.ndarray:
    """Seeded log-normal saturated conductivity, flat array of n cells (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(grid.shape)
    # numpy axes: 0 = z, 1 = y, 2 = x; corr is given as (lx, ly, lz) in cells.
    for axis, ell in ((2, corr[0]), (1, corr[1]), (0, corr[2])):
        rho = math.exp(-1.0 / ell)
        c = math.sqrt(1.0 - rho * rho)
        g = np.moveaxis(g, axis, 0).copy()
        for t in range(1, g.shape[0]):
            g[t] = rho * g[t - 1] + c * g[t]
        g = np.moveaxis(g, 0, axis)
    logk = math.log10(ks_mean) + sigma * g
    return np.ascontiguousarray(10.0 ** logk).reshape(-1)


def random_pressure(grid: Grid, seed: int, lo: float = -80.0, hi: float = -10.0) -> np.ndarray:
    """Uniform random unsaturated pressure head per cell (test input)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=grid.n)


def dt_schedule(kind: str, nsteps: int) -> List[float]:
    """Time-step schedule: 'ramp1to30' is dt_m = 1 + 29 m / (nsteps-1), else constant."""
    if kind == "ramp1to30":
        if nsteps == 1:
            return [1.0]
        return [1.0 + 29.0 * m / (nsteps - 1) for m in range(nsteps)]
    return [float(kind)] * nsteps


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    kmean: int
    steps: int
    dt: str
    krylov: str  # "fcg" or "fgmres"
    restart: int
    nu: int  # pre = post smoothing sweeps
    mixed: bool
    ks_sigma: float  # 0 = homogeneous
    ks_seed: int
    amg_seed: int
    coarse_max: int = 2000
    smooth_levels: int = 10  # AMG levels whose prolongator is smoothed (10 = all)
    problem: str = "column"  # "column": Dirichlet top, no-flux sides; "paper": Sec. 6 infiltration box


WORKLOADS = {
    "richards16_fp64": Workload("richards16_fp64", 16, KMEAN_ARITH, 5, "1", "fcg", 0, 1, False, 0.0, 0, 1),
    "richards128_fp64": Workload("richards128_fp64", 128, KMEAN_UPSTREAM, 20, "ramp1to30", "fgmres", 30, 2,
                                 False, 0.0, 0, 2, smooth_levels=2),
    "richards256_mixed": Workload("richards256_mixed", 256, KMEAN_HARMONIC, 5, "1", "fcg", 0, 1, True, 1.5, 3, 3,
                                  smooth_levels=2),
    "richards512_mixed": Workload("richards512_mixed", 512, KMEAN_ARITH, 10, "10", "fcg", 0, 1, True, 2.0, 4, 4,
                                  smooth_levels=2),
    # Sec. 6 strong-scaling problem: [0,64]x[0,64]x[0,1] with 800x800x40 nodes
    # (798x798x38 unknowns), upstream mean, GMRES(10), t in [0,2] with 10 steps;
    # h_r (not given in the paper) read as the dry state -61.5 cm of Supplementary D
    "paper_infiltration": Workload("paper_infiltration", 798, KMEAN_UPSTREAM, 10, "0.2", "fgmres", 10, 1, False,
                                   0.0, 0, 6, smooth_levels=2, problem="paper"),
}

PAPER_H_R = -61.5


def workload_inputs(w: Workload, n: Optional[int] = None):
    """Grid, soil, BC, Ks field (or None for homogeneous), initial p, dt list.

    n overrides the grid size (n^3 for the column workloads; n x n x (38 n / 798)
    cells on the paper's 64 x 64 x 1 box, at least 4 layers)."""
    nn = w.n if n is None else n
    if w.problem == "paper":
        nz = max(4, round(38 * nn / 798))
        grid = Grid(nn, nn, nz, 64.0, 64.0, 1.0)
        bc = paper_infiltration_bc(grid, PAPER_H_R)
        p0 = np.full(grid.n, PAPER_H_R)
        return grid, Soil(), bc, None, p0, dt_schedule(w.dt, w.steps)
    grid = Grid(nn, nn, nn)
    ks = ks_field(grid, w.ks_seed, w.ks_sigma) if w.ks_sigma > 0 else None
    p0 = np.full(grid.n, P_INITIAL)
    return grid, Soil(), infiltration_bc(P_TOP), ks, p0, dt_schedule(w.dt, w.steps)
