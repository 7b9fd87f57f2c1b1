"""Seeded synthetic workloads for the finite-difference LLG solver.

This module only draws random numbers and builds parameter records.  It holds
none of the method's arithmetic (no fields, no tensor, no integrator), so both
the CUDA path and the FP64 CPU oracle can take their inputs from here.

The workloads stand in for the paper's test problems (the muMAG standard
problem #4 thin film of Section 3 and the muMAG standard problem #3 cube used
for Table 1): same kind of geometry and material, seeded synthetic initial
states, no external data.

Conventions
-----------
* SI units throughout: delta in m, Ms in A/m, A in J/m, Ku in J/m^3, gamma in
  rad/(s T), b_ext (= mu0 H_ext) in tesla, dt in s.
* A magnetisation state is the unit vector field m = M / Ms, returned as a
  float32 array of shape (3, nz, ny, nx) (C order, x fastest), i.e. the
  device layout [3][nz][ny][nx].  States are generated in float64 and rounded
  to float32 once, so that every consumer sees the same rounded values.
* Seeds: workload ``c`` draws from ``numpy.random.default_rng(1000 * c + s)``;
  film ``b`` of the batched workload draws from ``default_rng(4000 + b)``.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Material:
    Ms: float = 8.0e5        # A/m
    A: float = 1.3e-11       # J/m
    Ku: float = 0.0          # J/m^3, easy axis x
    alpha: float = 0.02
    gamma: float = 1.76e11   # rad/(s T)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    grid: Tuple[int, int, int]          # (nx, ny, nz)
    delta: float                        # cubic cell edge, m
    mat: Material
    b_ext: Tuple[float, float, float]   # mu0 H_ext, tesla
    dt: float                           # s
    steps: int
    init: str                           # initial-state recipe name
    seed: int

    @property
    def ncells(self) -> int:
        nx, ny, nz = self.grid
        return nx * ny * nz


def thin_film_small() -> Workload:
    """40x10x1 cells of 5 nm (a 200x50x5 nm film), RK4 dt=1e-13 s, 10,000 steps."""
    return Workload("film_40x10x1", (40, 10, 1), 5e-9,
                    Material(Ms=8.0e5, A=1.3e-11, Ku=0.0, alpha=0.02, gamma=1.76e11),
                    (-20e-3, 5e-3, 0.0), 1e-13, 10_000, "tilted_x", 1000 * 1)


def film_256x256x16() -> Workload:
    """256x256x16 cells of 4 nm, Ku=5e4 J/m^3 along x, alpha=0.05, RK4 dt=5e-14 s, 2,000 steps."""
    return Workload("film_256x256x16", (256, 256, 16), 4e-9,
                    Material(Ms=8.0e5, A=1.3e-11, Ku=5e4, alpha=0.05, gamma=1.76e11),
                    (0.0, 0.0, 10e-3), 5e-14, 2_000, "random", 1000 * 2)


def film_512x512x8() -> Workload:
    """512x512x8 cells of 4 nm, vortex-like start, no applied field (precision study)."""
    return Workload("film_512x512x8", (512, 512, 8), 4e-9,
                    Material(Ms=8.0e5, A=1.3e-11, Ku=0.0, alpha=0.02, gamma=1.76e11),
                    (0.0, 0.0, 0.0), 1e-13, 200, "vortex", 1000 * 3)


def film_128x128x4() -> Workload:
    """128x128x4 cells of 4 nm (the differentiation study), RK4 dt=1e-13 s, 500 steps."""
    return Workload("film_128x128x4", (128, 128, 4), 4e-9,
                    Material(Ms=8.0e5, A=1.3e-11, Ku=0.0, alpha=0.02, gamma=1.76e11),
                    (0.0, 0.0, 0.0), 1e-13, 500, "tilted_x", 1000 * 5)


def film_16x8x1() -> Workload:
    """16x8x1 copy of the differentiation study, small enough for finite differences."""
    return Workload("film_16x8x1", (16, 8, 1), 4e-9,
                    Material(Ms=8.0e5, A=1.3e-11, Ku=0.0, alpha=0.02, gamma=1.76e11),
                    (0.0, 0.0, 0.0), 1e-13, 500, "tilted_x", 1000 * 5 + 1)


WORKLOADS = {
    w.name: w for w in (thin_film_small(), film_256x256x16(), film_512x512x8(),
                        film_128x128x4(), film_16x8x1())
}


# ---------------------------------------------------------------------------
# initial states
# ---------------------------------------------------------------------------

def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.sqrt((v * v).sum(axis=0, keepdims=True))


def initial_state(recipe: str, grid: Tuple[int, int, int], seed: int) -> np.ndarray:
    """Return a seeded unit-vector field, float32, shape (3, nz, ny, nx).

    recipes
      ``tilted_x``  unit((1, 0.1, 0) + U(-0.01, 0.01)^3) per cell
      ``random``    unit(N(0, I_3)) per cell
      ``vortex``    unit((-y, x, 0.1) / |(-y, x, 0.1)| + U(-0.02, 0.02)^3), with x, y
                    the cell-centre coordinates relative to the film centre divided
                    by the half-widths (so both lie in [-1, 1])
      ``uniform_x`` (1, 0, 0) everywhere (no randomness)
    """
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    shape = (3, nz, ny, nx)
    if recipe == "tilted_x":
        v = np.empty(shape)
        v[0], v[1], v[2] = 1.0, 0.1, 0.0
        v += rng.uniform(-0.01, 0.01, size=shape)
    elif recipe == "random":
        v = rng.standard_normal(size=shape)
    elif recipe == "vortex":
        xs = (np.arange(nx) + 0.5 - nx / 2.0) / (nx / 2.0)
        ys = (np.arange(ny) + 0.5 - ny / 2.0) / (ny / 2.0)
        X = np.broadcast_to(xs[None, None, :], (nz, ny, nx))
        Y = np.broadcast_to(ys[None, :, None], (nz, ny, nx))
        v = np.empty(shape)
        v[0], v[1], v[2] = -Y, X, 0.1
        v = _unit(v)
        v += rng.uniform(-0.02, 0.02, size=shape)
    elif recipe == "uniform_x":
        v = np.zeros(shape)
        v[0] = 1.0
    else:
        raise ValueError(f"unknown initial-state recipe {recipe!r}")
    return np.ascontiguousarray(_unit(v).astype(np.float32))


def workload_state(w: Workload) -> np.ndarray:
    return initial_state(w.init, w.grid, w.seed)


def random_state(grid: Tuple[int, int, int], seed: int) -> np.ndarray:
    """Random unit vectors (the ``random`` recipe) on an arbitrary grid."""
    return initial_state("random", grid, seed)


# ---------------------------------------------------------------------------
# per-cell maps of the differentiation study
# ---------------------------------------------------------------------------

def zeeman_map(grid: Tuple[int, int, int], seed: int, sigma_T: float = 5e-3) -> np.ndarray:
    """Per-cell applied field h (tesla), i.i.d. N(0, sigma) per component; (3, nz, ny, nx) float32."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.normal(0.0, sigma_T, size=(3, nz, ny, nx)).astype(np.float32))


def ku_map(grid: Tuple[int, int, int], seed: int, ku_max: float = 1e5) -> np.ndarray:
    """Per-cell anisotropy constant Ku (J/m^3), U[0, ku_max]; shape (nz, ny, nx) float32."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(0.0, ku_max, size=(nz, ny, nx)).astype(np.float32))


# ---------------------------------------------------------------------------
# batched films (hysteresis sweep)
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Film:
    index: int
    grid: Tuple[int, int, int]
    b_ext: Tuple[float, float, float]
    seed: int


def film_batch(nfilms: int = 256, nx_range=(32, 256), ny_range=(8, 128),
               nz_range=(1, 4), sweep_mT=(-50.0, 50.0)) -> list:
    """Independent films of uneven size, each with its own field along x.

    Sizes are drawn by ``default_rng(4)``; film b's field is swept linearly from
    sweep_mT[0] to sweep_mT[1] over the batch; film b's state seed is 4000 + b.
    """
    rng = np.random.default_rng(4)
    nxs = rng.integers(nx_range[0], nx_range[1] + 1, size=nfilms)
    nys = rng.integers(ny_range[0], ny_range[1] + 1, size=nfilms)
    nzs = rng.integers(nz_range[0], nz_range[1] + 1, size=nfilms)
    films = []
    for b in range(nfilms):
        frac = b / (nfilms - 1) if nfilms > 1 else 0.0
        bx = (sweep_mT[0] + (sweep_mT[1] - sweep_mT[0]) * frac) * 1e-3
        films.append(Film(b, (int(nxs[b]), int(nys[b]), int(nzs[b])), (bx, 0.0, 0.0), 4000 + b))
    return films


BATCH_MATERIAL = Material(Ms=8.0e5, A=1.3e-11, Ku=0.0, alpha=0.5, gamma=1.76e11)
BATCH_DELTA = 5e-9
BATCH_DT = 1e-13


# ---------------------------------------------------------------------------
# the standard-problem-4 protocol (Section 3, script of Appendix A)
# ---------------------------------------------------------------------------

_MU0 = 4.0e-7 * np.pi     # only to convert the schedule's kA/m values to tesla
_KAM = 1e3 * _MU0         # 1 kA/m of H as mu0 H, tesla


def sp4_film() -> Workload:
    """The paper's validation film: 500x125x3 nm as 166x42x1 cells of 3 nm,
    Ms 800 kA/m, A 1.3e-11 J/m, no anisotropy, damping 0.5 while relaxing,
    explicit Euler with dt = 5 fs for 150,000 steps, starting along x.
    gamma = 2.21e5 / mu0 is the gyromagnetic ratio the script's LLG prefactor
    (0.221 in its nm/ns/kA/m units) stands for."""
    return Workload("sp4_166x42x1", (166, 42, 1), 3e-9,
                    Material(Ms=8.0e5, A=1.3e-11, Ku=0.0, alpha=0.5, gamma=2.21e5 / _MU0),
                    (0.0, 0.0, 0.0), 5e-15, 150000, "uniform_x", 0)


def sp4_schedule(dt: float, n_sat: int = 4000, n_ramp: int = 6000, n_rev: int = 50000,
                 n_end: int = 150000, h_sat_kam: float = 100.0,
                 h_rev_kam=(-19.576, 3.422, 0.0), alpha_relax: float = 0.5,
                 alpha_rev: float = 0.02) -> list:
    """Field program segments (t_begin, t_end, b_begin, b_end, alpha) of the
    standard-problem-4 protocol, times in s and fields in tesla.

    The script counts steps t = 1, 2, ... and its step t moves the state from
    time (t - 1) dt to t dt with the field of index t; the segments below put
    that field at the step's start time n dt, n = t - 1:
      t < n_sat               h_sat along each of x, y, z            (saturate)
      n_sat <= t < n_ramp     h_sat (n_ramp - t) / (n_ramp - n_sat)   on each
                              component (the script's /20 for the default
                              2000-step ramp)                          (ramp down)
      n_ramp <= t <= n_rev    zero field
      t > n_rev               h_rev, damping alpha_rev                (reverse)
    Reading: the script's ramp lines add the ramp three times to H_x and none
    to H_y, H_z; the text says the saturating field along (1, 1, 1) is slowly
    reduced, so the ramp applies to each component (continuous with the
    saturation phase).  The discontinuous switch to the reverse field sits half
    a step before step index n_rev + 1 so that no rounding of the clock can move
    it by a step; the continuous ramp ends stay on step times.
    """
    sat = (h_sat_kam * _KAM,) * 3
    zero = (0.0, 0.0, 0.0)
    rev = tuple(h * _KAM for h in h_rev_kam)
    t_sat, t_ramp, t_rev = (n_sat - 1) * dt, (n_ramp - 1) * dt, (n_rev - 0.5) * dt
    return [
        (0.0, t_sat, sat, sat, alpha_relax),
        (t_sat, t_ramp, sat, zero, alpha_relax),
        (t_ramp, t_rev, zero, zero, alpha_relax),
        (t_rev, (n_end + 1) * dt, rev, rev, alpha_rev),
    ]


# ---------------------------------------------------------------------------
# the standard-problem-3 cube (Section 3, Table 1)
# ---------------------------------------------------------------------------

SP3_EDGE_LEX = 8.5   # cube edge in exchange lengths, near the flower/vortex crossover of the problem


def sp3_cube(n: int) -> Workload:
    """The paper's timing problem: an n x n x n cube, A 1e-11 J/m, Ms 1000 kA/m,
    anisotropy field 100 kA/m (Ku = mu0 Ms H_K / 2, easy axis x as in the
    paper's anisotropy code), large damping (1.0), explicit Euler.  The paper
    does not give the cube's size; it is taken as 8.5 exchange lengths
    (l_ex = sqrt(2A / (mu0 Ms^2)) = 3.99 nm), cut into n^3 cells.  dt keeps
    gamma * (largest exchange field) * dt at 0.05 so that every n is stable."""
    Ms, A, HK = 1.0e6, 1.0e-11, 1.0e5
    lex = np.sqrt(2.0 * A / (_MU0 * Ms * Ms))
    delta = SP3_EDGE_LEX * lex / n
    b_ex = 12.0 * A / (Ms * delta * delta)   # tesla: 6 neighbours of 2A/(Ms delta^2) at opposite sign
    dt = 0.05 / (1.76e11 * b_ex)
    return Workload(f"sp3_cube_{n}", (n, n, n), delta,
                    Material(Ms=Ms, A=A, Ku=0.5 * _MU0 * Ms * HK, alpha=1.0, gamma=1.76e11),
                    (0.0, 0.0, 0.0), dt, 1000, "vortex", 3000 + n)
