"""Plain FP64 CPU oracle of the finite-difference LLG method (arXiv:1501.07293).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The product path (the CUDA library and its Python binding) never calls it and
shares no code, constant or helper with it.

Every function follows the paper's own definitions in float64, written for a
reader who checks it against the paper by eye: no blocking, fusion or
reordering beyond what the definition states.  Library primitives (numpy
arithmetic, ``scipy.fft.fftn`` on all host cores) serve as steps.

Array convention of the oracle: a vector field is an array of shape
(3, nx, ny, nz) indexed [component, i, j, k] with i along x, as in the paper's
M(i, j, k).  (The device layout [3][nz][ny][nx] is the same data transposed;
``to_xyz`` / ``to_device`` convert.)

Which pin checks which function (tests/test_oracle_*.py, ``-m "not gpu"``):
  tensor.py    self term -I/3, trace identity, parities and axis permutations,
               far-field point-dipole limit, delta independence,
               uniformly magnetised slab / rod limits
  demag.py     brute force eq. 13 == FFT route eq. 14; the field of a
               uniformly magnetised box equals an independent surface-charge
               quadrature
  exchange.py  uniform field -> 0, linear ramp boundary values of eq. 7,
               Neumann cosine eigenvectors, hand-computed impulse response
  llg.py       macrospin closed-form precession and damping, RK4 order 4 and
               Euler order 1, |m| = 1 after renormalisation
  energy.py    pair-sum identity of the exchange energy, energy decay with
               damping, dE/dt = -mu0 Ms delta^3 sum H . dm/dt
  program.py   the appendix script's schedule conditions per step index,
               macrospin closed form under ramps and a damping switch,
               constant program == constant field, Euler across a switch
               == concatenated constant runs
  adjoint.py   central finite differences of the oracle's own trajectory
Parity unpinned: nothing in this oracle is checked against a printed
trajectory (the paper's Fig. 3 comparison with OOMMF has no data in the text).
"""
import numpy as np

MU0 = 4.0e-7 * np.pi   # vacuum permeability, SI (exact by the pre-2019 definition)


def to_xyz(a_dev):
    """(3, nz, ny, nx) device-order array -> (3, nx, ny, nz) float64 paper order."""
    a = np.asarray(a_dev, dtype=np.float64)
    if a.ndim == 3:
        return np.ascontiguousarray(a.transpose(2, 1, 0))
    return np.ascontiguousarray(a.transpose(0, 3, 2, 1))


def to_device(a_xyz):
    """(3, nx, ny, nz) paper-order array -> (3, nz, ny, nx) device order (float64)."""
    a = np.asarray(a_xyz, dtype=np.float64)
    if a.ndim == 3:
        return np.ascontiguousarray(a.transpose(2, 1, 0))
    return np.ascontiguousarray(a.transpose(0, 3, 2, 1))
