"""Anisotropy, Zeeman, effective field and the LLG right-hand side (FP64).

* Anisotropy, eq. 8: uniaxial with the easy axis along x,
      H_anis = (2 Ku / (mu0 Ms^2)) M_x x^ = (2 Ku / (mu0 Ms)) m_x x^,
  y and z components zero (the reading of the "permutation" remark that the
  anisotropy listing itself follows).  Ku may be a per-cell map.
* Zeeman: H_ext = (b_ext + h(r)) / mu0, with b_ext = mu0 H_ext uniform (tesla)
  and an optional per-cell map h (tesla).
* Effective field, eq. 3: H_eff = H_exch + H_anis + H_demag + H_ext.
* LLG, eq. 2, divided by Ms so that it acts on the unit vector m = M / Ms:
      dm/dt = -gamma/(1 + alpha^2) m x B - alpha gamma/(1 + alpha^2) m x (m x B),
  with B = mu0 H_eff.
* Integrators: the paper's explicit Euler with renormalisation after the step
  (the time loop of the appendix script), and classical RK4 with the same
  renormalisation applied once after the full step (never at the stages).
"""
import numpy as np

from . import MU0
from .demag import FFTDemag, demag_direct
from .exchange import exchange_field
from .tensor import demag_tensor

TERM_EXCHANGE = 1
TERM_ANISOTROPY = 2
TERM_DEMAG = 4
TERM_ZEEMAN = 8
TERM_ALL = 15


def anisotropy_field(m, Ms, Ku):
    """Eq. 8.  Ku: scalar or (nx, ny, nz) map in J/m^3."""
    H = np.zeros_like(np.asarray(m, dtype=np.float64))
    H[0] = 2.0 * np.asarray(Ku, dtype=np.float64) / (MU0 * Ms) * m[0]
    return H


def zeeman_field(shape, b_ext, h_map=None):
    """H_ext in A/m from mu0 H_ext = b_ext (tesla) plus an optional per-cell map (tesla)."""
    H = np.zeros(shape)
    for a in range(3):
        H[a] = b_ext[a] / MU0
    if h_map is not None:
        H += np.asarray(h_map, dtype=np.float64) / MU0
    return H


def llg_rhs(m, B, alpha, gamma):
    """Eq. 2 on unit vectors.  m, B: (3, ...) arrays; B in tesla."""
    mxB = np.cross(m, B, axis=0)
    mxmxB = np.cross(m, mxB, axis=0)
    g = gamma / (1.0 + alpha * alpha)
    return -g * mxB - alpha * g * mxmxB


def normalise(m):
    return m / np.sqrt((m * m).sum(axis=0, keepdims=True))


class Film:
    """One film of nx x ny x nz cubic cells: parameters + precomputed tensor.

    Parameters follow the solver's SI conventions; ``ku_map`` (nx, ny, nz) and
    ``h_map`` (3, nx, ny, nz) are optional per-cell maps in paper order.
    ``demag`` chooses the convolution route: "fft" (eq. 14) or "direct" (eq. 13).
    """

    def __init__(self, grid, delta, Ms, A, Ku, alpha, gamma, b_ext=(0.0, 0.0, 0.0),
                 h_map=None, ku_map=None, self_term=True, demag="fft"):
        self.grid = tuple(int(g) for g in grid)
        self.delta, self.Ms, self.A, self.Ku = float(delta), float(Ms), float(A), float(Ku)
        self.alpha, self.gamma = float(alpha), float(gamma)
        self.b_ext = tuple(float(b) for b in b_ext)
        self.h_map = None if h_map is None else np.asarray(h_map, dtype=np.float64)
        self.ku_map = None if ku_map is None else np.asarray(ku_map, dtype=np.float64)
        nx, ny, nz = self.grid
        self.K = demag_tensor(nx, ny, nz, self.delta, self_term=self_term)
        self.route = demag
        self._fft = FFTDemag(nx, ny, nz, self.K) if demag == "fft" else None

    # --- field terms -----------------------------------------------------
    def h_demag(self, m):
        if self.route == "fft":
            return self._fft.field(m, self.Ms)
        return demag_direct(m, self.Ms, self.K)

    def h_exchange(self, m):
        return exchange_field(m, self.Ms, self.A, self.delta)

    def h_anisotropy(self, m):
        ku = self.Ku if self.ku_map is None else self.ku_map
        return anisotropy_field(m, self.Ms, ku)

    def h_zeeman(self, m):
        return zeeman_field(m.shape, self.b_ext, self.h_map)

    def h_eff(self, m, terms=TERM_ALL):
        """Eq. 3 (A/m), restricted to the terms selected by the bit mask."""
        m = np.asarray(m, dtype=np.float64)
        H = np.zeros_like(m)
        if terms & TERM_EXCHANGE:
            H += self.h_exchange(m)
        if terms & TERM_ANISOTROPY:
            H += self.h_anisotropy(m)
        if terms & TERM_DEMAG:
            H += self.h_demag(m)
        if terms & TERM_ZEEMAN:
            H += self.h_zeeman(m)
        return H

    # --- dynamics ----------------------------------------------------------
    def rhs(self, m):
        return llg_rhs(m, MU0 * self.h_eff(m), self.alpha, self.gamma)

    def euler_step(self, m, dt):
        return normalise(m + dt * self.rhs(m))

    def rk4_step(self, m, dt):
        k1 = self.rhs(m)
        k2 = self.rhs(m + 0.5 * dt * k1)
        k3 = self.rhs(m + 0.5 * dt * k2)
        k4 = self.rhs(m + dt * k3)
        return normalise(m + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4))

    def run(self, m, dt, steps, integrator="rk4", sample_every=0, callback=None):
        """Advance ``steps`` steps; optionally call callback(step, m) every sample_every."""
        m = np.asarray(m, dtype=np.float64)
        step = self.rk4_step if integrator == "rk4" else self.euler_step
        for s in range(1, steps + 1):
            m = step(m, dt)
            if sample_every and callback is not None and s % sample_every == 0:
                callback(s, m)
        return m

    # --- observables -----------------------------------------------------
    def mean_m(self, m):
        return np.asarray(m, dtype=np.float64).reshape(3, -1).mean(axis=1)

    def max_dmdt(self, m):
        f = self.rhs(np.asarray(m, dtype=np.float64))
        return float(np.sqrt((f * f).sum(axis=0)).max())
