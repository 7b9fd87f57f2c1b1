"""Energies of eq. 1, discretised on the cell grid (FP64, joules).

    E_exch = A delta * sum over unordered neighbour pairs |m_i - m_j|^2
    E_anis = Ku delta^3 * sum (m_y^2 + m_z^2)               (easy axis x)
    E_demag = -1/2 mu0 delta^3 * sum M . H_demag
    E_zeeman = -mu0 delta^3 * sum M . H_ext

Eq. 1 prints the x component three times in its exchange term; it is read as
the sum over x, y and z.  The pair sum is the discrete energy whose gradient
is the eq. 5/7 stencil: for unit vectors it equals -1/2 mu0 delta^3 sum M . H_exch
(neighbours missing at a boundary contribute nothing, as in eq. 7).
"""
import numpy as np

from . import MU0


def exchange_energy_pairs(m, A, delta):
    m = np.asarray(m, dtype=np.float64)
    e = 0.0
    for ax in (1, 2, 3):
        d = np.diff(m, axis=ax)
        e += float((d * d).sum())
    return A * delta * e


def energies(film, m):
    """(E_exch, E_anis, E_demag, E_zeeman, E_total) in J for the oracle Film."""
    m = np.asarray(m, dtype=np.float64)
    d3 = film.delta ** 3
    Ms = film.Ms
    e_ex = exchange_energy_pairs(m, film.A, film.delta)
    ku = film.Ku if film.ku_map is None else film.ku_map
    e_an = float((np.asarray(ku) * (m[1] ** 2 + m[2] ** 2)).sum() * d3)
    e_d = float(-0.5 * MU0 * d3 * (Ms * m * film.h_demag(m)).sum())
    e_z = float(-MU0 * d3 * (Ms * m * film.h_zeeman(m)).sum())
    return (e_ex, e_an, e_d, e_z, e_ex + e_an + e_d + e_z)
