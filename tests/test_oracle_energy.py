"""Pins of the oracle's energies (eq. 1) against the field (eq. 3) and the dynamics (eq. 2)."""
import numpy as np

from oracle import MU0
from oracle.energy import energies, exchange_energy_pairs
from oracle.llg import Film


def _state(seed, grid):
    rng = np.random.default_rng(seed)
    m = np.zeros((3,) + grid)
    m[0] = 1.0
    m += 0.5 * rng.standard_normal(m.shape)
    return m / np.linalg.norm(m, axis=0)


def test_exchange_pair_sum_equals_field_form():
    film = Film((5, 4, 3), 4e-9, 8e5, 1.3e-11, 0.0, 0.1, 1.76e11)
    m = _state(0, (5, 4, 3))
    e_pairs = exchange_energy_pairs(m, film.A, film.delta)
    e_field = -0.5 * MU0 * film.delta ** 3 * (film.Ms * m * film.h_exchange(m)).sum()
    assert abs(e_pairs - e_field) < 1e-12 * abs(e_pairs)


def test_single_cell_demag_energy():
    # Uniformly magnetised cube: E_d = 1/2 mu0 N Ms^2 V with N = 1/3.
    film = Film((1, 1, 1), 5e-9, 8e5, 1.3e-11, 0.0, 0.1, 1.76e11)
    m = np.array([0.0, 0.6, 0.8]).reshape(3, 1, 1, 1)
    e = energies(film, m)
    assert np.isclose(e[2], 0.5 * MU0 * 8e5 ** 2 * (5e-9) ** 3 / 3.0, rtol=1e-13)


def test_energy_rate_matches_field():
    # dE/dt = sum_i dE/dm_i . dm_i/dt = -mu0 Ms delta^3 sum H_eff . dm/dt
    film = Film((6, 5, 2), 4e-9, 8e5, 1.3e-11, 5e4, 0.1, 1.76e11, b_ext=(0.02, 0.01, -0.01))
    m = _state(1, (6, 5, 2))
    f = film.rhs(m)
    h = 1e-16
    dE = (energies(film, m + h * f)[4] - energies(film, m - h * f)[4]) / (2 * h)
    want = -MU0 * film.Ms * film.delta ** 3 * (film.h_eff(m) * f).sum()
    assert abs(dE - want) < 1e-6 * abs(want)
    assert want < 0.0


def test_energy_decays_with_damping():
    film = Film((8, 6, 2), 4e-9, 8e5, 1.3e-11, 5e4, 0.05, 1.76e11, b_ext=(0.0, 0.0, 0.01))
    m = _state(2, (8, 6, 2))
    E = [energies(film, m)[4]]
    for _ in range(12):
        m = film.run(m, 5e-14, 10)
        E.append(energies(film, m)[4])
    dE = np.diff(E)
    assert np.all(dE <= 1e-12 * abs(E[0]))
