"""Pins of the oracle's hand-written adjoint against central finite differences
of its own forward RK4 trajectory (FP64), on random directions and single
entries of the initial state, the per-cell field map and the per-cell Ku map."""
import numpy as np
import pytest

from oracle.adjoint import AdjointFilm
from oracle.llg import Film

GRID = (6, 4, 2)
DT = 1e-13
STEPS = 6


def _setup(seed=0):
    rng = np.random.default_rng(seed)
    m0 = rng.standard_normal((3,) + GRID)
    m0 /= np.linalg.norm(m0, axis=0)
    h = rng.normal(0.0, 5e-3, size=(3,) + GRID)
    ku = rng.uniform(0.0, 1e5, size=GRID)
    w = rng.standard_normal((3,) + GRID)
    return m0, h, ku, w


def _loss(m0, h, ku, w):
    film = Film(GRID, 4e-9, 8e5, 1.3e-11, 0.0, 0.1, 1.76e11, b_ext=(0.01, 0.0, -0.005), h_map=h, ku_map=ku)
    m = film.run(m0, DT, STEPS)
    return float((w * m).sum())


def _grads(m0, h, ku, w):
    film = Film(GRID, 4e-9, 8e5, 1.3e-11, 0.0, 0.1, 1.76e11, b_ext=(0.01, 0.0, -0.005), h_map=h, ku_map=ku)
    adj = AdjointFilm(film)
    _, rec = adj.forward(m0, DT, STEPS)
    return adj.backward(rec, DT, w)


@pytest.fixture(scope="module")
def case():
    m0, h, ku, w = _setup()
    return (m0, h, ku, w), _grads(m0, h, ku, w)


def _fd(f, x, d, eps):
    return (f(x + eps * d) - f(x - eps * d)) / (2 * eps)


def test_initial_state_gradient(case):
    (m0, h, ku, w), (gm, gh, gk) = case
    rng = np.random.default_rng(1)
    for _ in range(3):
        d = rng.standard_normal(m0.shape)
        fd = _fd(lambda x: _loss(x, h, ku, w), m0, d, 1e-6)
        assert abs((gm * d).sum() - fd) <= 1e-6 * abs(fd) + 1e-12
    for idx in [(0, 0, 0, 0), (1, 3, 2, 1), (2, 5, 0, 1)]:
        d = np.zeros_like(m0)
        d[idx] = 1.0
        fd = _fd(lambda x: _loss(x, h, ku, w), m0, d, 1e-6)
        assert abs(gm[idx] - fd) <= 1e-6 * np.abs(gm).max()


def test_field_map_gradient(case):
    (m0, h, ku, w), (gm, gh, gk) = case
    rng = np.random.default_rng(2)
    for _ in range(3):
        d = rng.normal(0.0, 5e-3, size=h.shape)
        fd = _fd(lambda x: _loss(m0, x, ku, w), h, d, 1e-3)
        assert abs((gh * d).sum() - fd) <= 1e-6 * abs(fd) + 1e-12
    for idx in [(0, 1, 1, 0), (2, 4, 3, 1)]:
        d = np.zeros_like(h)
        d[idx] = 1e-3
        fd = _fd(lambda x: _loss(m0, x, ku, w), h, d, 1.0)
        assert abs(gh[idx] * 1e-3 - fd) <= 1e-6 * np.abs(gh).max() * 1e-3


def test_ku_map_gradient(case):
    (m0, h, ku, w), (gm, gh, gk) = case
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.uniform(-1e4, 1e4, size=ku.shape)
        fd = _fd(lambda x: _loss(m0, h, x, w), ku, d, 1e-2)
        assert abs((gk * d).sum() - fd) <= 1e-6 * abs(fd) + 1e-15
