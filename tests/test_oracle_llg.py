"""Pins of the oracle's LLG right-hand side and integrators (eq. 2, 3, 8)."""
import numpy as np
import pytest

from oracle import MU0
from oracle.llg import Film, anisotropy_field, llg_rhs

GAMMA = 1.76e11


def _macrospin(alpha, Bz, m0):
    # One cubic cell: exchange vanishes (eq. 7 on a single cell) and the self
    # demag field -M/3 is parallel to m, so only the applied field exerts torque.
    return Film((1, 1, 1), 5e-9, 8e5, 1.3e-11, 0.0, alpha, GAMMA, b_ext=(0.0, 0.0, Bz))


def _angles(m):
    return np.arccos(np.clip(m[2], -1, 1)), np.arctan2(m[1], m[0])


@pytest.mark.parametrize("alpha", [0.0, 0.02, 0.3])
def test_macrospin_closed_form(alpha):
    # Closed form of eq. 2 for a constant field B along z:
    #   phi(t) = phi0 + gamma B t / (1 + alpha^2)
    #   tan(theta/2) = tan(theta0/2) exp(-alpha gamma B t / (1 + alpha^2))
    Bz = 0.1
    th0, ph0 = 1.1, 0.3
    m0 = np.array([np.sin(th0) * np.cos(ph0), np.sin(th0) * np.sin(ph0), np.cos(th0)])
    film = _macrospin(alpha, Bz, m0)
    dt, steps = 2e-14, 500
    m = film.run(m0.reshape(3, 1, 1, 1), dt, steps)
    t = dt * steps
    g = GAMMA / (1 + alpha * alpha)
    phi = ph0 + g * Bz * t
    theta = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-alpha * g * Bz * t))
    want = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    assert np.abs(m.reshape(3) - want).max() < 1e-10


def test_rhs_is_tangent_and_gyromagnetic_sign():
    rng = np.random.default_rng(0)
    m = rng.standard_normal((3, 50))
    m /= np.linalg.norm(m, axis=0)
    B = rng.standard_normal((3, 50))
    f = llg_rhs(m, B, 0.1, GAMMA)
    assert np.abs((f * m).sum(axis=0)).max() < 1e-6 * GAMMA * 1e-9 + 1e-3
    # alpha = 0, m = x, B = z: dm/dt = -gamma x cross z = +gamma y
    f = llg_rhs(np.array([1.0, 0, 0]).reshape(3, 1), np.array([0, 0, 1.0]).reshape(3, 1), 0.0, GAMMA)
    assert np.allclose(f.reshape(3), [0, GAMMA, 0])


def _film_small(alpha=0.05):
    return Film((6, 4, 2), 4e-9, 8e5, 1.3e-11, 5e4, alpha, GAMMA, b_ext=(0.01, -0.02, 0.005))


def _state(seed, grid=(6, 4, 2)):
    rng = np.random.default_rng(seed)
    m = np.zeros((3,) + grid)
    m[0] = 1.0
    m += 0.3 * rng.standard_normal(m.shape)
    return m / np.linalg.norm(m, axis=0)


def test_rk4_is_fourth_order_and_euler_first_order():
    film = _film_small()
    m0 = _state(1)
    T = 4e-12
    ref = film.run(m0, T / 512, 512, "rk4")
    e = {}
    for integ, ns in (("rk4", (16, 32)), ("euler", (256, 512))):
        errs = [np.abs(film.run(m0, T / n, n, integ) - ref).max() for n in ns]
        e[integ] = errs[0] / errs[1]
    assert 12.0 < e["rk4"] < 20.0
    assert 1.6 < e["euler"] < 2.5


def test_unit_length_after_steps():
    film = _film_small()
    m = film.run(_state(2), 1e-13, 20, "rk4")
    assert np.abs(np.linalg.norm(m, axis=0) - 1.0).max() < 1e-14
    m = film.run(_state(2), 1e-13, 20, "euler")
    assert np.abs(np.linalg.norm(m, axis=0) - 1.0).max() < 1e-14


def test_anisotropy_field_value():
    # eq. 8 with H_K = 2 Ku / (mu0 Ms): Ku = 5e4, Ms = 8e5 -> H_K = 99471.8 A/m
    m = np.array([0.6, 0.8, 0.0]).reshape(3, 1, 1, 1)
    H = anisotropy_field(m, 8e5, 5e4)
    assert np.isclose(H[0].item(), 0.6 * 1e5 / (MU0 * 8e5), rtol=1e-15)
    assert np.isclose(1e5 / (MU0 * 8e5), 99471.839432, rtol=1e-9)
    assert H[1].item() == 0.0 and H[2].item() == 0.0
