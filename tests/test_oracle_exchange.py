"""Pins of the oracle's exchange field (Section 2.1, eq. 5 with the Neumann rule eq. 6/7)."""
import os

import numpy as np
import pytest

from oracle import MU0
from oracle.exchange import exchange_field

Ms, A, D = 8e5, 1.3e-11, 5e-9
C = 2.0 * A / (MU0 * Ms * D * D)   # H per unit of sum(m_nb - m)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "exchange_impulse_3x3x3.txt")


def test_uniform_state_has_no_exchange_field():
    m = np.zeros((3, 5, 4, 3))
    m[0], m[1], m[2] = 0.6, 0.0, 0.8
    assert np.abs(exchange_field(m, Ms, A, D)).max() == 0.0


def test_linear_ramp_boundary_values():
    # eq. 7: at i = 1 the second difference becomes (M(2) - M(1)) / delta^2.
    n = 7
    slope = 0.01
    m = np.zeros((3, n, 3, 2))
    m[1] = (slope * np.arange(n))[:, None, None]
    H = exchange_field(m, Ms, A, D)
    assert np.allclose(H[1, 1:-1], 0.0, atol=1e-9 * C)
    assert np.allclose(H[1, 0], C * slope, rtol=1e-13)
    assert np.allclose(H[1, -1], -C * slope, rtol=1e-13)
    assert np.abs(H[0]).max() == 0.0 and np.abs(H[2]).max() == 0.0


@pytest.mark.parametrize("n,k", [(8, 1), (8, 3), (5, 4), (16, 7)])
def test_neumann_cosine_eigenvectors(n, k):
    # The cell-centred Neumann second difference has eigenvectors
    # cos(pi k (i + 1/2) / n) with eigenvalues -4 sin^2(pi k / (2 n)).
    i = np.arange(n)
    v = np.cos(np.pi * k * (i + 0.5) / n)
    lam = -4.0 * np.sin(np.pi * k / (2 * n)) ** 2
    for ax in range(3):
        shape = [1, 1, 1]
        shape[ax] = n
        m = np.zeros((3,) + tuple(shape))
        m[2] = v.reshape(shape)
        H = exchange_field(m, Ms, A, D)
        assert np.allclose(H[2], C * lam * m[2], atol=1e-12 * C)


def test_separable_eigenvector_3d():
    nx, ny, nz = 6, 5, 4
    kx, ky, kz = 2, 1, 3
    vx = np.cos(np.pi * kx * (np.arange(nx) + 0.5) / nx)
    vy = np.cos(np.pi * ky * (np.arange(ny) + 0.5) / ny)
    vz = np.cos(np.pi * kz * (np.arange(nz) + 0.5) / nz)
    lam = sum(-4.0 * np.sin(np.pi * k / (2 * n)) ** 2 for k, n in ((kx, nx), (ky, ny), (kz, nz)))
    m = np.zeros((3, nx, ny, nz))
    m[0] = vx[:, None, None] * vy[None, :, None] * vz[None, None, :]
    H = exchange_field(m, Ms, A, D)
    assert np.allclose(H[0], C * lam * m[0], atol=1e-12 * C)


def test_impulse_response_golden():
    rows = np.loadtxt(GOLDEN, comments="#")
    for src in {tuple(int(v) for v in r[:3]) for r in rows}:
        m = np.zeros((3, 3, 3, 3))
        m[(0,) + src] = 1.0
        H = exchange_field(m, Ms, A, D) / C
        want = np.zeros((3, 3, 3))
        for r in rows:
            if tuple(int(v) for v in r[:3]) == src:
                want[int(r[3]), int(r[4]), int(r[5])] = r[6]
        assert np.allclose(H[0], want, atol=1e-13)
        assert np.abs(H[1:]).max() == 0.0


def test_operator_is_symmetric():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((3, 5, 4, 3))
    b = rng.standard_normal((3, 5, 4, 3))
    La = exchange_field(a, Ms, A, D)
    Lb = exchange_field(b, Ms, A, D)
    assert abs((a * Lb).sum() - (La * b).sum()) < 1e-12 * np.abs(La).max() * a.size
