"""Pins of the oracle's demagnetising field (Section 2.3, eq. 12-14).

* The FFT route (eq. 14 with the paper's 2n zero padding) equals the brute
  force double sum (eq. 13) on small grids of odd and degenerate shapes.
* The field of uniformly magnetised samples and of a single magnetised cell
  equals an independent quadrature of the Coulomb field of the surface
  charges sigma = M . n (scipy dblquad), which fixes the tensor's sign,
  prefactor and the convolution's index order without using eq. 10/11.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle.demag import demag_at_cells, demag_direct, demag_fft
from oracle.tensor import demag_tensor


def _random_unit(shape, seed):
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((3,) + shape)
    return m / np.linalg.norm(m, axis=0)


@pytest.mark.parametrize("grid", [(5, 4, 3), (7, 1, 1), (1, 6, 1), (3, 5, 2), (1, 1, 1), (8, 6, 3)])
def test_fft_route_equals_direct_sum(grid):
    m = _random_unit(grid, 11)
    K = demag_tensor(*grid)
    Hd = demag_direct(m, 8e5, K)
    Hf = demag_fft(m, 8e5, K)
    assert np.abs(Hd - Hf).max() <= 1e-13 * np.abs(Hd).max()


def _surface_charge_field(lo, hi, p, a):
    """Field (per unit M) at p of a box magnetised along axis a, from its two charged faces."""
    H = np.zeros(3)
    b, c = [ax for ax in range(3) if ax != a]
    for face, sig in ((hi[a], 1.0), (lo[a], -1.0)):
        for comp in range(3):
            def f(v, u):
                r = np.zeros(3)
                r[a], r[b], r[c] = face, u, v
                d = p - r
                return sig * d[comp] / np.linalg.norm(d) ** 3
            val, _ = integrate.dblquad(f, lo[b], hi[b], lo[c], hi[c], epsabs=1e-13, epsrel=1e-11)
            H[comp] += val / (4.0 * np.pi)
    return H


@pytest.mark.parametrize("a", [0, 1, 2])
def test_uniform_box_matches_surface_charges(a):
    nx, ny, nz = 6, 4, 3
    d = 2.5e-9
    K = demag_tensor(nx, ny, nz, d)
    m = np.zeros((3, nx, ny, nz))
    m[a] = 1.0
    Ms = 8e5
    H = demag_fft(m, Ms, K)
    lo, hi = np.zeros(3), np.array([nx, ny, nz], float)
    for cell in [(0, 0, 0), (2, 1, 1), (5, 3, 2), (4, 0, 1)]:
        p = np.array(cell, float) + 0.5
        Hq = Ms * _surface_charge_field(lo, hi, p, a)
        assert np.abs(H[(slice(None),) + cell] - Hq).max() < 1e-9 * Ms


def test_single_cell_source_matches_surface_charges():
    nx, ny, nz = 5, 4, 3
    K = demag_tensor(nx, ny, nz)
    src = (1, 2, 0)
    for a in range(3):
        m = np.zeros((3, nx, ny, nz))
        m[(a,) + src] = 1.0
        H = demag_direct(m, 1.0, K)
        for tgt in [(1, 2, 0), (4, 0, 2), (0, 3, 1), (3, 2, 0)]:
            # target at the origin; the source cell spans src - tgt -/+ 1/2
            off = np.array(src, float) - np.array(tgt, float)
            Hq = _surface_charge_field(off - 0.5, off + 0.5, np.zeros(3), a)
            assert np.abs(H[(slice(None),) + tgt] - Hq).max() < 1e-10


def test_demag_is_linear_and_symmetric():
    # <a, K b> = <K a, b>: the discrete operator is symmetric (used by the adjoint).
    grid = (4, 3, 2)
    K = demag_tensor(*grid)
    a = _random_unit(grid, 1)
    b = _random_unit(grid, 2)
    Ka = demag_fft(a, 1.0, K)
    Kb = demag_fft(b, 1.0, K)
    assert abs((a * Kb).sum() - (Ka * b).sum()) < 1e-13
    assert np.allclose(demag_fft(2.0 * a + b, 1.0, K), 2.0 * Ka + Kb, atol=1e-13)


@pytest.mark.parametrize("grid", [(5, 4, 3), (7, 1, 1), (1, 6, 1), (1, 1, 5), (3, 5, 2), (1, 1, 1)])
@pytest.mark.parametrize("self_term", [True, False])
def test_demag_at_cells_equals_direct_sum_everywhere(grid, self_term):
    # the sampled route of eq. 13 (used for full-size parity) is the same sum as the
    # brute force at every cell, for both readings of the self offset
    m = _random_unit(grid, 5)
    K = demag_tensor(*grid, self_term=self_term)
    Hd = demag_direct(m, 8e5, K)
    cells = [(i, j, k) for i in range(grid[0]) for j in range(grid[1]) for k in range(grid[2])]
    Hc = demag_at_cells(m, 8e5, cells, self_term=self_term)
    ref = np.array([Hd[(slice(None),) + c] for c in cells])
    assert np.abs(Hc - ref).max() <= 1e-13 * np.abs(Hd).max()


def test_demag_at_cells_self_term_is_minus_third_of_M():
    # a single cell: with the self offset H = -M/3 (the cube's demagnetising factors),
    # without it H = 0
    m = np.zeros((3, 1, 1, 1))
    m[:, 0, 0, 0] = [0.6, -0.8, 0.0]
    H = demag_at_cells(m, 8e5, [(0, 0, 0)])[0]
    assert np.abs(H + 8e5 * m[:, 0, 0, 0] / 3).max() <= 1e-9
    assert np.abs(demag_at_cells(m, 8e5, [(0, 0, 0)], self_term=False)).max() == 0.0


@pytest.mark.parametrize("a", [0, 2])
def test_demag_at_cells_uniform_box_matches_surface_charges(a):
    # a uniformly magnetised 7 x 5 x 2 box, at cells away from the centre (a corner,
    # an edge, a face): the Coulomb field of its two charged faces, by quadrature
    # independent of eq. 10/11
    nx, ny, nz = 7, 5, 2
    m = np.zeros((3, nx, ny, nz))
    m[a] = 1.0
    Ms = 8e5
    cells = [(0, 0, 0), (6, 4, 1), (3, 0, 1), (6, 2, 0)]
    H = demag_at_cells(m, Ms, cells)
    lo, hi = np.zeros(3), np.array([nx, ny, nz], float)
    for q, cell in enumerate(cells):
        p = np.array(cell, float) + 0.5
        Hq = Ms * _surface_charge_field(lo, hi, p, a)
        assert np.abs(H[q] - Hq).max() < 1e-9 * Ms


@pytest.mark.parametrize("self_term", [True, False])
def test_demag_at_cells_with_a_precomputed_tensor(self_term):
    # the sliced route (tensor given) is the per-cell route and the brute force
    grid = (6, 5, 3)
    m = _random_unit(grid, 9)
    K = demag_tensor(*grid, self_term=self_term)
    cells = [(0, 0, 0), (5, 4, 2), (2, 3, 1), (5, 0, 0), (0, 4, 2)]
    Hk = demag_at_cells(m, 8e5, cells, K=K)
    Hc = demag_at_cells(m, 8e5, cells, self_term=self_term)
    Hd = demag_direct(m, 8e5, K)
    ref = np.array([Hd[(slice(None),) + c] for c in cells])
    assert np.abs(Hk - Hc).max() <= 1e-13 * np.abs(Hc).max()
    assert np.abs(Hk - ref).max() <= 1e-13 * np.abs(ref).max()
