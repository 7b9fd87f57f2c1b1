"""Pins of the oracle's demagnetising tensor (Section 2.3, eq. 10/11).

None of these re-types the oracle's formula: each checks a property that
physics or the geometry fixes independently (self-demag factors of a cube,
Gauss's law for the trace, point-dipole far field, parity and axis
permutations of a cube, scale invariance).
"""
import numpy as np
import pytest

from oracle.tensor import COMPONENTS, box_point_tensor, demag_tensor, tensor_matrix


def test_self_term_is_minus_one_third():
    # A uniformly magnetised cube has demag factors 1/3 along each axis
    # (cubic symmetry + N_xx + N_yy + N_zz = 1); K = -N.
    K = demag_tensor(2, 2, 2)
    T = tensor_matrix(K, 0, 0, 0, 2, 2, 2)
    assert np.allclose(T, -np.eye(3) / 3.0, atol=1e-15, rtol=0)


def test_self_term_flag_zeroes_only_the_centre():
    a = demag_tensor(3, 2, 2, self_term=True)
    b = demag_tensor(3, 2, 2, self_term=False)
    for c in COMPONENTS:
        d = a[c] - b[c]
        d[2, 1, 1] = 0.0
        assert np.all(d == 0.0)
        assert b[c][2, 1, 1] == 0.0


def test_trace_vanishes_outside_the_source():
    # Gauss: the potential of a cube is harmonic outside it, so the trace of
    # the field-gradient tensor is 0 at every other cell centre.
    K = demag_tensor(6, 5, 4)
    tr = K["xx"] + K["yy"] + K["zz"]
    tr[5, 4, 3] = 0.0
    assert np.abs(tr).max() < 1e-15


def test_parities():
    nx, ny, nz = 5, 4, 3
    K = demag_tensor(nx, ny, nz)
    flip = {0: lambda a: a[::-1, :, :], 1: lambda a: a[:, ::-1, :], 2: lambda a: a[:, :, ::-1]}
    odd_axes = {"xx": (), "yy": (), "zz": (), "xy": (0, 1), "xz": (0, 2), "yz": (1, 2)}
    for c in COMPONENTS:
        for ax in range(3):
            sign = -1.0 if ax in odd_axes[c] else 1.0
            assert np.allclose(flip[ax](K[c]), sign * K[c], atol=1e-15, rtol=0), (c, ax)
    # full inversion R -> -R leaves every component unchanged (eq. 12 order immaterial)
    for c in COMPONENTS:
        assert np.allclose(K[c][::-1, ::-1, ::-1], K[c], atol=1e-15, rtol=0)


def test_axis_permutations():
    # Cubic cells: swapping two axes of the offset swaps the matching components.
    n = 4
    K = demag_tensor(n, n, n)
    T = lambda c, perm: np.transpose(K[c], perm)
    assert np.allclose(K["yy"], T("xx", (1, 0, 2)), atol=1e-15)
    assert np.allclose(K["zz"], T("xx", (2, 1, 0)), atol=1e-15)
    assert np.allclose(K["xz"], T("xy", (0, 2, 1)), atol=1e-15)
    assert np.allclose(K["yz"], T("xy", (2, 1, 0)), atol=1e-15)
    assert np.allclose(K["xy"], T("xy", (1, 0, 2)), atol=1e-15)


@pytest.mark.parametrize("off", [(20, 13, 7), (30, -20, 15), (-39, 29, -19), (0, 35, 0), (25, 25, 0)])
def test_far_field_is_a_point_dipole(off):
    # Far from the source the cube acts as a point dipole of moment M delta^3:
    # H = (3 n n^T - I) M / (4 pi |n|^3), n the offset in cells.  A cube has no
    # quadrupole correction, so the relative gap falls at least like |n|^-4.
    K = demag_tensor(40, 36, 20)
    T = tensor_matrix(K, *off, 40, 36, 20)
    v = np.array(off, dtype=float)
    r = np.linalg.norm(v)
    u = v / r
    D = (3.0 * np.outer(u, u) - np.eye(3)) / (4.0 * np.pi * r ** 3)
    assert np.abs(T - D).max() / np.abs(D).max() < 1.0 / r ** 4


def test_independent_of_cell_size():
    a = demag_tensor(4, 3, 2, delta=1.0)
    b = demag_tensor(4, 3, 2, delta=3e-9)
    for c in COMPONENTS:
        assert np.abs(a[c] - b[c]).max() < 1e-12


def test_box_tensor_of_one_cell_equals_cell_tensor():
    K = demag_tensor(4, 4, 3)
    for off in [(0, 0, 0), (1, 2, 0), (-3, 1, 2), (2, -3, -1)]:
        # source cell centred at the offset, target at the origin
        lo = np.array(off, float) - 0.5
        hi = np.array(off, float) + 0.5
        T = box_point_tensor(lo, hi, np.zeros(3))
        assert np.allclose(T, tensor_matrix(K, *off, 4, 4, 3), atol=1e-15)


def test_thin_film_and_long_rod_limits():
    # Field at the centre of a uniformly magnetised box: a wide thin plate has
    # N_zz -> 1 (H_z = -M_z), a long square rod has N_xx -> 0, N_yy = N_zz -> 1/2.
    p = np.zeros(3)
    plate = box_point_tensor(np.array([-5e3, -5e3, -0.5]), np.array([5e3, 5e3, 0.5]), p)
    assert abs(plate[2, 2] + 1.0) < 1e-3 and abs(plate[0, 0]) < 1e-3
    rod = box_point_tensor(np.array([-5e3, -0.5, -0.5]), np.array([5e3, 0.5, 0.5]), p)
    assert abs(rod[0, 0]) < 1e-6 and abs(rod[1, 1] + 0.5) < 1e-6 and abs(rod[2, 2] + 0.5) < 1e-6


def test_mp_tensor_equals_fp64_near_the_source():
    # near the source the 50-digit and FP64 corner sums agree to the FP64 sums'
    # cancellation bound, a few eps |n|^3 relative
    from oracle.tensor import tensor_at, tensor_at_mp
    for off in [(0, 0, 0), (1, 0, 0), (1, 2, 0), (2, 1, 3), (3, 3, 1), (0, 4, 2), (5, 1, 1)]:
        mp = tensor_at_mp(*off)
        f = tensor_at(*off)
        scale = max(abs(v) for v in mp.values())
        n = np.sqrt(sum(v * v for v in off))
        for c in mp:
            assert abs(float(f[c]) - mp[c]) <= (1e-15 + 4e-16 * n ** 3) * scale, (off, c)


def test_mp_tensor_self_term_trace_and_far_field_rate():
    from oracle.tensor import tensor_at_mp
    mp = tensor_at_mp(0, 0, 0)
    assert abs(mp["xx"] + 1 / 3) < 1e-16 and abs(mp["xy"]) < 1e-16
    # trace zero off the source, to the precision of the 50-digit sums
    for off in [(40, 25, 3), (300, 7, 15), (1000, 500, 60)]:
        t = tensor_at_mp(*off)
        assert abs(t["xx"] + t["yy"] + t["zz"]) <= 1e-15 * max(abs(v) for v in t.values()), off

    # the gap to the point dipole (3 n n^T - I) / (4 pi |n|^3) falls as |n|^-4
    def gap(n):
        t = tensor_at_mp(*n)
        r = np.sqrt(sum(v * v for v in n))
        u = np.array(n, float) / r
        dip = (3 * np.outer(u, u) - np.eye(3)) / (4 * np.pi * r ** 3)
        m = np.array([[t["xx"], t["xy"], t["xz"]], [t["xy"], t["yy"], t["yz"]], [t["xz"], t["yz"], t["zz"]]])
        return np.abs(m - dip).max() / np.abs(dip).max()
    for n in [(20, 13, 7), (50, 30, 10)]:
        ratio = gap(n) / gap(tuple(2 * v for v in n))
        assert 14.0 < ratio < 18.0, (n, ratio)
