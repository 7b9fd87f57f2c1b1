"""The set-up's FP64 tensor (eq. 10/11 near the source, its multipole series
beyond 9 cells) through mm_tensor_eval, against the 50-digit evaluation of
eq. 10/11 (oracle.tensor.tensor_at_mp) and, at the switch-over, against the
FP64 corner sums (oracle.tensor.tensor_at)."""
import numpy as np
import pytest

from oracle.tensor import tensor_at, tensor_at_mp

pytestmark = pytest.mark.gpu

COMP = ("xx", "yy", "zz", "xy", "xz", "yz")

# near the source, around the switch-over radius 9 and every change of the
# series order (20, 50, 160 cells), and far out (up to the largest padded grids)
OFFSETS = [(0, 0, 0), (1, 0, 0), (3, 2, 1), (7, 5, 2), (8, 0, 0), (6, 5, 3), (9, 0, 0), (7, 5, 3),
           (11, 0, 0), (8, 8, 3), (11, 3, 2), (12, 0, 0), (10, 7, 0), (9, 7, 3), (12, 1, 1), (19, 0, 3), (16, 11, 2), (20, 0, 0),
           (35, 35, 1), (49, 9, 0), (50, 1, 0), (40, 30, 7), (159, 5, 0), (150, 60, 10),
           (160, 0, 0), (255, 255, 15), (3, 300, 0), (511, 511, 7), (700, 20, 60), (1023, 1023, 3)]


def _rel(dev_row, ref):
    r = np.array([ref[c] for c in COMP])
    return float(np.abs(dev_row - r).max() / np.abs(r).max())


def test_setup_tensor_matches_50_digit_sums():
    from paper_1501_07293_b300.solver import tensor_eval
    dev = tensor_eval(OFFSETS)
    for row, off in zip(dev, OFFSETS):
        e = _rel(row, tensor_at_mp(*off))
        n = np.sqrt(sum(v * v for v in off))
        assert e <= 1e-12, (off, e)
        if n >= 9:    # the series: ~1e-15, ~3e-14 at the switch-over
            assert e <= 5e-14, (off, e)
        else:         # the FP64 corner sums: their cancellation bound, a few eps |n|^3
            assert e <= 1e-15 + 1e-15 * n ** 3, (off, e)


def test_switch_over_matches_fp64_corner_sums():
    # the series just beyond 9 cells against the FP64 eq. 10/11 corner sums there
    # (which are good to ~6e-13 at that distance)
    from paper_1501_07293_b300.solver import tensor_eval
    ring = [(9, 0, 0), (7, 5, 3), (8, 4, 1), (6, 6, 3), (9, 1, 1), (7, 4, 4), (8, 3, 3)]
    dev = tensor_eval(ring)
    for row, off in zip(dev, ring):
        assert sum(v * v for v in off) >= 81
        f = tensor_at(*off)
        e = _rel(row, {c: float(f[c]) for c in COMP})
        assert e <= 1e-12, (off, e)


def test_setup_tensor_parities():
    # K(-I, J, K): xy, xz odd; K(I, -J, K): xy, yz odd; K(I, J, -K): xz, yz odd
    # (to the rounding of two independent evaluations; a wrong sign is off by 2x)
    from paper_1501_07293_b300.solver import tensor_eval
    base = [(5, 3, 2), (30, 17, 4), (200, 90, 9)]
    sig = {(-1, 1, 1): [1, 1, 1, -1, -1, 1], (1, -1, 1): [1, 1, 1, -1, 1, -1], (1, 1, -1): [1, 1, 1, 1, -1, -1]}
    for off in base:
        ref = tensor_eval([off])[0]
        for s, f in sig.items():
            got = tensor_eval([tuple(a * b for a, b in zip(off, s))])[0]
            assert np.allclose(got, ref * np.array(f), rtol=1e-12, atol=1e-18), (off, s)
