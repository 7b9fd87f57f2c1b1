"""Exchange field, Section 2.1, eq. 4, 5 and the Neumann rule eq. 6/7 (FP64).

    H_exch(i, j, k) = 2A / (mu0 Ms^2) * sum over the six neighbours of
                      (M(neighbour) - M(i, j, k)) / delta^2

A neighbour that does not exist (outside the grid) is replaced by the cell
itself (eq. 7), so its term vanishes; along an axis with a single cell both
terms vanish.  Written with an edge-replicated ghost layer, which is exactly
"the non-existing neighbour is the centre cell".
"""
import numpy as np

from . import MU0


def exchange_field(m, Ms, A, delta):
    """m: (3, nx, ny, nz) unit vectors -> H_exch in A/m."""
    M = Ms * np.asarray(m, dtype=np.float64)
    g = np.pad(M, ((0, 0), (1, 1), (1, 1), (1, 1)), mode="edge")
    c = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
    lap = (g[:, 2:, 1:-1, 1:-1] + g[:, :-2, 1:-1, 1:-1]
           + g[:, 1:-1, 2:, 1:-1] + g[:, 1:-1, :-2, 1:-1]
           + g[:, 1:-1, 1:-1, 2:] + g[:, 1:-1, 1:-1, :-2]
           - 6.0 * g[c]) / (delta * delta)
    return 2.0 * A / (MU0 * Ms * Ms) * lap
