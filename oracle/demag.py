"""Demagnetising field as a discrete convolution, Section 2.3 (FP64).

Two routes that must agree:

* ``demag_direct``: the plain definition, eq. 12/13,
      H_a(i, j, k) = sum_{l, m, n} sum_b M_b(l, m, n) K_ab(l - i, m - j, n - k),
  an O(N^2) double loop (tiny grids only).
* ``demag_fft``: the convolution theorem, eq. 14, with the zero padding of
  Fig. 1 and the padded-convolution listing: the tensor is placed in an
  array of size 2nx x 2ny x 2nz at index (I + nx - 1, J + ny - 1, K + nz - 1),
  M is zero padded to the same size, both are transformed with ``fftn``, the
  per-frequency 3x3 product of eq. 14 is taken, ``ifftn`` brings it back, the
  real part is kept and the window starting at index (nx - 1, ny - 1, nz - 1)
  is cut out (the paper's truncation, 0-based).

The transforms are ``scipy.fft.fftn`` / ``ifftn`` (the same pocketfft
algorithm as ``numpy.fft``) with ``workers`` set to the host cores this
process may run on, so that a timed oracle uses the whole host.
"""
import os

import numpy as np
import scipy.fft

# host cores the transforms may use (the process's CPU affinity)
WORKERS = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)

from .tensor import COMPONENTS, tensor_at

_PAIRS = {(0, 0): "xx", (1, 1): "yy", (2, 2): "zz",
          (0, 1): "xy", (1, 0): "xy", (0, 2): "xz", (2, 0): "xz",
          (1, 2): "yz", (2, 1): "yz"}


def demag_direct(m, Ms, K):
    """Eq. 13 by brute force.  m: (3, nx, ny, nz) unit vectors; K from demag_tensor."""
    _, nx, ny, nz = m.shape
    M = Ms * np.asarray(m, dtype=np.float64)
    H = np.zeros_like(M)
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                # K(l - i, m - j, n - k) for l = 0..nx-1 sits at index (l - i) + nx - 1
                sl = (slice(nx - 1 - i, 2 * nx - 1 - i),
                      slice(ny - 1 - j, 2 * ny - 1 - j),
                      slice(nz - 1 - k, 2 * nz - 1 - k))
                for a in range(3):
                    tot = 0.0
                    for b in range(3):
                        tot += np.sum(M[b] * K[_PAIRS[(a, b)]][sl])
                    H[a, i, j, k] = tot
    return H


def demag_at_cells(m, Ms, cells, self_term=True, K=None):
    """Eq. 13 by brute force at a few target cells only (for grids too large for demag_direct).

    Without K the tensor is evaluated (eq. 10/11) at exactly the offsets l - i
    the sum needs, per target cell.  With K (the dict demag_tensor returns for
    this grid, holding its own choice of the self offset) the offsets are
    sliced out of it as demag_direct does, which is faster for many cells.
    Returns an array (len(cells), 3).
    """
    _, nx, ny, nz = m.shape
    M = Ms * np.asarray(m, dtype=np.float64)
    L = np.arange(nx)[:, None, None]
    Mm = np.arange(ny)[None, :, None]
    Nn = np.arange(nz)[None, None, :]
    out = np.zeros((len(cells), 3))
    for q, (i, j, k) in enumerate(cells):
        if K is None:
            Kc = tensor_at(L - i, Mm - j, Nn - k)
            if not self_term:
                for c in COMPONENTS:
                    Kc[c][i, j, k] = 0.0
        else:
            # K(l - i, m - j, n - k) for l = 0..nx-1 sits at index (l - i) + nx - 1
            sl = (slice(nx - 1 - i, 2 * nx - 1 - i),
                  slice(ny - 1 - j, 2 * ny - 1 - j),
                  slice(nz - 1 - k, 2 * nz - 1 - k))
            Kc = {c: K[c][sl] for c in COMPONENTS}
        for a in range(3):
            out[q, a] = sum(np.sum(M[b] * Kc[_PAIRS[(a, b)]]) for b in range(3))
    return out


class FFTDemag:
    """Eq. 14 with the paper's 2n zero padding.  Transforms the tensor once (setup)."""

    def __init__(self, nx, ny, nz, K):
        self.n = (nx, ny, nz)
        self.p = (2 * nx, 2 * ny, 2 * nz)
        self.Kf = {}
        for c in COMPONENTS:
            Kp = np.zeros(self.p)
            Kp[: 2 * nx - 1, : 2 * ny - 1, : 2 * nz - 1] = K[c]
            self.Kf[c] = scipy.fft.fftn(Kp, workers=WORKERS)

    def field(self, m, Ms):
        nx, ny, nz = self.n
        Mf = []
        for b in range(3):
            Mp = np.zeros(self.p)
            Mp[:nx, :ny, :nz] = Ms * m[b]
            Mf.append(scipy.fft.fftn(Mp, workers=WORKERS))
        H = np.empty((3, nx, ny, nz))
        for a in range(3):
            Hf = (Mf[0] * self.Kf[_PAIRS[(a, 0)]] + Mf[1] * self.Kf[_PAIRS[(a, 1)]]
                  + Mf[2] * self.Kf[_PAIRS[(a, 2)]])
            h = scipy.fft.ifftn(Hf, workers=WORKERS).real
            H[a] = h[nx - 1: 2 * nx - 1, ny - 1: 2 * ny - 1, nz - 1: 2 * nz - 1]
        return H


def demag_fft(m, Ms, K):
    _, nx, ny, nz = m.shape
    return FFTDemag(nx, ny, nz, K).field(np.asarray(m, dtype=np.float64), Ms)
