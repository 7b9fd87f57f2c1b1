"""Demagnetising tensor, Section 2.3, eq. 10 and eq. 11 (FP64).

For an offset (I, J, K) between two cubic cells of edge delta, the paper sums
over the eight corners (i, j, k in {0, 1}) of the source cell, seen from the
centre of the target cell, with

    x = (I + i - 1/2) delta,  y = (J + j - 1/2) delta,  z = (K + k - 1/2) delta,
    r = sqrt(x^2 + y^2 + z^2),  s = (-1)^(i + j + k),

    Kxx =  1/(4 pi) sum s atan(y z / (x r))          (eq. 10)
    Kyy =  1/(4 pi) sum s atan(x z / (y r))          (eq. 10 permuted)
    Kzz =  1/(4 pi) sum s atan(y x / (z r))          (eq. 10 permuted)
    Kxy = -1/(4 pi) sum s log(z + r)                 (eq. 11)
    Kxz = -1/(4 pi) sum s log(y + r)                 (eq. 11 permuted)
    Kyz = -1/(4 pi) sum s log(x + r)                 (eq. 11 permuted)

``tensor_at_mp`` evaluates the same sums with mpmath at 50 digits: the
reference for offsets far from the source, where the FP64 corner sums lose
~eps |n|^3 of relative accuracy to cancellation.

The printed sum limit "i = 1 to 1" of eq. 10/11 is read as i in {0, 1}, the
range the paper's own tensor listing loops over.  The coordinates are
half-integers times delta, so no denominator vanishes.

With this sign convention K is minus the usual demagnetising tensor N:
H_demag = K * M (eq. 9), and K(0, 0, 0) = -I/3 for a cube.  The paper's
listing skips the self offset (0, 0, 0); ``self_term=True`` (the default here)
keeps the value the formula gives there, ``self_term=False`` reproduces the
listing.
"""
import numpy as np

COMPONENTS = ("xx", "yy", "zz", "xy", "xz", "yz")


def tensor_at(I, J, Kk, delta=1.0):
    """Eq. 10/11 at offsets (I, J, K) given as broadcastable arrays of integers.

    Returns a dict component -> float64 array of the broadcast shape.
    """
    I = np.asarray(I, dtype=np.float64)
    J = np.asarray(J, dtype=np.float64)
    Kk = np.asarray(Kk, dtype=np.float64)
    shape = np.broadcast_shapes(I.shape, J.shape, Kk.shape)
    acc = {c: np.zeros(shape) for c in COMPONENTS}
    for i in (0, 1):
        for j in (0, 1):
            for k in (0, 1):
                s = (-1.0) ** (i + j + k)
                x = (I + i - 0.5) * delta
                y = (J + j - 0.5) * delta
                z = (Kk + k - 0.5) * delta
                r = np.sqrt(x * x + y * y + z * z)
                acc["xx"] += s * np.arctan(y * z / (x * r))
                acc["yy"] += s * np.arctan(x * z / (y * r))
                acc["zz"] += s * np.arctan(y * x / (z * r))
                acc["xy"] += s * np.log(z + r)
                acc["xz"] += s * np.log(y + r)
                acc["yz"] += s * np.log(x + r)
    pref = 1.0 / (4.0 * np.pi)
    return {
        "xx": pref * acc["xx"], "yy": pref * acc["yy"], "zz": pref * acc["zz"],
        "xy": -pref * acc["xy"], "xz": -pref * acc["xz"], "yz": -pref * acc["yz"],
    }


def demag_tensor(nx, ny, nz, delta=1.0, self_term=True):
    """K_ab(I, J, K) for all |I| < nx, |J| < ny, |K| < nz.

    Returns a dict component -> float64 array of shape (2nx-1, 2ny-1, 2nz-1)
    indexed [I + nx - 1, J + ny - 1, K + nz - 1].
    """
    I = np.arange(-nx + 1, nx)[:, None, None]
    J = np.arange(-ny + 1, ny)[None, :, None]
    Kk = np.arange(-nz + 1, nz)[None, None, :]
    out = tensor_at(I, J, Kk, delta)
    if not self_term:
        for c in COMPONENTS:
            out[c][nx - 1, ny - 1, nz - 1] = 0.0
    return out


def tensor_matrix(K, I, J, Kk, nx, ny, nz):
    """The symmetric 3x3 matrix K(I, J, K) from the dict returned by demag_tensor."""
    a, b, c = I + nx - 1, J + ny - 1, Kk + nz - 1
    xx, yy, zz = K["xx"][a, b, c], K["yy"][a, b, c], K["zz"][a, b, c]
    xy, xz, yz = K["xy"][a, b, c], K["xz"][a, b, c], K["yz"][a, b, c]
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def box_point_tensor(lo, hi, p):
    """Eq. 10/11 for one uniformly magnetised box [lo, hi] (3-vectors, m) seen from point p.

    The same corner sums as demag_tensor, but with arbitrary box corners; used
    to express the field of a whole uniformly magnetised sample at a cell
    centre (prism superposition).
    """
    out = np.zeros((3, 3))
    for i, xc in enumerate((lo[0], hi[0])):
        for j, yc in enumerate((lo[1], hi[1])):
            for k, zc in enumerate((lo[2], hi[2])):
                s = (-1.0) ** (i + j + k)
                x, y, z = xc - p[0], yc - p[1], zc - p[2]
                r = np.sqrt(x * x + y * y + z * z)
                out[0, 0] += s * np.arctan(y * z / (x * r))
                out[1, 1] += s * np.arctan(x * z / (y * r))
                out[2, 2] += s * np.arctan(y * x / (z * r))
                out[0, 1] -= s * np.log(z + r)
                out[0, 2] -= s * np.log(y + r)
                out[1, 2] -= s * np.log(x + r)
    out[1, 0], out[2, 0], out[2, 1] = out[0, 1], out[0, 2], out[1, 2]
    return out / (4.0 * np.pi)


def tensor_at_mp(I, J, Kk, dps=50):
    """Eq. 10/11 at one integer offset, evaluated with mpmath at `dps` significant
    digits (the same eight-corner sums as tensor_at, without FP64 cancellation:
    far from the source the corner terms are O(1) while their sum is O(|n|^-3)).

    Returns a dict component -> Python float (the correctly rounded value).
    """
    import mpmath
    with mpmath.workdps(dps):
        half = mpmath.mpf(1) / 2
        acc = {c: mpmath.mpf(0) for c in COMPONENTS}
        for i in (0, 1):
            for j in (0, 1):
                for k in (0, 1):
                    s = -1 if (i + j + k) % 2 else 1
                    x = mpmath.mpf(I) + i - half
                    y = mpmath.mpf(J) + j - half
                    z = mpmath.mpf(Kk) + k - half
                    r = mpmath.sqrt(x * x + y * y + z * z)
                    acc["xx"] += s * mpmath.atan(y * z / (x * r))
                    acc["yy"] += s * mpmath.atan(x * z / (y * r))
                    acc["zz"] += s * mpmath.atan(y * x / (z * r))
                    acc["xy"] += s * mpmath.log(z + r)
                    acc["xz"] += s * mpmath.log(y + r)
                    acc["yz"] += s * mpmath.log(x + r)
        pref = 1 / (4 * mpmath.pi)
        out = {c: float(pref * acc[c]) for c in ("xx", "yy", "zz")}
        out.update({c: float(-pref * acc[c]) for c in ("xy", "xz", "yz")})
    return out
