"""Effective-field parity: CUDA path (mm_heff through the C ABI) vs the FP64 oracle.

Bar (FP32 path): relative L2 error <= 1e-5 per field term and for the sum,
over all cells and components, the oracle evaluated on the same float32
state the GPU holds.
"""
import numpy as np
import pytest

from oracle.demag import demag_at_cells
from oracle.llg import TERM_ALL, TERM_ANISOTROPY, TERM_DEMAG, TERM_EXCHANGE, TERM_ZEEMAN
from paper_1501_07293_b300 import inputs

from _util import gpu_heff, make_film, make_solver, per_cell_rel, rel_l2, sample_cells, to_device, to_xyz

pytestmark = pytest.mark.gpu

TOL = 1e-5
TERMS = [TERM_EXCHANGE, TERM_ANISOTROPY, TERM_DEMAG, TERM_ZEEMAN, TERM_ALL]

# small grids: several tiles along y, ragged tails, degenerate axes, odd sizes
GRIDS = [(40, 10, 1), (7, 5, 3), (1, 1, 1), (2, 1, 1), (1, 9, 1), (1, 1, 7), (9, 1, 1), (16, 8, 2), (5, 130, 3), (3, 300, 1),
         (33, 17, 5), (64, 32, 4), (3, 40, 2), (100, 3, 16), (48, 48, 9),
         # thick samples: the chunked z product (17..32 and 33..64 planes), ragged chunks
         (8, 8, 17), (5, 3, 33), (20, 9, 24), (1, 1, 40), (3, 1, 64), (24, 20, 64),
         # columns beyond one CTA: the split y/z pass (y transforms and z product through a buffer)
         (20, 200, 40), (6, 5, 100), (9, 70, 65), (1, 40, 128),
         # the z product as a length-32 transform along z (9..16 planes, padded y of 256 / 512)
         (9, 100, 11), (6, 130, 16), (12, 70, 9), (3, 256, 16), (5, 129, 13)]


def _compare(grid, delta=4e-9, Ku=5e4, b_ext=(0.01, -0.02, 0.005), seed=7, self_term=True,
             hmap=False, kumap=False, zform="auto"):
    m = inputs.random_state(grid, seed)
    hm = inputs.zeeman_map(grid, seed + 1) if hmap else None
    km = inputs.ku_map(grid, seed + 2) if kumap else None
    s = make_solver(grid, delta, Ku=Ku, self_term=self_term, zform=zform)
    import torch
    s.set_field(b_ext, None if hm is None else torch.from_numpy(hm).cuda(),
                None if km is None else torch.from_numpy(km).cuda())
    film = make_film(grid, delta, Ku=Ku, b_ext=b_ext, h_map_dev=hm, ku_map_dev=km, self_term=self_term)
    mo = to_xyz(m)
    out = {}
    for t in TERMS:
        Hg = gpu_heff(s, m, t)
        Ho = to_device(film.h_eff(mo, t))
        out[t] = rel_l2(Hg, Ho) if np.linalg.norm(Ho) > 0 else float(np.abs(Hg).max())
    s.close()
    return out


@pytest.mark.parametrize("grid", GRIDS)
def test_heff_matches_oracle(grid):
    err = _compare(grid)
    for t, e in err.items():
        assert e <= TOL, (grid, t, e)


@pytest.mark.parametrize("grid", [(9, 100, 11), (6, 130, 16)])
def test_heff_direct_z_sum_matches_oracle(grid):
    # the same grids with the z product forced to the direct Toeplitz sum
    err = _compare(grid, zform="direct")
    for t, e in err.items():
        assert e <= TOL, (grid, t, e)


@pytest.mark.parametrize("grid", [(40, 10, 1), (12, 7, 3), (6, 130, 16)])
def test_heff_with_maps(grid):
    err = _compare(grid, hmap=True, kumap=True)
    for t, e in err.items():
        assert e <= TOL, (grid, t, e)


def test_heff_without_self_term():
    err = _compare((20, 6, 2), self_term=False)
    for t, e in err.items():
        assert e <= TOL, (t, e)


def test_demag_direct_sum_route():
    # also against the brute-force eq. 13 (not only the oracle's FFT route)
    grid = (9, 6, 3)
    m = inputs.random_state(grid, 3)
    s = make_solver(grid, 5e-9)
    Hg = gpu_heff(s, m, TERM_DEMAG)
    film = make_film(grid, 5e-9, demag="direct")
    Ho = to_device(film.h_demag(to_xyz(m)))
    assert rel_l2(Hg, Ho) <= TOL


@pytest.mark.parametrize("zform", ["auto", "direct"])
def test_heff_full_size_256x256x16(zform):
    w = inputs.film_256x256x16()
    m = inputs.workload_state(w)
    s = make_solver(w.grid, w.delta, Ms=w.mat.Ms, A=w.mat.A, Ku=w.mat.Ku, alpha=w.mat.alpha, zform=zform)
    s.set_field(w.b_ext)
    film = make_film(w.grid, w.delta, Ms=w.mat.Ms, A=w.mat.A, Ku=w.mat.Ku, b_ext=w.b_ext)
    mo = to_xyz(m)
    for t in (TERM_DEMAG, TERM_ALL):
        Hg = gpu_heff(s, m, t)
        Ho = to_device(film.h_eff(mo, t))
        assert rel_l2(Hg, Ho) <= TOL, t
    s.close()


def test_heff_full_size_512x512x8_sampled():
    # full size of the precision study; the oracle evaluates eq. 13 at 42 sampled
    # cells (corners, edges, both z faces, random interior cells), each to the
    # FP32 bar relative to its own field
    from oracle.tensor import demag_tensor
    w = inputs.film_512x512x8()
    m = inputs.workload_state(w)
    s = make_solver(w.grid, w.delta, Ms=w.mat.Ms, A=w.mat.A)
    Hg = gpu_heff(s, m, TERM_DEMAG)
    s.close()
    cells = sample_cells(w.grid, 16, 8)
    assert len(cells) >= 32
    K = demag_tensor(*w.grid, delta=w.delta)
    Ho = demag_at_cells(to_xyz(m), w.mat.Ms, cells, K=K)
    err = per_cell_rel(Hg, Ho, cells)
    assert err <= TOL, err


@pytest.mark.parametrize("grid", [(8, 8, 129), (2000, 4, 4)])
def test_unsupported_grid_is_refused_cleanly(grid):
    # more than 128 planes; a padded x size beyond 2048
    from paper_1501_07293_b300.solver import MM_EUNSUPPORTED, MMError
    with pytest.raises(MMError) as e:
        make_solver(grid, 4e-9)
    assert e.value.code == MM_EUNSUPPORTED


def test_bad_arguments_return_einval():
    from paper_1501_07293_b300.solver import MM_EINVAL, MMError
    with pytest.raises(MMError) as e:
        make_solver((0, 8, 1), 4e-9)
    assert e.value.code == MM_EINVAL
    s = make_solver((8, 8, 1), 4e-9)
    with pytest.raises(MMError) as e:
        s.step(-1, 1e-13)
    assert e.value.code == MM_EINVAL
    with pytest.raises(MMError):
        s.heff(99)
    s.close()


def test_nonfinite_state_is_reported():
    import torch
    from paper_1501_07293_b300.solver import MM_ENONFINITE, MMError
    grid = (8, 4, 1)
    m = inputs.random_state(grid, 1)
    m[0, 0, 0, 3] = np.nan
    s = make_solver(grid, 4e-9)
    s.set_m(torch.from_numpy(m).cuda())
    with pytest.raises(MMError) as e:
        s.sync()
    assert e.value.code == MM_ENONFINITE
    s.close()


def test_bounded_wait_timeout_is_reported_and_recoverable():
    # a kernel whose wait runs out sets the flag; the host sees MM_ETIMEOUT, the context keeps working
    import torch
    from paper_1501_07293_b300.solver import MM_ETIMEOUT, MMError
    from oracle.llg import TERM_ALL
    grid = (16, 8, 2)
    m = inputs.random_state(grid, 4)
    s = make_solver(grid, 4e-9)
    s.set_m(torch.from_numpy(m).cuda())
    s.selftest_wait_timeout(2000)
    with pytest.raises(MMError) as e:
        s.sync()
    assert e.value.code == MM_ETIMEOUT
    s.sync()   # flag cleared
    Hg = gpu_heff(s, m, TERM_ALL)
    Ho = to_device(make_film(grid, 4e-9).h_eff(to_xyz(m), TERM_ALL))
    assert rel_l2(Hg, Ho) <= TOL
    s.close()
