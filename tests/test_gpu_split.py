"""Split-precision z product (MM_SPLIT_BF16 / MM_SPLIT_FP16: the DFT along z as
tensor-core GEMMs with 16-bit hi+lo operands) vs the FP64 oracle.

Bar: effective-field relative L2 error <= 1e-4 per term (the split path's
bar); state after a short RK4 run within 1e-4 of the oracle's."""
import numpy as np
import pytest

from oracle.demag import demag_at_cells
from oracle.llg import TERM_ALL, TERM_DEMAG
from paper_1501_07293_b300 import inputs

from _util import gpu_heff, make_film, make_solver, rel_l2, to_device, to_xyz

pytestmark = pytest.mark.gpu

TOL = 1e-4
PRECS = ["split_bf16", "split_fp16"]
# nz 5 .. 8 (8-plane DFT operands) and 9 .. 16; ny from 33 (py = 128); ragged chunks of ky
GRIDS = [(100, 70, 9), (64, 130, 16), (33, 40, 5), (7, 33, 8), (48, 200, 12)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("grid", GRIDS)
def test_split_heff_matches_oracle(grid, prec):
    m = inputs.random_state(grid, 11)
    s = make_solver(grid, 4e-9, Ku=5e4, precision=prec)
    s.set_field((0.01, -0.02, 0.005))
    film = make_film(grid, 4e-9, Ku=5e4, b_ext=(0.01, -0.02, 0.005))
    mo = to_xyz(m)
    for t in (TERM_DEMAG, TERM_ALL):
        Hg = gpu_heff(s, m, t)
        Ho = to_device(film.h_eff(mo, t))
        assert rel_l2(Hg, Ho) <= TOL, (grid, prec, t, rel_l2(Hg, Ho))
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_split_heff_full_size_256x256x16(prec):
    w = inputs.film_256x256x16()
    m = inputs.workload_state(w)
    s = make_solver(w.grid, w.delta, Ms=w.mat.Ms, A=w.mat.A, Ku=w.mat.Ku, precision=prec)
    s.set_field(w.b_ext)
    film = make_film(w.grid, w.delta, Ms=w.mat.Ms, A=w.mat.A, Ku=w.mat.Ku, b_ext=w.b_ext)
    Hg = gpu_heff(s, m, TERM_DEMAG)
    Ho = to_device(film.h_eff(to_xyz(m), TERM_DEMAG))
    assert rel_l2(Hg, Ho) <= TOL, rel_l2(Hg, Ho)
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_split_heff_precision_study_512x512x8_sampled(prec):
    # the precision study's film: the oracle evaluates eq. 13 at sampled cells
    w = inputs.film_512x512x8()
    m = inputs.workload_state(w)
    s = make_solver(w.grid, w.delta, Ms=w.mat.Ms, A=w.mat.A, precision=prec)
    Hg = gpu_heff(s, m, TERM_DEMAG)
    cells = [(0, 0, 0), (511, 511, 7), (256, 17, 3), (100, 400, 5), (3, 260, 0)]
    Ho = demag_at_cells(to_xyz(m), w.mat.Ms, cells)
    Hgc = np.array([[Hg[a, k, j, i] for a in range(3)] for (i, j, k) in cells])
    assert np.abs(Hgc - Ho).max() <= TOL * np.abs(Hg).max()
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_split_rk4_trajectory(prec):
    import torch
    grid, dt, n = (40, 36, 6), 5e-14, 30
    m0 = inputs.random_state(grid, 12)
    s = make_solver(grid, 4e-9, Ku=5e4, alpha=0.05, precision=prec)
    s.set_field((0.0, 0.0, 0.01))
    s.set_m(torch.from_numpy(m0).cuda())
    s.step(n, dt)
    mg = s.get_m().cpu().numpy()
    film = make_film(grid, 4e-9, Ku=5e4, alpha=0.05, b_ext=(0.0, 0.0, 0.01))
    mo = to_device(film.run(to_xyz(m0), dt, n, "rk4"))
    assert np.abs(mg - mo).max() <= TOL, np.abs(mg - mo).max()
    s.close()


@pytest.mark.parametrize("grid", [(64, 64, 4), (64, 20, 8), (64, 64, 17)])
def test_split_unsupported_shapes_are_refused(grid):
    # nz < 5 or > 16, ny < 33
    from paper_1501_07293_b300.solver import MM_EUNSUPPORTED, MMError
    with pytest.raises(MMError) as e:
        make_solver(grid, 4e-9, precision="split_bf16")
    assert e.value.code == MM_EUNSUPPORTED


def test_split_batch_is_refused():
    from paper_1501_07293_b300.solver import MM_EUNSUPPORTED, Batch, MMError
    with pytest.raises(MMError) as e:
        Batch([(40, 40, 8)], 5e-9, 8e5, 1.3e-11, 0.0, 0.5, 1.76e11, precision="split_bf16")
    assert e.value.code == MM_EUNSUPPORTED
