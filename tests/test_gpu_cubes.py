"""The standard-problem-3 cubes of Table 1 (n^3, n = 8 .. 64, and 128^3): effective
field and explicit-Euler steps through the C ABI vs the FP64 oracle.  The thick
cubes (n >= 32) run the chunked z product; 128^3 runs the split y/z pass."""
import numpy as np
import pytest

from oracle.demag import demag_at_cells
from oracle.llg import TERM_ALL, TERM_DEMAG
from paper_1501_07293_b300 import inputs

from _util import gpu_heff, make_film, make_solver, per_cell_rel, rel_l2, sample_cells, to_device, to_xyz

pytestmark = pytest.mark.gpu


def _parts(n, integrator="euler"):
    w = inputs.sp3_cube(n)
    mat = w.mat
    s = make_solver(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=mat.Ku, alpha=mat.alpha, gamma=mat.gamma,
                    integrator=integrator)
    film = make_film(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=mat.Ku, alpha=mat.alpha, gamma=mat.gamma)
    return w, s, film


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_sp3_cube_heff(n):
    w, s, film = _parts(n)
    m = inputs.workload_state(w)
    mo = to_xyz(m)
    for t in (TERM_DEMAG, TERM_ALL):
        Hg = gpu_heff(s, m, t)
        Ho = to_device(film.h_eff(mo, t))
        assert rel_l2(Hg, Ho) <= 1e-5, (n, t, rel_l2(Hg, Ho))
    s.close()


@pytest.mark.parametrize("n", [16, 32])
def test_sp3_cube_euler_steps(n):
    import torch
    w, s, film = _parts(n)
    m0 = inputs.workload_state(w)
    s.set_m(torch.from_numpy(m0).cuda())
    s.step(20, w.dt)
    mg = s.get_m().cpu().numpy()
    mo = to_device(film.run(to_xyz(m0), w.dt, 20, "euler"))
    assert np.abs(mg - mo).max() <= 2e-5, np.abs(mg - mo).max()
    assert np.abs(mo - m0).max() > 1e-3   # the state moves
    s.close()


def test_sp3_cube_128_sampled():
    # the oracle evaluates eq. 13 at 42 sampled cells (corners, edges, faces, random
    # interior cells: the whole 2M-cell source sum each), each to the FP32 bar
    # relative to its own field
    from oracle.tensor import demag_tensor
    w = inputs.sp3_cube(128)
    mat = w.mat
    s = make_solver(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=mat.Ku, alpha=mat.alpha, gamma=mat.gamma,
                    integrator="euler")
    m = inputs.workload_state(w)
    Hg = gpu_heff(s, m, TERM_DEMAG)
    s.close()
    cells = sample_cells(w.grid, 16, 128)
    K = demag_tensor(*w.grid, delta=w.delta)
    Ho = demag_at_cells(to_xyz(m), w.mat.Ms, cells, K=K)
    err = per_cell_rel(Hg, Ho, cells)
    assert err <= 1e-5, err
