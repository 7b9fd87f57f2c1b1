"""Combinations of the paths against the FP64 oracle: the adjoint through the
split y/z pass, Euler with the split-precision z product, and a field program
driving the tensor-core path."""
import numpy as np
import pytest

from oracle import to_device, to_xyz
from oracle.adjoint import AdjointFilm, tangent_project
from oracle.program import program_for, run_program
from paper_1501_07293_b300 import inputs

from _util import make_film, make_solver, rel_l2

pytestmark = pytest.mark.gpu


def test_adjoint_through_the_split_yz_pass():
    # 70 planes: the y/z pass runs as three kernels, in the stages and in the
    # adjoint's applications of the exchange + demag operator
    import torch
    grid, dt, n = (6, 5, 70), 1e-13, 8
    m0 = inputs.random_state(grid, 61)
    h = inputs.zeeman_map(grid, 62)
    ku = inputs.ku_map(grid, 63)
    s = make_solver(grid, 4e-9, Ku=0.0, alpha=0.1)
    assert s.tuning()[0] == 2
    s.set_field((0.0, 0.0, 0.0), torch.from_numpy(h).cuda(), torch.from_numpy(ku).cuda())
    s.set_m(torch.from_numpy(m0).cuda())
    m0n = s.get_m().cpu().numpy()
    w = np.random.default_rng(64).standard_normal(m0.shape).astype(np.float32)   # dL/dm_final of L = <w, m_n>
    gr = s.adjoint(n, dt, 3, torch.from_numpy(w).cuda())
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()}
    film = make_film(grid, 4e-9, Ku=0.0, alpha=0.1, h_map_dev=h, ku_map_dev=ku)
    adj = AdjointFilm(film)
    _, rec = adj.forward(to_xyz(m0n), dt, n)
    gm, gh, gk = adj.backward(rec, dt, to_xyz(w))
    assert rel_l2(got["m0"], to_device(tangent_project(to_xyz(m0n), gm))) <= 1e-3
    assert rel_l2(got["h"], to_device(gh)) <= 1e-3
    assert rel_l2(got["ku"], to_device(gk)) <= 1e-3
    s.close()


@pytest.mark.parametrize("prec", ["split_bf16", "split_fp16"])
def test_euler_with_the_split_precision_product(prec):
    import torch
    grid, dt, n = (40, 36, 6), 5e-14, 40
    m0 = inputs.random_state(grid, 65)
    s = make_solver(grid, 4e-9, Ku=5e4, alpha=0.05, integrator="euler", precision=prec)
    s.set_field((0.0, 0.01, 0.0))
    s.set_m(torch.from_numpy(m0).cuda())
    s.step(n, dt)
    film = make_film(grid, 4e-9, Ku=5e4, alpha=0.05, b_ext=(0.0, 0.01, 0.0))
    mo = to_device(film.run(to_xyz(m0), dt, n, "euler"))
    assert np.abs(s.get_m().cpu().numpy() - mo).max() <= 1e-4
    s.close()


def test_field_program_on_the_tensor_core_path():
    import torch
    grid, dt, n = (40, 36, 6), 1e-13, 30
    segs = [(0.0, 15 * dt, (0.0, 0.05, 0.0), (0.1, -0.05, 0.02), 0.3),
            (15 * dt, 1.0, (0.1, -0.05, 0.02), (-0.1, 0.2, 0.0), 0.05)]
    m0 = inputs.random_state(grid, 66)
    s = make_solver(grid, 4e-9, Ku=3e4, alpha=0.1, precision="split_bf16")
    s.set_m(torch.from_numpy(m0).cuda())
    s.set_program(segs)
    s.step(n, dt)
    film = make_film(grid, 4e-9, Ku=3e4, alpha=0.1)
    mo, _ = run_program(film, to_xyz(m0), 0.0, dt, n, program_for(film, segs), "rk4")
    assert np.abs(s.get_m().cpu().numpy() - to_device(mo)).max() <= 1e-4
    s.close()
