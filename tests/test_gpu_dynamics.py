"""Time-integration parity: mm_step / mm_energy / mm_observables vs the FP64 oracle."""
import numpy as np
import pytest

from paper_1501_07293_b300 import inputs

from _util import make_film, make_solver, rel_l2, to_device, to_xyz

pytestmark = pytest.mark.gpu


def _solver_for(w, **kw):
    mat = w.mat
    s = make_solver(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=mat.Ku, alpha=mat.alpha, gamma=mat.gamma, **kw)
    s.set_field(w.b_ext)
    return s


def _film_for(w, **kw):
    mat = w.mat
    return make_film(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=mat.Ku, alpha=mat.alpha, gamma=mat.gamma,
                     b_ext=w.b_ext, **kw)


def test_mean_m_trajectory_1ns_film_40x10x1():
    # RK4, dt = 0.1 ps, 10,000 steps (1 ns); <m> sampled every 100 steps (10 ps)
    import torch
    w = inputs.thin_film_small()
    m0 = inputs.workload_state(w)
    s = _solver_for(w)
    s.set_m(torch.from_numpy(m0).cuda())
    gpu = []
    for _ in range(w.steps // 100):
        s.step(100, w.dt)
        gpu.append(s.observables()[:3])
    film = _film_for(w)
    ora = []
    film.run(to_xyz(m0), w.dt, w.steps, "rk4", sample_every=100, callback=lambda k, m: ora.append(film.mean_m(m)))
    gpu, ora = np.array(gpu), np.array(ora)
    assert np.abs(gpu - ora).max() <= 1e-3
    # the film actually moves (the test is not vacuous)
    assert np.abs(ora[-1] - ora[0]).max() > 0.05
    s.close()


@pytest.mark.parametrize("integ", ["rk4", "euler"])
def test_short_trajectory_state_parity(integ):
    import torch
    grid = (24, 12, 3)
    w = inputs.Workload("t", grid, 4e-9, inputs.Material(Ms=8e5, A=1.3e-11, Ku=5e4, alpha=0.05),
                        (0.0, 0.0, 0.01), 5e-14, 60, "random", 99)
    m0 = inputs.workload_state(w)
    s = _solver_for(w, integrator=integ)
    s.set_m(torch.from_numpy(m0).cuda())
    s.step(w.steps, w.dt)
    mg = s.get_m().cpu().numpy()
    film = _film_for(w)
    mo = to_device(film.run(to_xyz(m0), w.dt, w.steps, integ))
    assert np.abs(mg - mo).max() <= 2e-5, np.abs(mg - mo).max()
    assert np.abs(np.linalg.norm(mg, axis=0) - 1.0).max() <= 1e-6
    s.close()


def test_short_trajectory_ragged_tiles_px512():
    # px = 512 with a ragged last tile (150 = 18 x 8 + 6 rows) and 75 pairs of cells per row:
    # the x kernel's tensor-copy tile path and two-pass transforms, and the z product's
    # transform form (9 planes, py = 512)
    import torch
    grid = (150, 150, 9)
    w = inputs.Workload("t", grid, 4e-9, inputs.Material(Ms=8e5, A=1.3e-11, Ku=5e4, alpha=0.05),
                        (0.0, 0.0, 0.01), 5e-14, 20, "random", 98)
    m0 = inputs.workload_state(w)
    s = _solver_for(w)
    s.set_m(torch.from_numpy(m0).cuda())
    s.step(w.steps, w.dt)
    mg = s.get_m().cpu().numpy()
    film = _film_for(w)
    mo = to_device(film.run(to_xyz(m0), w.dt, w.steps, "rk4"))
    assert np.abs(mg - mo).max() <= 2e-5, np.abs(mg - mo).max()
    s.close()


def test_two_steps_full_size_256x256x16():
    import torch
    w = inputs.film_256x256x16()
    m0 = inputs.workload_state(w)
    s = _solver_for(w)
    s.set_m(torch.from_numpy(m0).cuda())
    s.step(2, w.dt)
    mg = s.get_m().cpu().numpy()
    film = _film_for(w)
    mo = to_device(film.run(to_xyz(m0), w.dt, 2, "rk4"))
    assert np.abs(mg - mo).max() <= 1e-5, np.abs(mg - mo).max()
    s.close()


def test_200_steps_full_size_256x256x16_against_the_stored_oracle_trajectory():
    # the bench workload over 200 RK4 steps (10 fs): <m> every 10 steps and the
    # state at 512 seeded cells at steps 100 and 200, against the FP64 oracle's
    # trajectory stored by tests/golden/make_film_256x256x16_rk4_200.py
    import json
    import os
    import torch
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "film_256x256x16_rk4_200.json")) as f:
        g = json.load(f)
    w = inputs.film_256x256x16()
    s = _solver_for(w)
    s.set_m(torch.from_numpy(inputs.workload_state(w)).cuda())
    cells = g["cells"]
    mean_err, cell_err = 0.0, {}
    for row in g["mean_m"]:
        step = int(row[0])
        s.step(10, w.dt)
        mean_err = max(mean_err, float(np.abs(s.observables()[:3] - np.array(row[1:])).max()))
        if str(step) in g["states"]:
            mg = s.get_m().cpu().numpy()
            got = np.array([[mg[a, k, j, i] for a in range(3)] for (i, j, k) in cells])
            cell_err[step] = float(np.abs(got - np.array(g["states"][str(step)])).max())
    s.close()
    print("200-step trajectory: max |<m> - oracle|", mean_err, "max cell error", cell_err)
    assert mean_err <= MEAN_TOL_200, mean_err
    assert max(cell_err.values()) <= CELL_TOL_200, cell_err


# Tolerances of the 200-step comparison.  An FP32 trajectory leaves the FP64
# one by the rounding of every step, amplified by the stiff exchange dynamics of
# the random start (the measured cell error grows from 9e-7 at step 100 to 8e-6
# at step 200); <m> averages 2^20 cells and stays within 1e-8.  The bars are
# about ten times the measured errors.
MEAN_TOL_200 = 1e-7
CELL_TOL_200 = 1e-4


def test_energy_and_observables_match_oracle():
    import torch
    from oracle.energy import energies
    grid = (20, 12, 3)
    w = inputs.Workload("e", grid, 4e-9, inputs.Material(Ms=8e5, A=1.3e-11, Ku=5e4, alpha=0.05),
                        (0.02, -0.01, 0.03), 5e-14, 0, "random", 5)
    m0 = inputs.workload_state(w)
    s = _solver_for(w)
    s.set_m(torch.from_numpy(m0).cuda())
    E = s.energy()
    obs = s.observables()
    film = _film_for(w)
    mo = to_xyz(m0)
    Eo = np.array(energies(film, mo))
    assert np.abs(E - Eo).max() <= 1e-5 * np.abs(Eo).max()
    assert np.abs(obs[:3] - film.mean_m(mo)).max() <= 1e-6
    assert abs(obs[3] - film.max_dmdt(mo)) <= 1e-5 * film.max_dmdt(mo)
    s.close()


def test_energy_decays_on_gpu():
    import torch
    w = inputs.Workload("d", (32, 16, 2), 4e-9, inputs.Material(Ms=8e5, A=1.3e-11, Ku=5e4, alpha=0.1),
                        (0.0, 0.0, 0.01), 5e-14, 0, "random", 6)
    s = _solver_for(w)
    s.set_m(torch.from_numpy(inputs.workload_state(w)).cuda())
    E = [s.energy()[4]]
    for _ in range(10):
        s.step(10, w.dt)
        E.append(s.energy()[4])
    dE = np.diff(E)
    assert np.all(dE <= 1e-6 * abs(E[0])), dE
    s.close()


def test_launch_count_and_graph_replay():
    import torch
    s = make_solver((16, 8, 2), 4e-9)
    s.set_m(torch.from_numpy(inputs.random_state((16, 8, 2), 1)).cuda())
    before = s.launch_count()
    s.step(5, 1e-13)
    s.sync()
    # one x-transform to start the pipeline, then 4 RK4 stages x 2 kernels per step
    assert s.launch_count() - before == 1 + 5 * 8
    before = s.launch_count()
    s.step(3, 1e-13)
    s.sync()
    assert s.launch_count() - before == 3 * 8
    s.close()
