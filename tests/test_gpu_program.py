"""Field programs on the device (mm_set_program / mm_set_time / mm_get_time)
and in-place graph updates (mm_set_field between steps) vs the FP64 oracle."""
import numpy as np
import pytest

from oracle.program import FieldProgram, program_for, run_program
from paper_1501_07293_b300 import inputs

from _util import make_film, make_solver, to_device, to_xyz

pytestmark = pytest.mark.gpu


def _sp4_parts(self_term):
    w = inputs.sp4_film()
    mat = w.mat
    s = make_solver(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=mat.Ku, alpha=mat.alpha, gamma=mat.gamma,
                    integrator="euler", self_term=self_term)
    film = make_film(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=mat.Ku, alpha=mat.alpha, gamma=mat.gamma,
                     self_term=self_term)
    return w, s, film


@pytest.mark.parametrize("self_term", [False, True])
def test_sp4_protocol_compressed_paper_mode(self_term):
    # the paper's film, Euler at its dt, the protocol with its phases shortened
    # (saturate 40 steps, ramp to step 60, relax to 100, reverse to 200);
    # self_term False is the paper's tensor (self offset skipped)
    import torch
    w, s, film = _sp4_parts(self_term)
    segs = inputs.sp4_schedule(w.dt, n_sat=40, n_ramp=60, n_rev=100, n_end=200)
    m0 = inputs.workload_state(w)
    s.set_m(torch.from_numpy(m0).cuda())
    s.set_program(segs)
    gpu_means = []
    for _ in range(5):
        s.step(40, w.dt)
        gpu_means.append(s.observables()[:3])
    mg = s.get_m().cpu().numpy()
    assert abs(s.time() - 200 * w.dt) <= 1e-12 * 200 * w.dt
    ora_means = []
    mo, t = run_program(film, to_xyz(m0), 0.0, w.dt, 200, program_for(film, segs), "euler",
                        sample_every=40, callback=lambda k, t, m: ora_means.append(film.mean_m(m)))
    assert np.abs(mg - to_device(mo)).max() <= 2e-5, np.abs(mg - to_device(mo)).max()
    assert np.abs(np.array(gpu_means) - np.array(ora_means)).max() <= 1e-5
    # the protocol moves the state (saturation tilts m toward (1,1,1))
    assert np.abs(ora_means[-1] - np.array([1.0, 0.0, 0.0])).max() > 1e-3
    s.close()


@pytest.mark.parametrize("grid,n", [((33, 17, 3), 60), ((12, 40, 70), 30)])
def test_rk4_program_stage_times_ragged_film(grid, n):
    # ramps on all three components and a damping switch: the four RK4 stages
    # read their own drive slots (t, t + dt/2, t + dt/2, t + dt); the 70-plane
    # film runs the split y/z pass, whose first kernel advances the clock
    import torch
    delta, dt = 4e-9, 1e-13
    segs = [(0.0, 25 * dt, (0.0, 0.05, -0.02), (0.2, -0.1, 0.05), 0.3),
            (25 * dt, 1.0, (0.2, -0.1, 0.05), (-0.1, 0.4, 0.1), 0.02)]
    m0 = inputs.random_state(grid, 31)
    s = make_solver(grid, delta, Ku=3e4, alpha=0.1)
    s.set_m(torch.from_numpy(m0).cuda())
    s.set_program(segs)
    s.step(n, dt)
    mg = s.get_m().cpu().numpy()
    film = make_film(grid, delta, Ku=3e4, alpha=0.1)
    mo, _ = run_program(film, to_xyz(m0), 0.0, dt, n, program_for(film, segs), "rk4")
    assert np.abs(mg - to_device(mo)).max() <= 2e-5, np.abs(mg - to_device(mo)).max()
    s.close()


def test_clock_offset_heff_energy_at_the_clock():
    import torch
    from oracle.energy import energies
    from oracle.llg import TERM_ZEEMAN
    grid, delta, dt = (20, 12, 2), 4e-9, 5e-14
    segs = [(1e-9, 1e-9 + 40 * dt, (0.01, 0.0, 0.0), (0.05, -0.02, 0.01), 0.2)]
    m0 = inputs.random_state(grid, 32)
    s = make_solver(grid, delta, Ku=5e4, alpha=0.05)
    s.set_field((0.0, 0.0, 0.003))
    s.set_m(torch.from_numpy(m0).cuda())
    s.set_program(segs)
    s.set_time(1e-9)
    s.step(30, dt)
    t = s.time()
    assert abs(t - (1e-9 + 30 * dt)) <= 1e-12 * t
    film = make_film(grid, delta, Ku=5e4, alpha=0.05, b_ext=(0.0, 0.0, 0.003))
    prog = program_for(film, segs)
    mo, to = run_program(film, to_xyz(m0), 1e-9, dt, 30, prog, "rk4")
    mg = s.get_m().cpu().numpy()
    assert np.abs(mg - to_device(mo)).max() <= 2e-5
    # field, energy and |dm/dt| at the clock use the program's value there
    b, alpha = prog.at(to)
    H = s.heff(TERM_ZEEMAN).cpu().numpy()
    from oracle import MU0
    for c in range(3):
        assert np.allclose(H[c], b[c] / MU0, rtol=1e-6, atol=1e-3)
    at = make_film(grid, delta, Ku=5e4, alpha=alpha, b_ext=tuple(b))
    E = s.energy()
    Eo = np.array(energies(at, to_xyz(mg)))
    assert np.abs(E - Eo).max() <= 1e-5 * np.abs(Eo).max()
    obs = s.observables()
    assert abs(obs[3] - at.max_dmdt(to_xyz(mg))) <= 1e-5 * at.max_dmdt(to_xyz(mg))
    s.close()


def test_removing_the_program_restores_the_constant_field_bitwise():
    import torch
    grid, delta, dt = (24, 10, 2), 4e-9, 1e-13
    m0 = torch.from_numpy(inputs.random_state(grid, 33)).cuda()
    a = make_solver(grid, delta, alpha=0.1)
    a.set_field((0.01, 0.0, -0.01))
    a.set_m(m0)
    a.set_program([(0.0, 1.0, (0.3, 0.0, 0.0), (0.3, 0.0, 0.0), 0.5)])
    a.step(5, dt)
    a.set_program([])
    a.set_m(m0)
    a.step(20, dt)
    b = make_solver(grid, delta, alpha=0.1)
    b.set_field((0.01, 0.0, -0.01))
    b.set_m(m0)
    b.step(20, dt)
    assert np.array_equal(a.get_m().cpu().numpy(), b.get_m().cpu().numpy())
    a.close()
    b.close()


def test_field_sweep_updates_the_step_graph_in_place():
    # a host-driven sweep: mm_set_field between steps patches the captured graph;
    # every point equals a fresh context bitwise, and the oracle within the bar
    import torch
    grid, delta, dt = (30, 14, 1), 4e-9, 1e-13
    m0 = inputs.random_state(grid, 34)
    s = make_solver(grid, delta, alpha=0.2)
    s.set_m(torch.from_numpy(m0).cuda())
    film = make_film(grid, delta, alpha=0.2)
    mo = to_xyz(m0)
    for k, bx in enumerate((-0.05, 0.0, 0.05)):
        before = s.launch_count()
        s.set_field((bx, 0.01, 0.0))
        s.step(10, dt)
        s.sync()
        # one stream-ordered write of the field, then 8 kernels per step (the
        # x-transform restarting the pipeline only before the first point)
        assert s.launch_count() - before == 1 + 10 * 8 + (1 if k == 0 else 0)
        film.b_ext = (bx, 0.01, 0.0)
        mo = film.run(mo, dt, 10, "rk4")
    mg = s.get_m().cpu().numpy()
    assert np.abs(mg - to_device(mo)).max() <= 2e-5
    s.close()
