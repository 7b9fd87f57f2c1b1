"""Pins of the oracle's field program (oracle/program.py) and of the
standard-problem-4 schedule (Section 3, script of Appendix A)."""
import numpy as np
import pytest

from oracle import MU0
from oracle.llg import Film
from oracle.program import FieldProgram, program_for, run_program
from paper_1501_07293_b300 import inputs

GAMMA = 1.76e11


def _script_field(t):
    """The script's applied field (kA/m) and damping for its step index t = 1, 2, ...,
    with the ramp applied to every component (the reading stated in sp4_schedule)."""
    if t < 4000:
        return np.array([100.0, 100.0, 100.0]), 0.5
    if t < 6000:
        return np.full(3, (6000 - t) / 20.0), 0.5
    if t <= 50000:
        return np.zeros(3), 0.5
    return np.array([-19.576, 3.422, 0.0]), 0.02


def test_sp4_schedule_matches_the_scripts_step_conditions():
    dt = inputs.sp4_film().dt
    prog = FieldProgram(inputs.sp4_schedule(dt), alpha_base=0.5)
    ts = [1, 2, 3998, 3999, 4000, 4001, 4500, 5998, 5999, 6000, 6001, 20000, 49999, 50000, 50001,
          50002, 149999, 150000]
    clock = 0.0
    n = 0
    for t in ts:
        # the clock as a device would hold it: dt added once per step
        while n < t - 1:
            clock += dt
            n += 1
        for time in (clock, (t - 1) * dt):
            b, alpha = prog.at(time)
            want_h, want_alpha = _script_field(t)
            assert np.allclose(b / MU0 / 1e3, want_h, rtol=1e-9, atol=1e-9), (t, b / MU0 / 1e3, want_h)
            assert alpha == want_alpha, t


def test_sp4_reverse_field_is_the_papers_tesla_values():
    # Section 3 quotes the reversing field as (-24.6, 4.3, 0) mT
    b = inputs.sp4_schedule(5e-15)[-1][2]
    assert abs(b[0] * 1e3 + 24.6) < 0.01 and abs(b[1] * 1e3 - 4.3) < 0.01 and b[2] == 0.0


def test_macrospin_closed_form_under_a_program_rk4():
    # One cell: only the applied field exerts torque (see test_oracle_llg).  For
    # b(t) along z, eq. 2 integrates to
    #   phi(t) = phi0 + int gamma/(1+alpha^2) b dt
    #   ln tan(theta/2) = ln tan(theta0/2) - int alpha gamma/(1+alpha^2) b dt,
    # whatever the time dependence.  The program ramps b down to zero, switches
    # the damping while b = 0, then ramps b negative; every kink sits on a step
    # time, so RK4 sees a field linear in t within each step and stays at its
    # O(dt^4) accuracy.  Stage times taken at t_n instead would be off by ~1e-2 rad.
    dt, n1, n2, n3 = 2e-13, 400, 600, 1000
    segs = [(0.0, n1 * dt, (0, 0, 0.5), (0, 0, 0.0), 0.5),
            (n1 * dt, n2 * dt, (0, 0, 0.0), (0, 0, 0.0), 0.02),
            (n2 * dt, (n3 + n3 - n2) * dt, (0, 0, 0.0), (0, 0, -0.6), 0.02)]   # -0.3 T at n3 dt
    film = Film((1, 1, 1), 5e-9, 8e5, 1.3e-11, 0.0, 0.5, GAMMA, demag="direct")
    th0, ph0 = 1.0, 0.3
    m0 = np.array([np.sin(th0) * np.cos(ph0), np.sin(th0) * np.sin(ph0), np.cos(th0)]).reshape(3, 1, 1, 1)
    m, t = run_program(film, m0, 0.0, dt, n3, program_for(film, segs), "rk4")
    assert abs(t - n3 * dt) < 1e-12 * n3 * dt
    gA, gC = GAMMA / (1 + 0.25), GAMMA / (1 + 0.02 ** 2)
    areaA, areaC = 0.5 * n1 * dt / 2, -0.3 * (n3 - n2) * dt / 2
    phi = ph0 + gA * areaA + gC * areaC
    theta = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-0.5 * gA * areaA - 0.02 * gC * areaC))
    want = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    assert np.abs(m.reshape(3) - want).max() < 1e-8


def test_constant_program_equals_the_constant_field_integrator():
    grid = (6, 4, 2)
    rng = np.random.default_rng(7)
    h = rng.normal(0, 5e-3, size=(3,) + grid)
    ku = rng.uniform(0, 1e5, size=grid)
    m0 = rng.standard_normal((3,) + grid)
    m0 /= np.sqrt((m0 * m0).sum(axis=0))
    b, alpha = (0.01, -0.02, 0.005), 0.1
    ref = Film(grid, 5e-9, 8e5, 1.3e-11, 0.0, alpha, GAMMA, b_ext=b, h_map=h, ku_map=ku)
    want = ref.run(m0, 1e-13, 10, "rk4")
    film = Film(grid, 5e-9, 8e5, 1.3e-11, 0.0, 0.5, GAMMA, b_ext=(0.3, 0.3, 0.3), h_map=h, ku_map=ku)
    got, _ = run_program(film, m0, 0.0, 1e-13, 10, program_for(film, [(0.0, 1.0, b, b, alpha)]), "rk4")
    assert np.abs(got - want).max() < 1e-14


def test_euler_program_step_equals_concatenated_constant_runs():
    # Euler evaluates the program only at t_n: a switch at 5.5 dt gives 6 steps
    # with the first field and the rest with the second, exactly
    grid = (5, 3, 1)
    rng = np.random.default_rng(8)
    m0 = rng.standard_normal((3,) + grid)
    m0 /= np.sqrt((m0 * m0).sum(axis=0))
    dt = 1e-13
    b1, b2 = (0.02, 0.0, 0.01), (-0.03, 0.01, 0.0)
    first = Film(grid, 5e-9, 8e5, 1.3e-11, 0.0, 0.5, GAMMA, b_ext=b1)
    second = Film(grid, 5e-9, 8e5, 1.3e-11, 0.0, 0.02, GAMMA, b_ext=b2)
    want = second.run(first.run(m0, dt, 6, "euler"), dt, 4, "euler")
    film = Film(grid, 5e-9, 8e5, 1.3e-11, 0.0, 0.5, GAMMA)
    prog = program_for(film, [(0.0, 5.5 * dt, b1, b1, -1.0), (5.5 * dt, 1.0, b2, b2, 0.02)])
    got, _ = run_program(film, m0, 0.0, dt, 10, prog, "euler")
    assert np.abs(got - want).max() < 1e-14


def test_program_lookup_first_segment_wins_and_base_outside():
    prog = FieldProgram([(0.0, 2.0, (1, 0, 0), (3, 0, 0), -1.0), (1.0, 4.0, (0, 5, 0), (0, 5, 0), 0.3)],
                        b_base=(0, 0, 7), alpha_base=0.9)
    b, a = prog.at(1.5)
    assert np.allclose(b, (2.5, 0, 0)) and a == 0.9
    b, a = prog.at(2.0)
    assert np.allclose(b, (0, 5, 0)) and a == 0.3
    b, a = prog.at(4.0)
    assert np.allclose(b, (0, 0, 7)) and a == 0.9
    b, a = prog.at(-1.0)
    assert np.allclose(b, (0, 0, 7)) and a == 0.9
