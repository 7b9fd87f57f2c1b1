"""Time-dependent uniform field and damping (a field program), FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3 runs the standard-problem-4 film through a protocol (the script of
Appendix A): a saturating field along (1, 1, 1), a linear ramp down to zero,
relaxation at zero field, then the reversing field with the damping lowered
from 0.5 to 0.02.  A program is a list of segments
(t_begin, t_end, b_begin, b_end, alpha): at time t the first segment with
t_begin <= t < t_end applies, with the field linear in t between its end
values and alpha < 0 meaning the film's own damping; outside every segment the
film's b_ext and alpha apply.

The program turns eq. 2 into dm/dt = f(t, m), and the integrators evaluate it
where a time-dependent ODE is evaluated: explicit Euler at t_n, classical RK4
at t_n, t_n + dt/2, t_n + dt/2 and t_n + dt.  Renormalisation after the full
step as in the constant-field integrators of llg.py.

Pins (tests/test_oracle_program.py): the paper's schedule conditions written
per step index; the macrospin closed form under a piecewise-linear field along
z with a damping switch where the field is zero.
"""
import numpy as np

from . import MU0
from .llg import TERM_ALL, TERM_ZEEMAN, llg_rhs, normalise, zeeman_field


class FieldProgram:
    def __init__(self, segments, b_base=(0.0, 0.0, 0.0), alpha_base=0.0):
        self.segments = [(float(t0), float(t1), np.asarray(b0, dtype=np.float64),
                          np.asarray(b1, dtype=np.float64), float(al)) for t0, t1, b0, b1, al in segments]
        self.b_base = np.asarray(b_base, dtype=np.float64)
        self.alpha_base = float(alpha_base)

    def at(self, t):
        """(b_ext (tesla, shape (3,)), alpha) at time t."""
        for t0, t1, b0, b1, al in self.segments:
            if t0 <= t < t1:
                f = (t - t0) / (t1 - t0)
                return b0 + f * (b1 - b0), (al if al >= 0.0 else self.alpha_base)
        return self.b_base.copy(), self.alpha_base


def program_for(film, segments):
    """The program of ``segments`` with the film's own b_ext and alpha outside them."""
    return FieldProgram(segments, film.b_ext, film.alpha)


def rhs_at(film, m, t, program):
    """Eq. 2 at time t: every field term of the film except its uniform field,
    which (with the damping) comes from the program."""
    b, alpha = program.at(t)
    H = film.h_eff(m, TERM_ALL & ~TERM_ZEEMAN) + zeeman_field(m.shape, b, film.h_map)
    return llg_rhs(m, MU0 * H, alpha, film.gamma)


def euler_step_at(film, m, t, dt, program):
    return normalise(m + dt * rhs_at(film, m, t, program))


def rk4_step_at(film, m, t, dt, program):
    k1 = rhs_at(film, m, t, program)
    k2 = rhs_at(film, m + 0.5 * dt * k1, t + 0.5 * dt, program)
    k3 = rhs_at(film, m + 0.5 * dt * k2, t + 0.5 * dt, program)
    k4 = rhs_at(film, m + dt * k3, t + dt, program)
    return normalise(m + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4))


def run_program(film, m, t0, dt, steps, program, integrator="rk4", sample_every=0, callback=None):
    """Advance ``steps`` steps from time t0; callback(step, t, m) every sample_every steps.
    Returns (m, t) with t = t0 + steps dt accumulated step by step."""
    m = np.asarray(m, dtype=np.float64)
    step = rk4_step_at if integrator == "rk4" else euler_step_at
    t = float(t0)
    for s in range(1, steps + 1):
        m = step(film, m, t, dt, program)
        t = t + dt
        if sample_every and callback is not None and s % sample_every == 0:
            callback(s, t, m)
    return m, t
