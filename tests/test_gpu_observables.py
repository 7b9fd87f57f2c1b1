"""Observables recorded inside the step graph (mm_opts.obs_every, mm_get_series)
vs the FP64 oracle's trajectory: <m> of the state after every obs_every-th step,
max|dm/dt| at that step's start, the clock and the step count."""
import numpy as np
import pytest

from paper_1501_07293_b300 import inputs

from _util import make_film, make_solver, to_xyz

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("integ", ["rk4", "euler"])
def test_series_matches_oracle(integ):
    import torch
    grid, dt, every = (24, 12, 3), 5e-14, 10
    m0 = inputs.random_state(grid, 41)
    s = make_solver(grid, 4e-9, Ku=5e4, alpha=0.05, integrator=integ, obs_every=every)
    s.set_field((0.0, 0.0, 0.01))
    s.set_m(torch.from_numpy(m0).cuda())
    before = s.launch_count()
    s.step(23, dt)            # the cadence runs across calls
    s.step(27, dt)
    s.sync()
    per_step = (8 if integ == "rk4" else 2) + 1
    assert s.launch_count() - before == 1 + 50 * per_step
    rec = s.series()
    assert rec.shape == (5, 6)
    film = make_film(grid, 4e-9, Ku=5e4, alpha=0.05, b_ext=(0.0, 0.0, 0.01))
    step = film.rk4_step if integ == "rk4" else film.euler_step
    m = to_xyz(m0)
    want = []
    for k in range(1, 51):
        if k % every == 0:
            start_rate = film.max_dmdt(m)
        m = step(m, dt)
        if k % every == 0:
            want.append((k * dt, k, *film.mean_m(m), start_rate))
    want = np.array(want)
    assert np.allclose(rec[:, 0], want[:, 0], rtol=1e-12)
    assert np.array_equal(rec[:, 1], want[:, 1])
    assert np.abs(rec[:, 2:5] - want[:, 2:5]).max() <= 1e-5
    assert np.all(np.abs(rec[:, 5] - want[:, 5]) <= 1e-4 * want[:, 5])
    s.close()


def test_series_restarts_with_the_state_and_off_is_einval():
    import torch
    from paper_1501_07293_b300.solver import MM_EINVAL, MMError
    grid = (16, 8, 2)
    s = make_solver(grid, 4e-9, obs_every=3)
    m0 = torch.from_numpy(inputs.random_state(grid, 42)).cuda()
    s.set_m(m0)
    s.step(7, 1e-13)
    assert s.series().shape[0] == 2
    s.set_m(m0)
    assert s.series().shape[0] == 0
    s.step(3, 1e-13)
    r = s.series()
    assert r.shape[0] == 1 and r[0, 1] == 3
    s.close()
    t = make_solver(grid, 4e-9)
    with pytest.raises(MMError) as e:
        t.series()
    assert e.value.code == MM_EINVAL
    t.close()
