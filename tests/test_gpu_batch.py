"""Batched films (mm_batch_*) vs the same films advanced one context at a time,
which are themselves parity-tested against the oracle; and the field sweep of
256 films of uneven size."""
import numpy as np
import pytest

from paper_1501_07293_b300 import inputs

pytestmark = pytest.mark.gpu

MAT = inputs.BATCH_MATERIAL
D = inputs.BATCH_DELTA
DT = inputs.BATCH_DT
GRIDS = [(40, 10, 1), (33, 17, 3), (64, 32, 4), (40, 12, 1), (17, 9, 2), (100, 3, 4), (1, 6, 2)]


def _batch(grids):
    from paper_1501_07293_b300.solver import Batch
    return Batch(grids, D, MAT.Ms, MAT.A, MAT.Ku, MAT.alpha, MAT.gamma)


def _single(grid):
    from paper_1501_07293_b300.solver import Solver
    return Solver(grid, D, MAT.Ms, MAT.A, MAT.Ku, MAT.alpha, MAT.gamma)


def _init(b, grids, seed0=100):
    import torch
    states = []
    for f, g in enumerate(grids):
        m = inputs.initial_state("tilted_x", g, seed0 + f)
        bx = (-50.0 + 100.0 * f / max(1, len(grids) - 1)) * 1e-3
        b.films[f].set_field((bx, 2e-3, 0.0))
        b.films[f].set_m(torch.from_numpy(m).cuda())
        states.append((m, (bx, 2e-3, 0.0)))
    return states


def test_batch_matches_single_contexts():
    import torch
    b = _batch(GRIDS)
    assert b.group_count() < len(GRIDS)   # films 0 and 3 share padded sizes
    assert b.schedule() == "grouped"      # film (1, 6, 2) has no persistent body
    states = _init(b, GRIDS)
    b.step(30, DT)
    for f, g in enumerate(GRIDS):
        s = _single(g)
        s.set_field(states[f][1])
        s.set_m(torch.from_numpy(states[f][0]).cuda())
        s.step(30, DT)
        want = s.get_m().cpu().numpy()
        got = b.films[f].get_m().cpu().numpy()
        assert np.abs(got - want).max() <= 1e-6, (g, np.abs(got - want).max())
        s.close()
    b.close()


def test_batch_run_stops_converged_films():
    import torch
    b = _batch(GRIDS)
    states = _init(b, GRIDS, seed0=300)
    b.step(5, DT)
    mx = b.max_dmdt()
    tol = float(np.median(mx))            # about half of the films are already below it
    b2 = _batch(GRIDS)
    _init(b2, GRIDS, seed0=300)
    steps = b2.run(60, DT, tol, check_every=10)
    assert min(steps) < 60 and max(steps) == 60, steps
    for f, g in enumerate(GRIDS):
        s = _single(g)
        s.set_field(states[f][1])
        s.set_m(torch.from_numpy(states[f][0]).cuda())
        s.step(steps[f], DT)
        want = s.get_m().cpu().numpy()
        got = b2.films[f].get_m().cpu().numpy()
        assert np.abs(got - want).max() <= 1e-6, (g, steps[f])
        s.close()
    b.close()
    b2.close()


def test_field_sweep_256_films_sampled():
    # the sweep workload: 256 films, nx in 32..256, ny in 8..128, nz in 1..4, fields -50..50 mT
    import torch
    films = inputs.film_batch()
    grids = [f.grid for f in films]
    b = _batch(grids)
    for f in films:
        b.films[f.index].set_field(f.b_ext)
        b.films[f.index].set_m(torch.from_numpy(inputs.initial_state("tilted_x", f.grid, f.seed)).cuda())
    before = b.launch_count()
    b.step(10, DT)
    torch.cuda.synchronize()
    # persistent: one kernel per step (plus the batched x transforms that start the
    # pipeline); grouped: two kernels per stage and group
    per_step = 1 if b.schedule() == "persistent" else 8
    assert b.launch_count() - before >= 10 * per_step
    for idx in (0, 77, 128, 255):
        f = films[idx]
        s = _single(f.grid)
        s.set_field(f.b_ext)
        s.set_m(torch.from_numpy(inputs.initial_state("tilted_x", f.grid, f.seed)).cuda())
        s.step(10, DT)
        assert np.abs(b.films[idx].get_m().cpu().numpy() - s.get_m().cpu().numpy()).max() <= 1e-6
        s.close()
    b.close()


def test_batch_trajectories_match_oracle():
    # four films in four padded-size groups (nz 1..4), advanced together for 30 RK4
    # steps, element by element against the FP64 oracle's own trajectories
    from oracle import to_device, to_xyz
    from oracle.llg import Film
    grids = [(40, 10, 1), (33, 17, 3), (20, 30, 4), (64, 8, 2)]
    b = _batch(grids)
    assert b.group_count() == 4
    states = _init(b, grids, seed0=500)
    b.step(30, DT)
    for f, g in enumerate(grids):
        m0, bext = states[f]
        film = Film(g, D, MAT.Ms, MAT.A, MAT.Ku, MAT.alpha, MAT.gamma, b_ext=bext)
        want = to_device(film.run(to_xyz(m0), DT, 30, "rk4"))
        got = b.films[f].get_m().cpu().numpy()
        assert np.abs(got - want).max() <= 2e-5, (g, np.abs(got - want).max())
        assert np.abs(want - m0).max() > 1e-4   # the state moves
    b.close()


def test_persistent_and_grouped_schedules_agree_with_the_oracle():
    # the same films under both schedules, 30 RK4 steps: each equals the oracle's
    # trajectories and the two agree closely
    from oracle import to_device, to_xyz
    from oracle.llg import Film
    grids = [(40, 10, 1), (33, 17, 3), (20, 30, 4), (64, 8, 2), (17, 9, 2), (100, 9, 4)]
    out = {}
    for sched in ("persistent", "grouped"):
        b = _batch(grids)
        b.set_schedule(sched)
        assert b.schedule() == sched
        states = _init(b, grids, seed0=700)
        b.step(30, DT)
        b.sync()
        out[sched] = [b.films[f].get_m().cpu().numpy() for f in range(len(grids))]
        b.close()
    for f, g in enumerate(grids):
        m0, bext = states[f]
        film = Film(g, D, MAT.Ms, MAT.A, MAT.Ku, MAT.alpha, MAT.gamma, b_ext=bext)
        want = to_device(film.run(to_xyz(m0), DT, 30, "rk4"))
        for sched in out:
            assert np.abs(out[sched][f] - want).max() <= 2e-5, (g, sched)
        assert np.abs(out["persistent"][f] - out["grouped"][f]).max() <= 1e-6, g


PGRIDS = [(40, 10, 1), (33, 17, 3), (64, 32, 4), (40, 12, 1), (17, 9, 2), (100, 9, 4), (16, 16, 2)]


def test_persistent_run_stops_converged_films():
    # mm_batch_run under both schedules: the same stop steps, the same states
    b = _batch(PGRIDS)
    assert b.schedule() == "persistent"
    _init(b, PGRIDS, seed0=300)
    b.step(5, DT)
    tol = float(np.median(b.max_dmdt()))
    b.close()
    res = {}
    for sched in ("persistent", "grouped"):
        b2 = _batch(PGRIDS)
        b2.set_schedule(sched)
        _init(b2, PGRIDS, seed0=300)
        steps = b2.run(60, DT, tol, check_every=10)
        res[sched] = (steps, [b2.films[f].get_m().cpu().numpy() for f in range(len(PGRIDS))])
        b2.close()
    steps = res["persistent"][0]
    assert min(steps) < max(steps), steps   # some films stop before others
    assert steps == res["grouped"][0]
    for f in range(len(PGRIDS)):
        assert np.abs(res["persistent"][1][f] - res["grouped"][1][f]).max() <= 1e-6


def test_persistent_wait_timeout_is_reported_and_recoverable():
    import torch
    from paper_1501_07293_b300.solver import MM_ETIMEOUT, MMError
    grids = [(40, 10, 1), (33, 17, 3)]
    b = _batch(grids)
    _init(b, grids, seed0=900)
    before = [b.films[f].get_m().clone() for f in range(2)]
    b.selftest_wait_timeout(2000)
    with pytest.raises(MMError) as e:
        b.sync()
    assert e.value.code == MM_ETIMEOUT
    b.sync()   # cleared
    for f in range(2):   # the self-test launch did no work
        assert torch.equal(b.films[f].get_m(), before[f])
    b.step(3, DT)
    b.sync()
    b.close()
