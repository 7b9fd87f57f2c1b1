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
    assert b.launch_count() - before >= 10 * 8
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
