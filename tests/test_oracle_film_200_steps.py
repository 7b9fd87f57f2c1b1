"""The stored 200-step trajectory of the 256 x 256 x 16 film
(tests/golden/film_256x256x16_rk4_200.json, written by the oracle alone) is
reproduced by the oracle as it stands: the FP64 RK4 run of eq. 2 with the
fields of eq. 3 - 14 from the float32 initial state, <m> every 10 steps and
the state at 512 cells at steps 100 and 200.  About 20 minutes of host time,
so it runs only when selected (-m slow); the GPU test of the same 200 steps
compares the CUDA path against the stored values."""
import json
import os

import numpy as np
import pytest

from paper_1501_07293_b300 import inputs

pytestmark = pytest.mark.slow

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "film_256x256x16_rk4_200.json")


def test_oracle_reproduces_the_stored_200_step_trajectory():
    from oracle import to_xyz
    from oracle.llg import Film
    with open(GOLDEN) as f:
        g = json.load(f)
    w = inputs.film_256x256x16()
    mat = w.mat
    film = Film(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma, b_ext=w.b_ext)
    m = to_xyz(inputs.workload_state(w).astype(np.float32))
    m = m / np.sqrt((m * m).sum(axis=0, keepdims=True))
    means = {int(r[0]): np.array(r[1:]) for r in g["mean_m"]}
    for step in range(1, g["steps"] + 1):
        m = film.rk4_step(m, w.dt)
        if step in means:
            assert np.abs(film.mean_m(m) - means[step]).max() <= 1e-12, step
        if str(step) in g["states"]:
            got = np.array([[m[a, i, j, k] for a in range(3)] for (i, j, k) in g["cells"]])
            assert np.abs(got - np.array(g["states"][str(step)])).max() <= 1e-12, step
    # the film moves: the test is not vacuous
    assert np.abs(means[g["steps"]] - means[10]).max() > 1e-4
