"""Writes film_256x256x16_rk4_200.json: 200 classical RK4 steps of the
256 x 256 x 16 film (the bench workload: random unit vectors, Ku 5e4 along x,
alpha 0.05, 10 mT along z, dt 5e-14 s) computed by the FP64 oracle alone
(oracle.llg.Film, eq. 2 with the fields of eq. 3 - 14), from the seeded
initial state rounded to float32 as the GPU receives it.

Stored: <m> every 10 steps, and the state at steps 100 and 200 at 512 cells
drawn with a fixed seed.  Run from the repository root:

    python tests/golden/make_film_256x256x16_rk4_200.py

(about 20 minutes on 8 host cores).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import to_xyz                    # noqa: E402
from oracle.llg import Film                  # noqa: E402
from paper_1501_07293_b300 import inputs     # noqa: E402


def main():
    w = inputs.film_256x256x16()
    mat = w.mat
    film = Film(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma, b_ext=w.b_ext)
    m = to_xyz(inputs.workload_state(w).astype(np.float32))
    m = m / np.sqrt((m * m).sum(axis=0, keepdims=True))
    nx, ny, nz = w.grid
    rng = np.random.default_rng(20200)
    cells = [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(512)]
    out = {"workload": w.name, "dt_s": w.dt, "steps": 200, "mean_m": [], "cells": cells, "states": {}}
    for step in range(1, 201):
        m = film.rk4_step(m, w.dt)
        if step % 10 == 0:
            out["mean_m"].append([step] + film.mean_m(m).tolist())
            print(step, out["mean_m"][-1][1:], flush=True)
        if step in (100, 200):
            out["states"][str(step)] = [[float(m[a, i, j, k]) for a in range(3)] for (i, j, k) in cells]
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "film_256x256x16_rk4_200.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
