"""The bounds-check build (libmm_b300_bc.so, -DMM_BOUNDS_CHECK): its kernels
check the shared-memory and global indices of their stores and bulk copies and
report an out-of-range one as MM_EBOUNDS instead of performing it.  Run in a
child process (the library is chosen when the binding first loads it) on small
grids that exercise every y/z route and x tile shape: no check may fire, and
the effective field and a few RK4 steps must still match the FP64 oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
from paper_1501_07293_b300 import inputs, solver
from oracle.llg import TERM_ALL
from _util import gpu_heff, make_film, make_solver, rel_l2, to_device, to_xyz
out = {"flags": solver.lib().mm_build_flags(), "cases": []}
for grid in [(40, 10, 1), (7, 5, 3), (33, 17, 5), (64, 32, 4), (100, 130, 2), (5, 3, 33), (20, 200, 40), (1, 9, 1)]:
    m = inputs.random_state(grid, 5)
    s = make_solver(grid, 4e-9, Ku=5e4, alpha=0.05)
    s.set_field((0.01, -0.02, 0.005))
    Hg = gpu_heff(s, m, TERM_ALL)
    film = make_film(grid, 4e-9, Ku=5e4, alpha=0.05, b_ext=(0.01, -0.02, 0.005))
    e = rel_l2(Hg, to_device(film.h_eff(to_xyz(m), TERM_ALL)))
    s.set_m(torch.from_numpy(m).cuda())
    s.step(3, 5e-14)
    mg = s.get_m().cpu().numpy()
    status = "ok"
    try:
        s.sync()
    except solver.MMError as err:
        status = solver.STATUS_NAMES.get(err.code, str(err.code))
    dm = float(np.abs(mg - to_device(film.run(to_xyz(m), 5e-14, 3, "rk4"))).max())
    out["cases"].append({"grid": grid, "heff_rel_l2": e, "state_diff": dm, "status": status})
    s.close()
b = solver.Batch([(40, 10, 1), (33, 17, 3), (64, 8, 2)], 5e-9, 8e5, 1.3e-11, 0.0, 0.5, 1.76e11)
for f in range(3):
    b.films[f].set_m(torch.from_numpy(inputs.random_state(b.grids[f], 9 + f)).cuda())
b.step(3, 1e-13)
try:
    b.sync(); out["batch"] = "ok"
except solver.MMError as err:
    out["batch"] = solver.STATUS_NAMES.get(err.code, str(err.code))
b.close()
print("RESULT " + json.dumps(out))
'''


def test_bounds_check_build_is_silent_and_correct():
    env = dict(os.environ, MM_B300_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                       text=True, timeout=900)
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")]
    assert r.returncode == 0 and line, r.stdout[-2000:] + r.stderr[-2000:]
    res = json.loads(line[0][len("RESULT "):])
    assert res["flags"] & 1, "the child process did not load the bounds-check build"
    for c in res["cases"]:
        assert c["status"] == "ok", c
        assert c["heff_rel_l2"] <= 1e-5, c
        assert c["state_diff"] <= 2e-5, c
    assert res["batch"] == "ok"
