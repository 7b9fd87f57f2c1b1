"""mm_set_m / mm_get_m with the three kinds of source memory.

mm_set_m reads page-locked host memory directly from its normalising kernel
(when the cell count is a multiple of 4), and copies device or pageable host
memory before normalising in place.  All routes must store the same unit
vectors bit for bit, keep a zero or non-finite input vector as given and flag
it (MM_ENONFINITE at the next synchronising call), and give the same state
after steps.
"""
import numpy as np
import pytest

from paper_1501_07293_b300 import inputs

from _util import make_solver

pytestmark = pytest.mark.gpu


def _raw_state(grid, seed):
    # unit vectors scaled by per-cell magnitudes in [0.5, 2): normalisation matters
    m = inputs.random_state(grid, seed).astype(np.float32)
    scale = np.random.default_rng(seed + 1).uniform(0.5, 2.0, size=m.shape[1:]).astype(np.float32)
    return np.ascontiguousarray(m * scale[None])


@pytest.mark.parametrize("grid", [(40, 10, 3), (25, 13, 3), (256, 256, 16)])
def test_set_m_routes_store_the_same_state(grid):
    import torch
    m = _raw_state(grid, 7)
    s = make_solver(grid, 4e-9)
    got = []
    for src in (torch.from_numpy(m).cuda(), torch.from_numpy(m).pin_memory(), torch.from_numpy(m.copy())):
        s.set_m(src)
        got.append(s.get_m().cpu().numpy())
        s.sync()
    s.close()
    ref = m / np.sqrt((m.astype(np.float64) ** 2).sum(axis=0))[None]
    assert np.abs(got[0] - ref).max() <= 5e-7
    for g in got[1:]:
        assert np.array_equal(g, got[0])


def test_set_m_from_pinned_memory_flags_a_nonfinite_vector():
    import torch
    from paper_1501_07293_b300.solver import MM_ENONFINITE, MMError
    grid = (8, 4, 2)
    m = _raw_state(grid, 2)
    m[1, 1, 2, 3] = np.nan
    m[:, 0, 0, 0] = 0.0
    h = torch.from_numpy(m).pin_memory()
    s = make_solver(grid, 4e-9)
    s.set_m(h)
    with pytest.raises(MMError) as e:
        s.sync()
    assert e.value.code == MM_ENONFINITE
    got = s.get_m().cpu().numpy()
    s.close()
    assert np.isnan(got[1, 1, 2, 3]) and (got[:, 0, 0, 0] == 0).all()   # passed through as given


def test_steps_from_pinned_and_device_sources_agree():
    import torch
    grid = (64, 32, 4)
    m = _raw_state(grid, 11)
    out = []
    for src in (torch.from_numpy(m).cuda(), torch.from_numpy(m).pin_memory()):
        s = make_solver(grid, 4e-9, Ku=5e4, alpha=0.05)
        s.set_field((0.0, 0.0, 0.01))
        s.set_m(src)
        s.step(5, 5e-14)
        out.append(s.get_m().cpu().numpy())
        s.close()
    assert np.array_equal(out[0], out[1])
