"""The y/z launch-shape autotuner (paper_1501_07293_b300.tune): every candidate
gives the same field, the tuner restores the state, and its JSON cache is
applied to a new solver of the same padded size."""
import numpy as np
import pytest

from paper_1501_07293_b300 import inputs

from _util import make_solver

pytestmark = pytest.mark.gpu


def test_routes_agree_and_autotune_round_trip(tmp_path):
    import torch
    from paper_1501_07293_b300.tune import autotune
    grid, dt = (48, 40, 40), 5e-14      # a column fits one CTA, and the split pass is also a candidate
    m0 = torch.from_numpy(inputs.random_state(grid, 51)).cuda()
    s = make_solver(grid, 4e-9, Ku=5e4, alpha=0.05)
    s.set_field((0.0, 0.0, 0.01))
    fields = {}
    for route, kb in [(1, 0), (2, 8), (2, 16), (2, 0)]:
        s.set_tuning(route, kb)
        assert s.tuning()[0] == route
        s.set_m(m0)
        fields[(route, kb)] = s.heff(15).cpu().numpy()
    ref = fields[(1, 0)]
    for k, H in fields.items():
        assert np.abs(H - ref).max() <= 1e-6 * np.abs(ref).max(), k
    # stepping under the two routes
    s.set_tuning(1, 0)
    s.set_m(m0)
    s.step(5, dt)
    a = s.get_m().cpu().numpy()
    s.set_tuning(2, 16)
    s.set_m(m0)
    s.step(5, dt)
    b = s.get_m().cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6
    # the tuner restores the state and the clock, applies its choice and caches it
    s.set_tuning(0, 0)
    s.set_m(m0)
    t0 = s.time()
    cache = str(tmp_path / "tune.json")
    rec = autotune(s, dt, cache=cache)
    assert len(rec["candidates"]) >= 3
    assert s.tuning() == (rec["yz_route"], rec["zt_block"] or s.tuning()[1])
    # (set_m renormalises: equal up to the rounding of a second normalisation)
    assert np.abs(s.get_m().cpu().numpy() - m0.cpu().numpy()).max() <= 1e-6
    assert s.time() == t0
    t = make_solver(grid, 4e-9, Ku=5e4, alpha=0.05, tune_cache=cache)
    assert t.tuning()[0] == rec["yz_route"]
    t.close()
    s.close()


def test_tuning_arguments():
    from paper_1501_07293_b300.solver import MM_EINVAL, MM_EUNSUPPORTED, MMError
    s = make_solver((20, 200, 40), 4e-9)    # a column does not fit one CTA: no fused route
    with pytest.raises(MMError) as e:
        s.set_tuning(1, 0)
    assert e.value.code == MM_EUNSUPPORTED
    with pytest.raises(MMError) as e:
        s.set_tuning(3, 0)
    assert e.value.code == MM_EINVAL
    with pytest.raises(MMError) as e:
        s.set_tuning(2, 4)
    assert e.value.code == MM_EINVAL
    s.close()
