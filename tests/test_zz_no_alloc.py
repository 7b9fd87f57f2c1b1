"""mm_heff_noalloc: the context-free, allocation-free effective field.

Some callers cannot call cudaMalloc -- code running during CUDA-graph stream
capture, or code whose device memory belongs to another allocator -- so the
library offers an entry point whose scratch is a static device array.  Its
result must equal mm_heff of a context created with the same parameters and
holding the same state, within the parity tolerance of the other tests
(relative L2 <= 1e-5), on two calls in a row (the second call reuses the
scratch the first one left behind).

This file is collected last so that a run stopped at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1501_07293_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm())


def _reference(grid, delta, Ms, A, Ku, b, m_np, mask, self_term):
    """H from the context-based entry point, and the normalised state it used."""
    import torch
    from paper_1501_07293_b300.solver import Solver
    s = Solver(grid, delta, Ms, A, Ku, 0.02, 1.76e11, self_term=self_term)
    s.set_field(b)
    s.set_m(torch.from_numpy(m_np).cuda())
    H = s.heff(mask).clone()
    m = s.get_m().clone()
    torch.cuda.synchronize()
    s.close()
    return H, m


def test_noalloc_matches_mm_heff_twice():
    import torch
    from paper_1501_07293_b300.solver import TERM_ALL, TERM_DEMAG, heff_noalloc
    cases = [((40, 10, 3), 5e-9, 8e5, 1.3e-11, 5e4, (0.01, -0.02, 0.005), TERM_ALL, True, 1),
             ((24, 33, 2), 4e-9, 8e5, 1.3e-11, 0.0, (0.0, 0.0, 0.01), TERM_DEMAG, False, 2)]
    for grid, delta, Ms, A, Ku, b, mask, self_term, seed in cases:
        m_np = inputs.random_state(grid, seed)
        H_ref, m = _reference(grid, delta, Ms, A, Ku, b, m_np, mask, self_term)
        H = torch.full_like(H_ref, float("nan"))
        heff_noalloc(grid, delta, Ms, A, Ku, b, m, H, mask, self_term)
        torch.cuda.synchronize()
        assert torch.isfinite(H).all()
        assert _rel(H, H_ref) <= TOL, (grid, _rel(H, H_ref))


def test_noalloc_refuses_grids_beyond_the_scratch():
    import torch
    from paper_1501_07293_b300.solver import MM_EUNSUPPORTED, MMError, heff_noalloc
    grid = (256, 256, 4)
    m = torch.zeros((3, 4, 256, 256), dtype=torch.float32, device="cuda")
    H = torch.zeros_like(m)
    with pytest.raises(MMError) as e:
        heff_noalloc(grid, 4e-9, 8e5, 1.3e-11, 0.0, (0, 0, 0), m, H)
    assert e.value.code == MM_EUNSUPPORTED
    assert float(H.abs().max()) == 0.0   # nothing was launched
