"""mm_heff_noalloc: the context-free, allocation-free effective field.

Some callers cannot call cudaMalloc -- a plug-in whose host application owns
the GPU's memory pool, code running where a caching allocator already holds
the free device memory, a loop that cannot take the device-wide
synchronisation of an allocation -- so the library offers an entry point whose
scratch is a static device array.  Its result must equal mm_heff of a context
created with the same parameters and holding the same state, within the
parity tolerance of the other tests (relative L2 <= 1e-5), on calls in a row
that reuse the scratch earlier calls left behind, including a repeat of the
first case after a different grid has overwritten the array.  The kernels'
error flags are read back by mm_noalloc_status; a wait that runs out on
purpose (the wait self-test) must be reported there and cleared.

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


def test_noalloc_matches_mm_heff_on_calls_in_a_row():
    import torch
    from paper_1501_07293_b300.solver import TERM_ALL, TERM_DEMAG, heff_noalloc, noalloc_status
    cases = [((40, 10, 3), 5e-9, 8e5, 1.3e-11, 5e4, (0.01, -0.02, 0.005), TERM_ALL, True, 1),
             ((24, 33, 2), 4e-9, 8e5, 1.3e-11, 0.0, (0.0, 0.0, 0.01), TERM_DEMAG, False, 2)]
    refs = []
    for grid, delta, Ms, A, Ku, b, mask, self_term, seed in cases:
        m_np = inputs.random_state(grid, seed)
        refs.append(_reference(grid, delta, Ms, A, Ku, b, m_np, mask, self_term))
    order = (0, 1, 0)   # case 1, case 2, then case 1 again over what case 2 left behind
    outs = [torch.empty_like(refs[q][0]) for q in order]
    # one call of each case first: the library's module and the kernels' local
    # memory are set up by the CUDA driver on first use, which is not the call's
    # own allocation; after that the device's free memory must not move
    for q in (0, 1):
        grid, delta, Ms, A, Ku, b, mask, self_term, _ = cases[q]
        heff_noalloc(grid, delta, Ms, A, Ku, b, refs[q][1], outs[q], mask, self_term)
    noalloc_status()
    for H in outs:
        H.fill_(float("nan"))
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for H, q in zip(outs, order):
        grid, delta, Ms, A, Ku, b, mask, self_term, _ = cases[q]
        heff_noalloc(grid, delta, Ms, A, Ku, b, refs[q][1], H, mask, self_term)
        noalloc_status()   # synchronises; no kernel flagged anything
    assert torch.cuda.mem_get_info()[0] == free_before
    for H, q in zip(outs, order):
        H_ref = refs[q][0]
        assert torch.isfinite(H).all()
        assert _rel(H, H_ref) <= TOL, (cases[q][0], _rel(H, H_ref))


def test_noalloc_reports_a_wait_that_ran_out():
    import torch
    from paper_1501_07293_b300.solver import (MM_ETIMEOUT, TERM_ALL, MMError, heff_noalloc,
                                              noalloc_selftest_wait_timeout, noalloc_status)
    noalloc_status()
    noalloc_selftest_wait_timeout(2000)   # sets the scratch's timeout flag, no fault
    with pytest.raises(MMError) as e:
        noalloc_status(torch.cuda.default_stream())
    assert e.value.code == MM_ETIMEOUT
    noalloc_status()                      # the flag was cleared
    grid = (16, 8, 2)
    m_np = inputs.random_state(grid, 3)
    H_ref, m = _reference(grid, 4e-9, 8e5, 1.3e-11, 0.0, (0, 0, 0.01), m_np, TERM_ALL, True)
    H = torch.zeros_like(H_ref)
    heff_noalloc(grid, 4e-9, 8e5, 1.3e-11, 0.0, (0, 0, 0.01), m, H)
    noalloc_status()
    assert _rel(H, H_ref) <= TOL


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
