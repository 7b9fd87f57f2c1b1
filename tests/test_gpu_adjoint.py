"""mm_adjoint (through the C ABI and the autograd wrapper) vs the FP64 oracle
adjoint, and vs finite differences of the GPU's own forward trajectory.

Bar (FP32): gradients within 1e-3 relative L2 of the oracle's FP64 adjoint
(which is itself pinned to FP64 finite differences), and directional
derivatives within 1e-3 of central differences at full size.
"""
import numpy as np
import pytest

from oracle import to_device, to_xyz
from oracle.adjoint import AdjointFilm, tangent_project
from paper_1501_07293_b300 import inputs

from _util import make_film, make_solver, rel_l2

pytestmark = pytest.mark.gpu

TARGET = np.array([0.0, 1.0, 0.0])


def _loss_grad_final(m):
    """L = ||<m> - (0,1,0)||^2 and dL/dm (the per-cell broadcast of 2 (<m> - t) / N)."""
    mean = m.reshape(3, -1).mean(axis=1)
    N = m[0].size
    g = np.broadcast_to((2.0 * (mean - TARGET) / N)[:, None, None, None], m.shape)
    return float(((mean - TARGET) ** 2).sum()), np.ascontiguousarray(g)


def _small_case(n_steps, ckpt):
    import torch
    w = inputs.film_16x8x1()
    mat = w.mat
    grid = w.grid
    m0 = inputs.workload_state(w)
    h = inputs.zeeman_map(grid, 5101)
    ku = inputs.ku_map(grid, 5102)
    s = make_solver(grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=0.0, alpha=mat.alpha, gamma=mat.gamma)
    s.set_field((0.0, 0.0, 0.0), torch.from_numpy(h).cuda(), torch.from_numpy(ku).cuda())
    s.set_m(torch.from_numpy(m0).cuda())
    m0n = s.get_m().cpu().numpy()
    s.step(n_steps, w.dt)
    mf = s.get_m().cpu().numpy().astype(np.float64)
    _, g = _loss_grad_final(mf)
    s.set_m(torch.from_numpy(m0n).cuda())
    gr = s.adjoint(n_steps, w.dt, ckpt, torch.from_numpy(g.astype(np.float32)).cuda())
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()}
    s.close()
    return w, m0n, h, ku, out


def test_adjoint_matches_oracle_16x8x1():
    n = 40
    w, m0n, h, ku, gpu = _small_case(n, 7)   # ragged last segment
    mat = w.mat
    film = make_film(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=0.0, alpha=mat.alpha, gamma=mat.gamma,
                     h_map_dev=h, ku_map_dev=ku)
    adj = AdjointFilm(film)
    m0x = to_xyz(m0n)
    mf, rec = adj.forward(m0x, w.dt, n)
    _, g = _loss_grad_final(to_device(mf))
    gm, gh, gk = adj.backward(rec, w.dt, to_xyz(g))
    gm = tangent_project(m0x, gm)
    assert rel_l2(gpu["m0"], to_device(gm)) <= 1e-3
    assert rel_l2(gpu["h"], to_device(gh)) <= 1e-3
    assert rel_l2(gpu["ku"], to_device(gk)) <= 1e-3


def test_adjoint_matches_oracle_16x8x1_full_500_steps():
    # the differentiation study's small copy over its full length: 500 RK4 steps,
    # a checkpoint every 50 (full-length segments: the captured segment graph)
    n = 500
    w, m0n, h, ku, gpu = _small_case(n, 50)
    mat = w.mat
    film = make_film(w.grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=0.0, alpha=mat.alpha, gamma=mat.gamma,
                     h_map_dev=h, ku_map_dev=ku)
    adj = AdjointFilm(film)
    m0x = to_xyz(m0n)
    mf, rec = adj.forward(m0x, w.dt, n)
    _, g = _loss_grad_final(to_device(mf))
    gm, gh, gk = adj.backward(rec, w.dt, to_xyz(g))
    gm = tangent_project(m0x, gm)
    assert rel_l2(gpu["m0"], to_device(gm)) <= 1e-3
    assert rel_l2(gpu["h"], to_device(gh)) <= 1e-3
    assert rel_l2(gpu["ku"], to_device(gk)) <= 1e-3


def test_adjoint_is_independent_of_checkpoint_spacing():
    ref = _small_case(12, 12)[4]
    for k in (1, 5):
        got = _small_case(12, k)[4]
        for key in ref:
            assert np.array_equal(got[key], ref[key]), (k, key)


def test_recorded_segments_give_the_same_gradients_bit_for_bit():
    # mm_set_adjoint_memory lets the forward pass record more trailing segments
    # (R = 1, 3, then all 7 of 47 steps at a checkpoint every 7, the last one
    # ragged); the sweep sees the same stage data, so every output and the
    # final state must equal the default's exactly, on one context in a row
    import torch
    w = inputs.film_16x8x1()
    mat = w.mat
    grid = w.grid
    n, k = 47, 7
    s = make_solver(grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=0.0, alpha=mat.alpha, gamma=mat.gamma)
    s.set_field((0.0, 0.0, 0.0), torch.from_numpy(inputs.zeeman_map(grid, 5201)).cuda(),
                torch.from_numpy(inputs.ku_map(grid, 5202)).cuda())
    m0 = torch.from_numpy(inputs.workload_state(w)).cuda()
    g = torch.full((3, grid[2], grid[1], grid[0]), 1e-3, dtype=torch.float32, device="cuda")
    slot = 12 * (8 * k + 1) * grid[0] * grid[1] * grid[2]
    runs = []
    for budget in (0, 3 * slot, 1e12, 0):
        s.set_adjoint_memory(budget)
        s.set_m(m0)
        gr = s.adjoint(n, w.dt, k, g)
        runs.append(({key: v.cpu().numpy() for key, v in gr.items()}, s.get_m().cpu().numpy()))
    s.close()
    ref, mref = runs[0]
    for got, mf in runs[1:]:
        assert np.array_equal(mf, mref)
        for key in ref:
            assert np.isfinite(got[key]).all()
            assert np.array_equal(got[key], ref[key]), key


def test_adjoint_memory_rejects_bad_budgets():
    from paper_1501_07293_b300.solver import MM_EINVAL, MMError
    s = make_solver((8, 4, 1), 4e-9, Ms=8e5, A=1.3e-11, Ku=0.0, alpha=0.02, gamma=1.76e11)
    for bad in (-1.0, float("nan")):
        with pytest.raises(MMError) as e:
            s.set_adjoint_memory(bad)
        assert e.value.code == MM_EINVAL
    s.close()


def test_autograd_wrapper_full_size_directional_fd():
    # the differentiation study at full size: 128x128x4, 500 RK4 steps, checkpoint every 50
    import torch
    from paper_1501_07293_b300.autograd import llg_run
    w = inputs.film_128x128x4()
    mat = w.mat
    grid = w.grid
    s = make_solver(grid, w.delta, Ms=mat.Ms, A=mat.A, Ku=0.0, alpha=mat.alpha, gamma=mat.gamma)
    m0 = torch.from_numpy(inputs.workload_state(w)).cuda()
    h = torch.from_numpy(inputs.zeeman_map(grid, 5001)).cuda().requires_grad_(True)
    ku = torch.from_numpy(inputs.ku_map(grid, 5002)).cuda().requires_grad_(True)
    target = torch.tensor([0.0, 1.0, 0.0], device="cuda", dtype=torch.float64)

    def loss_of(mf):
        mean = mf.double().reshape(3, -1).mean(dim=1)
        return ((mean - target) ** 2).sum()

    mf = llg_run(s, m0, h, ku, w.steps, w.dt, 50)
    L = loss_of(mf)
    L.backward()
    gh, gk = h.grad.double(), ku.grad.double()

    def L_at(hh, kk):
        with torch.no_grad():
            return float(loss_of(llg_run(s, m0, hh, kk, w.steps, w.dt, 50)))

    # coherent directions give a change well above the FP32 noise of the loss
    dh = torch.zeros_like(h)
    dh[1] = 1e-3
    eps = 1.0
    fd = (L_at(h.detach() + eps * dh, ku.detach()) - L_at(h.detach() - eps * dh, ku.detach())) / (2 * eps)
    ad = float((gh * dh.double()).sum())
    assert abs(ad - fd) <= 1e-3 * abs(fd), (ad, fd)
    dk = torch.full_like(ku, 500.0)
    fd = (L_at(h.detach(), ku.detach() + dk) - L_at(h.detach(), ku.detach() - dk)) / 2.0
    ad = float((gk * dk.double()).sum())
    assert abs(ad - fd) <= 1e-3 * abs(fd), (ad, fd)
    s.close()
