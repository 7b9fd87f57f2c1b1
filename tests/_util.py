"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

from oracle import to_device, to_xyz


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_solver(w_or_grid, delta=None, Ms=8e5, A=1.3e-11, Ku=0.0, alpha=0.02, gamma=1.76e11, **kw):
    from paper_1501_07293_b300.solver import Solver
    return Solver(w_or_grid, delta, Ms, A, Ku, alpha, gamma, **kw)


def make_film(grid, delta, Ms=8e5, A=1.3e-11, Ku=0.0, alpha=0.02, gamma=1.76e11, b_ext=(0, 0, 0),
              h_map_dev=None, ku_map_dev=None, self_term=True, demag="fft"):
    from oracle.llg import Film
    return Film(grid, delta, Ms, A, Ku, alpha, gamma, b_ext=b_ext,
                h_map=None if h_map_dev is None else to_xyz(h_map_dev),
                ku_map=None if ku_map_dev is None else to_xyz(ku_map_dev),
                self_term=self_term, demag=demag)


def gpu_heff(solver, m_dev_np, mask):
    import torch
    solver.set_m(torch.from_numpy(m_dev_np).cuda())
    H = solver.heff(mask)
    torch.cuda.synchronize()
    return H.cpu().numpy().astype(np.float64)


__all__ = ["rel_l2", "make_solver", "make_film", "gpu_heff", "to_device", "to_xyz"]
