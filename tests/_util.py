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


def sample_cells(grid, n_random, seed):
    """Target cells for sampled parity: the 8 corners, the midpoints of the 12 edges,
    the centres of the 6 faces (so both z faces are covered), and n_random seeded
    cells; (i, j, k) in paper order."""
    nx, ny, nz = grid
    pick = lambda n: sorted({0, n // 2, n - 1})
    cells = set()
    for i in pick(nx):
        for j in pick(ny):
            for k in pick(nz):
                # corners (three end values), edge midpoints (one centre), face centres (two)
                centres = (i == nx // 2) + (j == ny // 2) + (k == nz // 2)
                if centres <= 2:
                    cells.add((i, j, k))
    rng = np.random.default_rng(seed)
    while len(cells) < 26 + n_random:
        cells.add((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    return sorted(cells)


def per_cell_rel(Hg_dev, Ho_cells, cells):
    """max over the sampled cells of |H_gpu - H_oracle| / |H_oracle| (vector norms)."""
    Hgc = np.array([[Hg_dev[a, k, j, i] for a in range(3)] for (i, j, k) in cells])
    num = np.linalg.norm(Hgc - Ho_cells, axis=1)
    den = np.linalg.norm(Ho_cells, axis=1)
    return float((num / den).max())


__all__ = ["sample_cells", "per_cell_rel", "rel_l2", "make_solver", "make_film", "gpu_heff", "to_device", "to_xyz"]
