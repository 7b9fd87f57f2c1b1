"""torch.autograd wrapper of an RK4 trajectory whose backward pass is mm_adjoint.

    m_final = llg_run(solver, m0, h, ku, n, dt, ckpt_every=50, b_ext=(0, 0, 0))

m0 ([3, nz, ny, nx]), h ([3, nz, ny, nx], tesla) and ku ([nz, ny, nx], J/m^3)
are CUDA float32 tensors; gradients flow to whichever of them requires grad.
The gradient of m0 is taken through the normalisation mm_set_m applies (it is
tangent to the sphere at the normalised initial state).  Argument marshalling
only: the forward steps and the reverse sweep run in the library's kernels.
"""
import torch


class _LLGRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m0, h, ku, solver, n, dt, ckpt_every, b_ext):
        solver.set_field(b_ext, h.detach().contiguous(), ku.detach().contiguous())
        solver.set_m(m0.detach().contiguous())
        m_start = solver.get_m().clone()
        solver.step(n, dt)
        ctx.solver = solver
        ctx.args = (n, dt, ckpt_every, b_ext)
        ctx.save_for_backward(m_start, h.detach(), ku.detach())
        return solver.get_m().clone()

    @staticmethod
    def backward(ctx, g):
        m_start, h, ku = ctx.saved_tensors
        n, dt, ckpt_every, b_ext = ctx.args
        solver = ctx.solver
        solver.set_field(b_ext, h.contiguous(), ku.contiguous())
        solver.set_m(m_start)
        gr = solver.adjoint(n, dt, ckpt_every, g.contiguous())
        return gr["m0"], gr["h"], gr["ku"], None, None, None, None, None


def llg_run(solver, m0, h, ku, n, dt, ckpt_every=50, b_ext=(0.0, 0.0, 0.0)):
    """Final state after n RK4 steps; differentiable in m0, h and ku."""
    return _LLGRun.apply(m0, h, ku, solver, int(n), float(dt), int(ckpt_every), tuple(float(b) for b in b_ext))
