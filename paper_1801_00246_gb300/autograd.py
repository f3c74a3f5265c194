"""torch.autograd wrappers of the SIPDG apply and the PCG solve.

The SIPDG operator A (Eq. ellipticOp1) is symmetric, so
  * for y = A u the vector-Jacobian product is  dL/du = A (dL/dy);
  * for x = A^{-1} b it is  dL/db = A^{-1} (dL/dx), a second PCG solve with the
    same operator and preconditioner (the adjoint solve).
Both directions run through the library's CUDA kernels; nothing is computed in
PyTorch beyond argument marshalling.
"""
import torch


class _Apply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, mesh, lam, degree):
        ctx.mesh, ctx.lam, ctx.degree = mesh, lam, degree
        return mesh.apply(u.contiguous(), lam=lam, degree=degree)

    @staticmethod
    def backward(ctx, g):
        return ctx.mesh.apply(g.contiguous(), lam=ctx.lam, degree=ctx.degree), None, None, None


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, mesh, lam, opts, adjoint_opts):
        ctx.mesh, ctx.lam, ctx.opts = mesh, lam, adjoint_opts if adjoint_opts is not None else opts
        x, info = mesh.solve(b.contiguous(), lam=lam, opts=opts)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, g):
        gb, info = ctx.mesh.solve(g.contiguous(), lam=ctx.lam, opts=ctx.opts)
        ctx.adjoint_info = info
        return gb, None, None, None, None


def sipdg_apply(mesh, u, lam=0.0, degree=0):
    """Differentiable A u (u: [B][K][Np] or [K][Np] CUDA tensor)."""
    return _Apply.apply(u, mesh, float(lam), int(degree or 0))


def sipdg_solve(mesh, b, lam=0.0, opts=None, adjoint_opts=None):
    """Differentiable x = A^{-1} b by PCG (float64 b); the backward pass is the
    adjoint PCG solve with `adjoint_opts` (default: the forward options)."""
    if opts is None:
        from ._binding import default_opts
        opts = default_opts()
    return _Solve.apply(b, mesh, float(lam), opts, adjoint_opts)
