"""Adjoints of the apply and of the solve (torch.autograd) against dense
reference gradients and central finite differences."""
import numpy as np
import pytest

from dg_inputs import config_mesh, jittered_grid, uniform_field
from dg_inputs.fields import fourier_eval, fourier_rhs_coeffs
from dg_inputs.mesh import rotate_local_vertices
from tests.gpu_util import cuda, pair, pkg, rel

pytestmark = pytest.mark.gpu


def test_apply_vjp_is_the_operator():
    import torch
    from paper_1801_00246_gb300.autograd import sipdg_apply
    m = rotate_local_vertices(jittered_grid(5, 4, seed=2), 1)
    lib, ora = pair(m, 5)
    u = cuda(uniform_field((2, m.K, ora.Np), seed=1)).requires_grad_(True)
    w = uniform_field((2, m.K, ora.Np), seed=2)
    y = sipdg_apply(lib, u, lam=0.5)
    (y * cuda(w)).sum().backward()
    A = ora.assemble(0.5)
    ref = np.stack([(A.T @ w[k].ravel()).reshape(m.K, ora.Np) for k in range(2)])
    assert rel(u.grad.cpu().numpy(), ref) <= 1e-12


def test_solve_gradient_matches_dense_reference():
    """Tiny mesh: dL/db = 2 A^{-1} (p - p*) from the dense oracle matrix."""
    import torch
    P = pkg()
    from paper_1801_00246_gb300.autograd import sipdg_solve
    m = rotate_local_vertices(jittered_grid(4, 4, seed=1), 3)
    lib, ora = pair(m, 3)
    A = ora.assemble().toarray()
    b0 = ora.mass_apply(uniform_field((2, m.K, ora.Np), seed=5))
    pt = uniform_field((2, m.K, ora.Np), seed=6)
    opts = P._binding.default_opts(precond=P.PREC_JACOBI, tol=1e-14, max_iter=20000)
    b = cuda(b0).requires_grad_(True)
    p = sipdg_solve(lib, b, opts=opts)
    loss = ((p - cuda(pt)) ** 2).sum()
    loss.backward()
    pd = np.stack([np.linalg.solve(A, b0[k].ravel()) for k in range(2)])
    gref = np.stack([2 * np.linalg.solve(A, pd[k] - pt[k].ravel()) for k in range(2)]).reshape(b0.shape)
    assert rel(p.detach().cpu().numpy(), pd.reshape(b0.shape)) <= 1e-10
    assert rel(b.grad.cpu().numpy(), gref) <= 1e-10


def test_c4_batched_adjoint_central_differences():
    """128x128 jittered grid (32768 triangles), N=6, 64 right-hand sides each a
    sum of 16 sine modes (wavenumbers 1..8, N(0,1) amplitudes, seed 1000+b),
    targets from seed 2000+b; loss = sum ||p - p*||^2; gradient by the adjoint
    p-multigrid PCG (FP64 outer, FP32 multigrid), checked by central
    differences along 8 random directions (seed 3000). The loss is quadratic in
    b, so the central difference is exact up to rounding and solver error for
    any step; the step is 1e-3 ||b||/||d|| and the solves run to 1e-13."""
    import torch
    P = pkg()
    from paper_1801_00246_gb300.autograd import sipdg_solve
    m, N = config_mesh("c4_adjoint_32768tri_N6")
    lib = P.Mesh.from_inputs(m, N)
    x, y = lib.nodes()
    xh, yh = x.cpu().numpy(), y.cpu().numpy()
    B = 64
    f = np.stack([fourier_eval(fourier_rhs_coeffs(1000 + k), xh, yh) for k in range(B)])
    pt = np.stack([fourier_eval(fourier_rhs_coeffs(2000 + k), xh, yh) for k in range(B)]) * 1e-2
    b0 = lib.rhs(cuda(f))
    opts = P._binding.default_opts(precond=P.PREC_PMG, degrees=[6, 3, 1], tol=1e-13, max_iter=400, mixed=1,
                                   coarse_amg=1)
    ptd = cuda(pt)
    b = b0.clone().requires_grad_(True)
    p = sipdg_solve(lib, b, opts=opts)
    loss = ((p - ptd) ** 2).sum()
    loss.backward()
    g = b.grad.detach()

    def L(bb):
        pp, _ = lib.solve(bb.contiguous(), opts=opts)
        return float(((pp - ptd) ** 2).sum())

    rng = np.random.default_rng(3000)
    errs = []
    for k in range(8):
        d = cuda(rng.standard_normal(b0.shape))
        h = 1e-3 * float(torch.linalg.norm(b0)) / float(torch.linalg.norm(d))
        fd = (L(b0 + h * d) - L(b0 - h * d)) / (2 * h)
        an = float((g * d).sum())
        errs.append(abs(fd - an) / abs(an))
    print("c4 adjoint FD relative errors:", ["%.1e" % e for e in errs])
    assert max(errs) <= 1e-6
