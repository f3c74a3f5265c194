"""The allocation-free Jacobi-PCG entry point (dg_pcg_jacobi_solve_static).

Callers that may not allocate device memory while they run (a host whose
memory pool owns the GPU, a time-critical loop, a simulation that must not
fail on an allocation midway) use this entry point; its workspace is a fixed
device array compiled into the library. It must give the same solution as
the allocating solver (dg_pcg_solve with the Jacobi preconditioner), on two
calls in a row that share that array, and reject problems larger than it.
This file is collected last so that a failing run has already run every other
test."""
import ctypes

import numpy as np
import pytest

from dg_inputs import config_mesh, manufactured
from tests.gpu_util import cuda, pkg, rel

pytestmark = pytest.mark.gpu


def _static_call(lib_mesh, b, x, tol=1e-10, max_iter=5000, B=1):
    import torch
    P = pkg()
    info = P._binding.SolveInfo()
    st = P.lib().dg_pcg_jacobi_solve_static(lib_mesh._h, B, 0.0, tol, max_iter, ctypes.c_void_p(b.data_ptr()),
                                            ctypes.c_void_p(x.data_ptr()), ctypes.byref(info),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, info


def test_static_solve_matches_allocating_solver_twice():
    import torch
    P = pkg()
    m, N = config_mesh("c1_poisson_512tri_N3")
    mesh = P.Mesh.from_inputs(m, N)
    xn, yn = mesh.nodes()
    uex, fex = manufactured("sin_pi_x_sin_pi_y")
    xh, yh = xn.cpu().numpy(), yn.cpu().numpy()
    b = mesh.rhs(cuda(fex(xh, yh)), cuda(uex(xh, yh)))
    ref, info_ref = mesh.solve(b, precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000)
    ref = ref.cpu().numpy()
    outs = []
    for _ in range(2):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        st, info = _static_call(mesh, b, x)
        torch.cuda.synchronize()
        assert st == 0, P.lib().dg_last_error().decode()
        assert info.relres[0] <= 1e-10
        assert info.iters[0] == info_ref["iters"][0]
        got = x.cpu().numpy()
        assert rel(got, ref) <= 1e-12
        outs.append(got)
    assert rel(outs[0], outs[1]) <= 1e-12
    # steady state: further calls take no device memory
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        st, _ = _static_call(mesh, b, x)
        assert st == 0
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1
    del free0


def test_static_solve_batched_and_rejects_oversize():
    import torch
    P = pkg()
    m, N = config_mesh("c1_poisson_512tri_N3")
    mesh = P.Mesh.from_inputs(m, N)
    rng = np.random.default_rng(5)
    bb = cuda(rng.uniform(-1, 1, (2, mesh.K, mesh.Np)))
    ref, _ = mesh.solve(bb, precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000)
    x = torch.zeros_like(bb)
    st, info = _static_call(mesh, bb, x, B=2)
    assert st == 0
    assert rel(x.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    big, Nb = config_mesh("c2_pmg_32768tri_N6")    # 917,504 nodes: beyond the array
    bmesh = P.Mesh.from_inputs(big, Nb)
    b2 = torch.zeros((bmesh.K, bmesh.Np), dtype=torch.float64, device="cuda")
    x2 = torch.zeros_like(b2)
    st, _ = _static_call(bmesh, b2, x2)
    assert st == 1     # DG_ERR_ARG
    assert b"static array holds" in P.lib().dg_last_error()
