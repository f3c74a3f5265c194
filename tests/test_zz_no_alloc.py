"""The allocation-free Jacobi-PCG entry point (dg_pcg_jacobi_solve_static).

Callers that may not allocate device memory while they run (a host whose
memory pool owns the GPU, a time-critical loop, a simulation that must not
fail on an allocation midway) use this entry point; its workspace is a fixed
device array compiled into the library. It must give the same solution as
the allocating solver (dg_pcg_solve with the Jacobi preconditioner), on two
calls in a row that share that array, and reject problems larger than it.
Its very first call, on a fresh mesh in a fresh process at a batch size and
lambda no earlier call used, must leave the device's free memory unchanged.
This file is collected last so that a failing run has already run every other
test."""
import ctypes
import json
import os
import subprocess
import sys

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


# Runs in a fresh process with eager module loading, so that loading a kernel
# on its first launch cannot show up as a change of free device memory; the
# device buffers come from cudaMalloc directly (no torch), and the static call
# is the first solve of the process: a new mesh, degree 4, B = 2, lambda > 0.
_FRESH = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_1801_00246_gb300 as P
from dg_inputs import jittered_grid
L = P.lib()
rt = ctypes.CDLL("libcudart.so.13")
vp, sz = ctypes.c_void_p, ctypes.c_size_t
def ck(e, what):
    if e != 0:
        raise SystemExit(what + ": CUDA error " + str(e))
ck(rt.cudaSetDevice(0), "cudaSetDevice")
N, B, lam = 4, 2, 1.5
m = jittered_grid(12, 12, jitter=0.1, seed=3)
mesh = P.Mesh(N, m.VX, m.VY, m.EToV, m.bc)
n = B * mesh.K * mesh.Np
bh = np.random.default_rng(7).uniform(-1.0, 1.0, n)
def dalloc():
    p = vp()
    ck(rt.cudaMalloc(ctypes.byref(p), sz(8 * n)), "cudaMalloc")
    ck(rt.cudaMemset(p, 0, sz(8 * n)), "cudaMemset")
    return p
b, x, xr = dalloc(), dalloc(), dalloc()
ck(rt.cudaMemcpy(b, bh.ctypes.data_as(vp), sz(8 * n), 1), "cudaMemcpy")
ck(rt.cudaDeviceSynchronize(), "sync")
free0, free1, total = sz(), sz(), sz()
ck(rt.cudaMemGetInfo(ctypes.byref(free0), ctypes.byref(total)), "cudaMemGetInfo")
info = P._binding.SolveInfo()
st = L.dg_pcg_jacobi_solve_static(mesh._h, B, lam, 1e-10, 5000, b, x, ctypes.byref(info), None)
ck(rt.cudaDeviceSynchronize(), "sync")
ck(rt.cudaMemGetInfo(ctypes.byref(free1), ctypes.byref(total)), "cudaMemGetInfo")
opts = P._binding.default_opts(precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000)
info_r = P._binding.SolveInfo()
st_r = L.dg_pcg_solve(mesh._h, ctypes.byref(opts), B, lam, b, xr, ctypes.byref(info_r), None)
ck(rt.cudaDeviceSynchronize(), "sync")
xh, xrh = np.empty(n), np.empty(n)
ck(rt.cudaMemcpy(xh.ctypes.data_as(vp), x, sz(8 * n), 2), "cudaMemcpy")
ck(rt.cudaMemcpy(xrh.ctypes.data_as(vp), xr, sz(8 * n), 2), "cudaMemcpy")
print(json.dumps(dict(status=st, status_ref=st_r, free0=free0.value, free1=free1.value,
                      relres=[info.relres[0], info.relres[1]],
                      rel=float(np.linalg.norm(xh - xrh) / np.linalg.norm(xrh)))))
"""


def test_first_static_call_on_fresh_mesh_allocates_nothing():
    pkg()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["status"] == 0 and out["status_ref"] == 0, out
    assert out["free1"] == out["free0"], out
    assert max(out["relres"]) <= 1e-10, out
    assert out["rel"] <= 1e-12, out
