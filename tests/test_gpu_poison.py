"""Solves and applies with every library scratch allocation filled with NaN
bytes (DG_POISON_SCRATCH=1, read once per process, hence the subprocess):
any kernel that reads scratch it has not written shows up as a breakdown or a
non-finite result instead of depending on what the allocator hands back."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import paper_1801_00246_gb300 as P
from paper_1801_00246_gb300 import build
from dg_inputs import jittered_grid, uniform_field
from dg_inputs.mesh import rotate_local_vertices
from oracle.sipdg import Sipdg
build.build()
m = rotate_local_vertices(jittered_grid(12, 10, seed=3), 4)
for N, degs in ((4, [4, 2, 1]), (6, [6, 3, 1])):
    ora = Sipdg(m.VX, m.VY, m.EToV, m.bc, N)
    bb = ora.mass_apply(uniform_field((3, m.K, ora.Np), seed=8))
    for amg in (0, 1):
        for mixed in (1, 0):
            for graph in (0, 1):
                lib = P.Mesh.from_inputs(m, N)
                x, info = lib.solve(torch.from_numpy(bb).cuda(), precond=P.PREC_PMG, degrees=degs, tol=1e-10,
                                    max_iter=200, mixed=mixed, coarse_amg=amg, graph=graph)
                xs = x.cpu().numpy()
                for k in range(3):
                    r = bb[k] - ora.apply(xs[k])
                    assert np.linalg.norm(r) / np.linalg.norm(bb[k]) <= 1.5e-10, (N, amg, mixed, graph)
    for prec, dt in ((P.DG_F64, torch.float64), (P.DG_F32, torch.float32)):
        for kern in (P.KERNEL_TILE, P.KERNEL_TENSOR, P.KERNEL_GEMM, P.KERNEL_EPT, P.KERNEL_TC05, P.KERNEL_TC64):
            lib = P.Mesh.from_inputs(m, N)
            try:
                lib.set_kernel(N, prec, 1, kern)
            except P.DgError:
                continue
            u = uniform_field((2, m.K, ora.Np), seed=1)
            got = lib.apply(torch.from_numpy(u).to(dt).cuda(), lam=2.0).cpu().numpy()
            assert np.isfinite(got).all(), (N, prec, kern)
    lib = P.Mesh.from_inputs(m, N)
    x, info = lib.solve(torch.from_numpy(bb[0]).cuda(), precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000)
    assert info["relres"][0] <= 1e-10
print("poisoned scratch: all solves converged")
'''


def test_solves_with_poisoned_scratch():
    env = dict(os.environ, DG_POISON_SCRATCH="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCRIPT], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "all solves converged" in r.stdout
