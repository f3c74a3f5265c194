"""Helpers shared by the GPU parity tests (build the library once, pair the
library mesh with the oracle on the same seeded input)."""
import functools

import numpy as np
import pytest


@functools.lru_cache(maxsize=None)
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    build.build()
    return P


def pair(mesh, N):
    from oracle.sipdg import Sipdg
    P = pkg()
    return P.Mesh.from_inputs(mesh, N), Sipdg(mesh.VX, mesh.VY, mesh.EToV, mesh.bc, N)


def cuda(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
