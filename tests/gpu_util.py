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


def kernels_for(P, N, f64):
    """The apply kernels available at degree N in FP64 (f64) or FP32: the tile
    kernel at every degree, the mma.sync tensor kernels to N = 9, the tcgen05
    FP64 kernel at every degree, the FP32 register GEMMs to N = 9, the tcgen05
    FP32 kernel to N = 8 (tensor memory) and one element per thread to N = 3."""
    ks = [P.KERNEL_TILE]
    if N <= 9:
        ks += [P.KERNEL_TENSOR, P.KERNEL_TENSOR_PIPE]
    if f64:
        ks.append(P.KERNEL_TC64)
    else:
        ks += ([P.KERNEL_GEMM] if N <= 9 else []) + ([P.KERNEL_TC05] if N <= 8 else [])
    if N <= 3:
        ks.append(P.KERNEL_EPT)
    return ks


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


def abs_bound(ora, u, lam=0.0):
    """(|A| |u|)_i per node: the scale against which a sliced or piecewise
    product's rounding is bounded entry by entry (small meshes: assembles A)."""
    A = ora.assemble(lam)
    A.data = np.abs(A.data)
    U = np.asarray(u, dtype=np.float64)
    if U.ndim == 3:
        return np.stack([(A @ np.abs(Ub).ravel()).reshape(Ub.shape) for Ub in U])
    return (A @ np.abs(U).ravel()).reshape(U.shape)


def max_entry_err(got, ref, bound):
    """max_i |got_i - ref_i| / bound_i (entries with a zero bound must match exactly)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.abs(got - ref)
    zero = bound == 0
    if np.any(d[zero] != 0):
        return float("inf")
    return float(np.max(d[~zero] / bound[~zero])) if np.any(~zero) else 0.0
