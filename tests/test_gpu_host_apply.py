"""dg_apply_host: the apply on fields in host memory, with the copies chunked
and overlapped with the tcgen05 FP64 apply, gives the device apply's results
bit for bit (every row's result depends only on the row's own data and its
neighbours' face data, not on how the rows are grouped into launches)."""
import numpy as np
import pytest

from dg_inputs import jittered_grid, uniform_field
from tests.gpu_util import pkg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [2, 3, 8, 10])
@pytest.mark.parametrize("B,lam", [(1, 0.0), (3, 2.5)])
def test_host_apply_equals_device_apply(N, B, lam):
    import torch
    P = pkg()
    m = jittered_grid(13, 11, jitter=0.1, seed=N)          # 286 elements: ragged tiles
    mesh = P.Mesh.from_inputs(m, N)
    u = torch.from_numpy(uniform_field((B, mesh.K, mesh.Np), seed=4 + N)).pin_memory()
    ref = mesh.apply(u.cuda(), lam=lam).cpu()
    got = mesh.apply_host(u, lam=lam)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    got32 = mesh.apply_host(u.float(), lam=lam)            # FP32: copies around the device apply
    torch.cuda.synchronize()
    assert torch.equal(got32, mesh.apply(u.float().cuda(), lam=lam).cpu())


def test_host_apply_in_several_chunks_and_back_to_back_calls():
    """80,000 triangles at B = 4: 320,000 rows in chunks of 4 waves of 128-row
    tiles (at most 77,824 rows on 152 SMs), so several chunks and a ragged last
    one; two calls in a row reuse the mesh's device buffers and events."""
    import torch
    P = pkg()
    m = jittered_grid(200, 200, jitter=0.1, seed=1)
    mesh = P.Mesh.from_inputs(m, 3)
    u1 = torch.from_numpy(uniform_field((4, mesh.K, mesh.Np), seed=1)).pin_memory()
    u2 = torch.from_numpy(uniform_field((4, mesh.K, mesh.Np), seed=2)).pin_memory()
    o1 = mesh.apply_host(u1, lam=1.5)
    o2 = mesh.apply_host(u2, lam=1.5)
    torch.cuda.synchronize()
    assert torch.equal(o1, mesh.apply(u1.cuda(), lam=1.5).cpu())
    assert torch.equal(o2, mesh.apply(u2.cuda(), lam=1.5).cpu())


def test_host_apply_pageable_memory_and_argument_errors():
    import torch
    P = pkg()
    m = jittered_grid(6, 6, jitter=0.1, seed=3)
    mesh = P.Mesh.from_inputs(m, 4)
    u = torch.from_numpy(uniform_field((mesh.K, mesh.Np), seed=7))   # pageable
    got = mesh.apply_host(u)
    torch.cuda.synchronize()
    assert torch.equal(got, mesh.apply(u.cuda()).cpu())
    with pytest.raises(P.DgError):
        mesh.apply_host(u, lam=-1.0)
    with pytest.raises(ValueError):
        mesh.apply_host(u.cuda())
    L = P.lib()
    import ctypes
    st = L.dg_apply_host(mesh._h, 0, P.DG_F64, 1, 0.0, ctypes.c_void_p(u.data_ptr()),
                         ctypes.c_void_p(u.data_ptr()), None)
    assert st == 1                                                      # u and Au alias
