"""Failure detection in the solver, caused on the host: a non-finite
right-hand side is reported as a Krylov breakdown (non-finite p^T A p) of that
right-hand side only, in the graph-captured and in the host-driven solve; the
other right-hand sides of the batch still converge and the mesh stays usable.
Nothing here faults or hangs the GPU: the NaN only flows through arithmetic
and every loop is bounded by its iteration cap."""
import numpy as np
import pytest

from dg_inputs import config_mesh, uniform_field
from tests.gpu_util import cuda, pair, pkg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graph", [1, 0])
def test_nan_right_hand_side_is_a_breakdown_of_that_entry_only(graph):
    P = pkg()
    m, N = config_mesh("c1_poisson_512tri_N3")
    lib, ora = pair(m, N)
    b = np.stack([ora.mass_apply(uniform_field((m.K, ora.Np), seed=s)) for s in (3, 4)])
    b[1, 5, 2] = np.nan
    x, info = lib.solve(cuda(b), precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000, graph=graph, check=False)
    assert info["status"] == "DG_ERR_BREAKDOWN"
    assert info["relres"][0] <= 1e-10
    r = b[0] - ora.apply(x[0].cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1.5e-10
    with pytest.raises(P.DgError, match="BREAKDOWN"):
        lib.solve(cuda(b[1]), precond=P.PREC_JACOBI, tol=1e-10, max_iter=100, graph=graph)
    x, info = lib.solve(cuda(b[0]), precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000, graph=graph)
    assert info["status"] == "DG_OK" and info["relres"][0] <= 1e-10


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A device-side wait on an mbarrier phase that nothing completes (the wait
    routine of every tensor-core kernel) gives up after its time limit: the call
    reports DG_ERR_TIMEOUT, the timeout is counted once in dg_tensor_timeouts,
    and the next apply on the same device is correct."""
    import time
    import torch
    P = pkg()
    L = P.lib()
    assert L.dg_tensor_timeouts() >= 0   # clear
    t0 = time.perf_counter()
    st = L.dg_wait_selftest(0.2, None)
    dt = time.perf_counter() - t0
    assert st == 6, L.dg_last_error()    # DG_ERR_TIMEOUT
    assert 0.15 < dt < 10.0
    assert L.dg_tensor_timeouts() == 1
    assert L.dg_tensor_timeouts() == 0   # reading clears
    m, N = config_mesh("c1_poisson_512tri_N3")
    lib, ora = pair(m, N)
    u = uniform_field((m.K, ora.Np), seed=9)
    got = lib.apply(cuda(u)).cpu().numpy()
    ref = ora.apply(u)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12
    got32 = lib.apply(cuda(u, torch.float32)).cpu().numpy()
    assert np.linalg.norm(got32 - ref) / np.linalg.norm(ref) <= 1e-5
