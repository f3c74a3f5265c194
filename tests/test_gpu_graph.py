"""The whole-solve CUDA graph (device-side WHILE/IF loops) against the
host-driven loop: same kernels, same order, so the iterates must agree bit for
bit, and both must pass the oracle's own residual check."""
import numpy as np
import pytest

from dg_inputs import jittered_grid, manufactured, uniform_field
from dg_inputs.mesh import rotate_local_vertices
from tests.gpu_util import cuda, pair, pkg

pytestmark = pytest.mark.gpu


def _oracle_relres(ora, x, b, lam=0.0):
    r = b - ora.apply(x, lam=lam)
    return np.linalg.norm(r) / np.linalg.norm(b)


def _both(lib, b, **kw):
    """Solve with the graph (twice: capture, then replay) and eagerly."""
    xg, ig = lib.solve(b, graph=1, **kw)
    xr, ir = lib.solve(b, graph=1, **kw)
    xe, ie = lib.solve(b, graph=0, **kw)
    return (xg.cpu().numpy(), ig), (xr.cpu().numpy(), ir), (xe.cpu().numpy(), ie)


def _assert_same(a, b):
    (xa, ia), (xb, ib) = a, b
    assert np.array_equal(xa, xb)
    assert ia["iters"] == ib["iters"]
    assert ia["relres"] == ib["relres"]
    assert ia["status"] == ib["status"]


@pytest.mark.parametrize("B", [1, 3])
def test_graph_jacobi_bitwise_equals_eager(B):
    P = pkg()
    m = rotate_local_vertices(jittered_grid(10, 9, seed=4), 3)
    lib, ora = pair(m, 4)
    bb = ora.mass_apply(uniform_field((B, m.K, ora.Np), seed=11))
    g, r, e = _both(lib, cuda(bb), precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000)
    _assert_same(g, e)
    _assert_same(r, e)
    assert g[1]["total_iters"] == max(g[1]["iters"])
    for k in range(B):
        assert _oracle_relres(ora, g[0][k], bb[k]) <= 1.5e-10


@pytest.mark.parametrize("mixed,amg", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_graph_pmg_bitwise_equals_eager(mixed, amg):
    """p-multigrid (6 -> 3 -> 1) with the coarse CG plain or AMG-preconditioned:
    two nested device-side loops inside the captured graph."""
    P = pkg()
    m = rotate_local_vertices(jittered_grid(12, 12, seed=0), 1)
    lib, ora = pair(m, 6)
    uex, fex = manufactured("sin_2pi_x_cos_3pi_y")
    f, g = fex(ora.x, ora.y), uex(ora.x, ora.y)
    b = lib.rhs(cuda(f), cuda(g))
    kw = dict(precond=P.PREC_PMG, degrees=[6, 3, 1], tol=1e-10, max_iter=200, mixed=mixed, coarse_amg=amg)
    gr, rp, ea = _both(lib, b, **kw)
    _assert_same(gr, ea)
    _assert_same(rp, ea)
    assert gr[1]["status"] == "DG_OK"
    assert gr[1]["coarse_iters"] > 0
    assert gr[1]["total_iters"] == gr[1]["iters"][0]
    assert _oracle_relres(ora, gr[0], ora.rhs(f, g)) <= 1.5e-10
    if amg:  # both check every coarse pass: the same number of passes
        assert gr[1]["coarse_iters"] == ea[1]["coarse_iters"]


def test_graph_helmholtz_batched_invmass_and_new_buffers():
    """A replay with new b / x tensors (the graph stages them) and a lambda
    change (a new capture) both give the eager answer."""
    P = pkg()
    m = rotate_local_vertices(jittered_grid(8, 8, seed=1), 2)
    lib, ora = pair(m, 5)
    for lam, seed in ((6000.0, 4), (6000.0, 5), (250.0, 6)):
        bb = ora.mass_apply(uniform_field((2, m.K, ora.Np), seed=seed))
        xg, ig = lib.solve(cuda(bb), lam=lam, precond=P.PREC_INVMASS, tol=1e-10, max_iter=500, graph=1)
        xe, ie = lib.solve(cuda(bb), lam=lam, precond=P.PREC_INVMASS, tol=1e-10, max_iter=500, graph=0)
        assert np.array_equal(xg.cpu().numpy(), xe.cpu().numpy())
        assert ig["iters"] == ie["iters"]
        for k in range(2):
            assert _oracle_relres(ora, xg[k].cpu().numpy(), bb[k], lam=lam) <= 1.5e-10


def test_graph_nonzero_initial_guess_and_iteration_cap():
    P = pkg()
    m = rotate_local_vertices(jittered_grid(9, 7, seed=8), 4)
    lib, ora = pair(m, 3)
    bb = ora.mass_apply(uniform_field((m.K, ora.Np), seed=2))
    x0 = uniform_field((m.K, ora.Np), seed=3)
    xg, ig = lib.solve(cuda(bb), x=cuda(x0), precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000, graph=1)
    xe, ie = lib.solve(cuda(bb), x=cuda(x0), precond=P.PREC_JACOBI, tol=1e-10, max_iter=5000, graph=0)
    assert np.array_equal(xg.cpu().numpy(), xe.cpu().numpy())
    assert _oracle_relres(ora, xg.cpu().numpy(), bb) <= 1.5e-10
    # a cap of 7 passes: not converged, the 7th iterate returned
    xg, ig = lib.solve(cuda(bb), precond=P.PREC_JACOBI, tol=1e-14, max_iter=7, graph=1, check=False)
    xe, ie = lib.solve(cuda(bb), precond=P.PREC_JACOBI, tol=1e-14, max_iter=7, graph=0, check=False)
    assert ig["status"] == "DG_ERR_NOT_CONVERGED" and ie["status"] == "DG_ERR_NOT_CONVERGED"
    assert ig["iters"] == [7] and ig["total_iters"] == 7
    # the eager loop runs its 7 passes too (cap reached between checks)
    assert np.array_equal(xg.cpu().numpy(), xe.cpu().numpy())
    # a cap of 0: no pass, x untouched
    xg, ig = lib.solve(cuda(bb), x=cuda(x0), precond=P.PREC_JACOBI, tol=1e-10, max_iter=0, graph=1, check=False)
    assert ig["total_iters"] == 0 and np.array_equal(xg.cpu().numpy(), x0)


def test_graph_recaptured_after_scratch_growth():
    """A larger-batch apply reallocates the mesh's apply scratch; the next
    solve must not replay a graph that addresses the freed buffer."""
    P = pkg()
    m = rotate_local_vertices(jittered_grid(10, 10, seed=6), 2)
    lib, ora = pair(m, 5)
    bb = ora.mass_apply(uniform_field((m.K, ora.Np), seed=9))
    kw = dict(precond=P.PREC_PMG, degrees=[5, 2, 1], tol=1e-10, max_iter=200, mixed=1)
    x1, i1 = lib.solve(cuda(bb), graph=1, **kw)
    big = cuda(uniform_field((8, m.K, ora.Np), seed=1))
    lib.apply(big)            # FP64 scratch for 8 right-hand sides
    lib.apply(big.float())    # FP32 face scratch for 8
    x2, i2 = lib.solve(cuda(bb), graph=1, **kw)
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    assert i1["iters"] == i2["iters"]


def test_graph_counts_the_kernels_it_runs():
    """With AMG on the coarse degree both loops check every pass, so the graph
    runs the eager kernels plus its loop-control kernels (head, tail, count)."""
    P = pkg()
    L = P.lib()
    m = rotate_local_vertices(jittered_grid(12, 12, seed=0), 1)
    lib, ora = pair(m, 6)
    b = cuda(ora.mass_apply(uniform_field((m.K, ora.Np), seed=1)))
    kw = dict(precond=P.PREC_PMG, degrees=[6, 3, 1], tol=1e-10, max_iter=200, mixed=1, coarse_amg=1)
    lib.solve(b, graph=1, **kw)  # capture
    lib.solve(b, graph=0, **kw)
    n0 = L.dg_launch_count()
    _, ie = lib.solve(b, graph=0, **kw)
    n_eager = L.dg_launch_count() - n0
    n0 = L.dg_launch_count()
    _, ig = lib.solve(b, graph=1, **kw)
    n_graph = L.dg_launch_count() - n0
    it, cit = ig["total_iters"], ig["coarse_iters"]
    # per outer pass: tail + count; per coarse solve: head; per coarse pass: tail (+ count when it continues)
    assert n_eager < n_graph <= n_eager + 2 * it + 2 * cit + (it + 1) + 4
