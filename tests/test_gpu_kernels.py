"""Every apply kernel (tile, FP32 GEMM, tensor-core FP64/FP32, element per thread)
against the FP64 oracle, chosen explicitly through the mesh's kernel table,
and the autotuner that fills that table. Tolerances as for the default
kernels: 1e-12 relative (FP64), 1e-5 (FP32)."""
import numpy as np
import pytest

from dg_inputs import jittered_grid, uniform_field
from dg_inputs.mesh import rotate_local_vertices, with_all_neumann
from tests.gpu_util import cuda, kernels_for, pair, pkg, rel

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


def _kernels(P, N, f64):
    return kernels_for(P, N, f64)


def _mixed_bc(n, seed):
    return jittered_grid(n, n, jitter=0.1, seed=seed, bc_sides=(1, 2, 2, 1))


@pytest.mark.parametrize("N", range(1, 11))
def test_every_kernel_matches_oracle(N):
    """Rotated local numbering (all face orientations), Dirichlet + Neumann
    sides, a ragged element count, Poisson and Helmholtz, batch of 2."""
    import torch
    P = pkg()
    for m in (rotate_local_vertices(_mixed_bc(7, 3), seed=N), with_all_neumann(jittered_grid(4, 5, seed=1))):
        lib, ora = pair(m, N)
        u = uniform_field((2, m.K, ora.Np), seed=20 + N)
        for lam in (0.0, 3.5):
            ref = ora.apply(u, lam=lam)
            for f64, prec in ((True, P.DG_F64), (False, P.DG_F32)):
                for k in _kernels(P, N, f64):
                    lib.set_kernel(N, prec, lam != 0.0, k)
                    assert lib.kernel(N, prec, lam != 0.0) == k
                    x = cuda(u) if f64 else cuda(u, torch.float32)
                    got = lib.apply(x, lam=lam).cpu().numpy()
                    assert P.lib().dg_tensor_timeouts() == 0  # no pipelined hand-off gave up
                    assert np.isfinite(got).all()
                    assert rel(got, ref) <= (TOL64 if f64 else TOL32), (N, f64, k, lam)
                lib.set_kernel(N, prec, lam != 0.0, P.KERNEL_AUTO)


def test_kernel_table_rejects_unavailable_kernels():
    P = pkg()
    lib, _ = pair(jittered_grid(2, 2, seed=0), 5)
    with pytest.raises(P.DgError):
        lib.set_kernel(5, P.DG_F64, 0, P.KERNEL_GEMM)      # FP32-only
    with pytest.raises(P.DgError):
        lib.set_kernel(5, P.DG_F32, 0, P.KERNEL_EPT)       # degrees 1-3
    with pytest.raises(P.DgError):
        lib.set_kernel(9, P.DG_F32, 0, P.KERNEL_TC05)      # tensor memory: degrees 1-8
    with pytest.raises(P.DgError):
        lib.set_kernel(10, P.DG_F32, 0, P.KERNEL_GEMM)     # shared memory: degrees 1-9
    with pytest.raises(P.DgError):
        lib.set_kernel(10, P.DG_F64, 0, P.KERNEL_TENSOR)   # the fill's lane map: degrees 1-9
    with pytest.raises(P.DgError):
        lib.set_kernel(11, P.DG_F32, 0, P.KERNEL_TILE)
    assert lib.kernel(11, P.DG_F64) == -1
    assert lib.kernel(10, P.DG_F64) == P.KERNEL_TC64 and lib.kernel(10, P.DG_F32) == P.KERNEL_TILE
    assert lib.kernel(9, P.DG_F32) == P.KERNEL_TENSOR
    for N in range(1, 11):
        for f64, prec in ((True, P.DG_F64), (False, P.DG_F32)):
            assert set(lib.kernels_available(N, prec)) == set(kernels_for(P, N, f64)), (N, f64)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_element_per_thread_full_size_sampled(N):
    """The 524,288-triangle workload with the element-per-thread kernel."""
    import torch
    from dg_inputs import config_mesh
    P = pkg()
    m, _ = config_mesh("c5_sweep_524288tri_N8")
    lib, ora = pair(m, N)
    u = uniform_field((m.K, ora.Np), seed=1)
    rng = np.random.default_rng(0)
    elems = np.unique(np.concatenate([rng.integers(0, m.K, 200), [0, 1, 1023, m.K - 1]]))
    ref = ora.apply(u, lam=1.0, elems=elems)
    for f64, prec, dt, tol in ((True, P.DG_F64, torch.float64, TOL64), (False, P.DG_F32, torch.float32, TOL32)):
        lib.set_kernel(N, prec, 1, P.KERNEL_EPT)
        got = lib.apply(cuda(u, dt), lam=1.0).cpu().numpy()
        assert np.isfinite(got).all()
        assert rel(got[elems], ref) <= tol


def test_autotune_fills_table_and_solves_stay_correct():
    """The autotuner times the candidates, keeps a valid winner per entry, and
    a (graph-captured) solve after it still meets the tolerance."""
    import torch
    P = pkg()
    m = rotate_local_vertices(jittered_grid(16, 16, seed=0), 1)
    lib, ora = pair(m, 4)
    lib.solve(cuda(ora.mass_apply(uniform_field((m.K, ora.Np), seed=4))), precond=P.PREC_PMG, degrees=[4, 2, 1],
              mixed=1, tol=1e-10)  # a graph captured with the built-in kernels
    times = lib.autotune(B=2, lam=1.0, degrees=(1, 4))
    for d in range(1, 5):
        for name, prec in (("f64", P.DG_F64), ("f32", P.DG_F32)):
            for h in (0, 1):
                row = times[(d, name, h)]
                assert set(row) == set(_kernels(P, d, name == "f64"))
                assert all(v > 0 for v in row.values())
                k = lib.kernel(d, prec, h)
                assert row[k] == min(row.values())
    u = uniform_field((m.K, ora.Np), seed=2)
    assert rel(lib.apply(cuda(u)).cpu().numpy(), ora.apply(u)) <= TOL64
    assert rel(lib.apply(cuda(u, torch.float32), lam=1.0).cpu().numpy(), ora.apply(u, lam=1.0)) <= TOL32
    b = ora.mass_apply(uniform_field((m.K, ora.Np), seed=4))
    x, info = lib.solve(cuda(b), precond=P.PREC_PMG, degrees=[4, 2, 1], mixed=1, tol=1e-10)
    r = b - ora.apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10
