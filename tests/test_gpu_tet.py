"""GPU parity of the tetrahedral SIPDG path (apply, right-hand side, nodes,
Jacobi-PCG) against the quadrature oracle on the same seeded meshes.

Tolerances: relative 2-norm error at most 1e-12 for the FP64 apply and 1e-5
for FP32 (FP32 storage and accumulation), as for triangles, except where the
reference operators themselves are less accurate: both sides build the nodal
basis by inverting the monomial Vandermonde matrix of the equispaced nodes,
whose 2-norm condition number is 4.8e3 at N = 4 and 5.7e4 at N = 5, so each
side's Dr, Ds, Dt and M may carry relative errors up to cond(V) eps; the FP64
bound is max(1e-12, cond(V) eps) (6.4e-12 at N = 5). The solve is
compared with a direct sparse solve of the oracle's assembled matrix, within
the PCG tolerance times a condition estimate."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from dg_inputs import uniform_field
from dg_inputs.tetmesh import jittered_tet_grid
from tests.gpu_util import cuda, pkg, rel

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
MIXED = (1, 2, 2, 1, 1, 2)   # Dirichlet on x0, y1, z0; Neumann on x1, y0, z1


def tol64(N):
    from oracle.tet import monomials, tet_nodes
    r, s, t = tet_nodes(N)
    return max(TOL64, np.linalg.cond(monomials(N, r, s, t)[0]) * np.finfo(np.float64).eps)


def _pair(mesh, N):
    from oracle.tet import TetSipdg
    P = pkg()
    return P.TetMesh.from_inputs(mesh, N), TetSipdg(mesh.VX, mesh.VY, mesh.VZ, mesh.EToV, mesh.bc, N)


@pytest.mark.parametrize("N", range(1, 6))
@pytest.mark.parametrize("lam", [0.0, 2.5])
def test_tet_apply_parity_mixed_boundaries(N, lam):
    import torch
    m = jittered_tet_grid(3, jitter=0.12, seed=N, bc_sides=MIXED)     # 162 elements: a ragged last block
    lib, ora = _pair(m, N)
    u = uniform_field((2, m.K, ora.Np), seed=20 + N)
    ref = ora.apply(u, lam=lam)
    got64 = lib.apply(cuda(u), lam=lam).cpu().numpy()             # products on the tensor cores
    assert rel(got64, ref) <= tol64(N)
    gotp = lib.apply(cuda(u), lam=lam, fp64_pipe=True).cpu().numpy()
    assert rel(gotp, ref) <= tol64(N)
    got32 = lib.apply(cuda(u, torch.float32), lam=lam).cpu().numpy()
    assert rel(got32, ref) <= TOL32
    # right-hand sides are independent
    one = lib.apply(cuda(u[1]), lam=lam).cpu().numpy()
    assert rel(one, ref[1]) <= tol64(N)


@pytest.mark.parametrize("N", [2, 4])
def test_tet_apply_all_neumann_and_all_dirichlet(N):
    for sides in ((2,) * 6, (1,) * 6):
        m = jittered_tet_grid(2, jitter=0.1, seed=7, bc_sides=sides)
        lib, ora = _pair(m, N)
        u = uniform_field((m.K, ora.Np), seed=3)
        assert rel(lib.apply(cuda(u)).cpu().numpy(), ora.apply(u)) <= tol64(N)
    # all-Neumann: constants are in the kernel
    m = jittered_tet_grid(2, jitter=0.1, seed=7, bc_sides=(2,) * 6)
    lib, ora = _pair(m, N)
    assert np.abs(lib.apply(cuda(np.ones((m.K, ora.Np)))).cpu().numpy()).max() < 1e-11


def test_tet_apply_parity_past_one_grid_stride():
    """20,250 elements (15 cubes a side) at B = 4: 81,000 element applies, more
    than one resident wave of blocks covers at N = 2 (batches of 50 elements;
    at most 8 blocks per SM of 152), so both kernels' block loops run more
    than once, and the last batch is ragged."""
    m = jittered_tet_grid(15, jitter=0.1, seed=11, bc_sides=MIXED)
    lib, ora = _pair(m, 2)
    u = uniform_field((4, m.K, ora.Np), seed=5)
    ref = ora.apply(u, lam=0.7)
    assert rel(lib.apply(cuda(u), lam=0.7).cpu().numpy(), ref) <= TOL64
    assert rel(lib.apply(cuda(u), lam=0.7, fp64_pipe=True).cpu().numpy(), ref) <= TOL64


@pytest.mark.parametrize("N", [1, 3, 5])
def test_tet_nodes_and_rhs_parity(N):
    m = jittered_tet_grid(3, jitter=0.1, seed=2, bc_sides=MIXED)
    lib, ora = _pair(m, N)
    x, y, z = (t.cpu().numpy() for t in lib.nodes())
    assert max(np.abs(x - ora.x).max(), np.abs(y - ora.y).max(), np.abs(z - ora.z).max()) < 1e-14
    f = np.cos(ora.x + 2 * ora.y) * ora.z
    g = np.sin(ora.x) + ora.y * ora.z
    F = np.stack([f, 2 * f + 1])
    G = np.stack([g, -g])
    ref = np.stack([ora.rhs(F[k], G[k]) for k in range(2)])
    got = lib.rhs(cuda(F), cuda(G)).cpu().numpy()
    assert rel(got, ref) <= tol64(N)


@pytest.mark.parametrize("N,lam,sides", [(2, 0.0, (1,) * 6), (3, 0.0, MIXED), (2, 4.0, (2,) * 6)])
def test_tet_jacobi_pcg_matches_direct_solve(N, lam, sides):
    m = jittered_tet_grid(3, jitter=0.1, seed=4, bc_sides=sides)
    lib, ora = _pair(m, N)
    A = ora.assemble(lam).tocsc()
    bs = np.stack([ora.mass_apply(np.cos(np.pi * ora.x) * np.sin(ora.y + ora.z)),
                   ora.mass_apply(uniform_field((m.K, ora.Np), seed=9))])
    x, info = lib.solve(cuda(bs), lam=lam, tol=1e-11)
    assert info["status"] == "DG_OK"
    assert all(0 < it < 2000 for it in info["iters"]) and max(info["relres"]) <= 1e-11
    x = x.cpu().numpy()
    for k in range(2):
        ref = spla.spsolve(A, bs[k].ravel()).reshape(bs[k].shape)
        # ||x - x*|| / ||x*|| <= cond(A) relres; the oracle's 2-norm cond(A) for these three cases is 5e2, 2.8e3, 2.7e3
        assert rel(x[k], ref) <= 1e-6
        # and the residual measured by the oracle operator
        assert rel(ora.apply(x[k], lam=lam), bs[k]) <= 2e-11


def test_tet_solve_converges_to_a_smooth_solution():
    """-lap u = 3 pi^2 u for u = sin(pi x) sin(pi y) sin(pi z), Dirichlet data u:
    the device right-hand side and solve reach the discretisation error, whose
    nodal maximum falls by more than 4x from 2 to 4 cubes a side at N = 2 (the
    oracle's direct solve gives 0.113 and 0.0212, log2 ratio 2.42)."""
    P = pkg()
    errs = []
    for n in (2, 4):
        m = jittered_tet_grid(n, jitter=0.0)
        lib = P.TetMesh.from_inputs(m, 2)
        x, y, z = lib.nodes()
        import torch
        u = torch.sin(np.pi * x) * torch.sin(np.pi * y) * torch.sin(np.pi * z)
        b = lib.rhs(3 * np.pi ** 2 * u, u)
        sol, info = lib.solve(b, tol=1e-12)
        errs.append(float((sol - u).abs().max()))
    assert np.log2(errs[0] / errs[1]) > 2.0, errs


def test_tet_argument_errors():
    import torch
    P = pkg()
    m = jittered_tet_grid(2, jitter=0.1, seed=1)
    lib = P.TetMesh.from_inputs(m, 2)
    u = torch.zeros((m.K, lib.Np), dtype=torch.float64, device="cuda")
    with pytest.raises(P.DgError):
        lib.apply(u, lam=-1.0)
    with pytest.raises(P.DgError):
        lib.solve(u, tol=0.0)
    with pytest.raises(P.DgError):
        P.TetMesh.from_inputs(m, 6)


@pytest.mark.parametrize("N", range(1, 6))
def test_tet_apply_parity_renumbered_local_vertices(N):
    """Each element's vertices renumbered by a seeded even permutation: every
    pairing of local faces and every rotation of a shared face's nodes occurs,
    so the neighbour face-node matching is exercised in all its cases."""
    import torch
    from dg_inputs.tetmesh import permute_local_vertices
    m = permute_local_vertices(jittered_tet_grid(3, jitter=0.1, seed=9, bc_sides=MIXED), seed=N)
    lib, ora = _pair(m, N)
    u = uniform_field((2, m.K, ora.Np), seed=40 + N)
    ref = ora.apply(u, lam=1.25)
    assert rel(lib.apply(cuda(u), lam=1.25).cpu().numpy(), ref) <= tol64(N)
    assert rel(lib.apply(cuda(u), lam=1.25, fp64_pipe=True).cpu().numpy(), ref) <= tol64(N)
    assert rel(lib.apply(cuda(u, torch.float32), lam=1.25).cpu().numpy(), ref) <= TOL32


@pytest.mark.parametrize("N", [2, 4])
def test_tet_apply_entrywise_against_abs_bound(N):
    """Node by node: |A u - (A u)_oracle|_i <= tol (|A| |u|)_i, the scale that
    bounds the rounding of each node's sum whatever the cancellation."""
    import torch
    m = jittered_tet_grid(2, jitter=0.1, seed=6, bc_sides=MIXED)
    lib, ora = _pair(m, N)
    u = uniform_field((m.K, ora.Np), seed=8)
    A = ora.assemble(0.0)
    bound = (abs(A) @ np.abs(u).ravel()).reshape(u.shape)
    ref = ora.apply(u)
    got64 = lib.apply(cuda(u)).cpu().numpy()
    gotp = lib.apply(cuda(u), fp64_pipe=True).cpu().numpy()
    got32 = lib.apply(cuda(u, torch.float32)).cpu().numpy()
    assert np.all(np.abs(got64 - ref) <= tol64(N) * bound)
    assert np.all(np.abs(gotp - ref) <= tol64(N) * bound)
    assert np.all(np.abs(got32 - ref) <= TOL32 * bound)
