"""Pins of the oracle's SIPDG operator (Eq. ellipticOp1 / Eq. INS_SD_5)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from dg_inputs import jittered_grid, manufactured
from dg_inputs.mesh import rotate_local_vertices, with_all_neumann
from oracle.sipdg import Sipdg


def _mesh(n, seed=0, rotate=None):
    m = jittered_grid(n, n, jitter=0.1, seed=seed)
    return rotate_local_vertices(m, rotate) if rotate is not None else m


def _sip(m, N):
    return Sipdg(m.VX, m.VY, m.EToV, m.bc, N)


@pytest.mark.parametrize("n,N", [(1, 1), (1, 8), (2, 2), (2, 5), (4, 3), (4, 8), (2, 10)])
def test_symmetric_positive_definite(n, N):
    S = _sip(_mesh(n, rotate=3), N)
    A = S.assemble().toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max() * 10
    np.linalg.cholesky(0.5 * (A + A.T))
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


@pytest.mark.parametrize("N", [1, 3, 6])
def test_all_neumann_kills_constants(N):
    S = _sip(with_all_neumann(_mesh(3, rotate=1)), N)
    A = S.assemble()
    one = np.ones(S.K * S.Np)
    assert np.abs(A @ one).max() < 1e-11 * abs(A).max()


@pytest.mark.parametrize("N", range(1, 11))
@pytest.mark.parametrize("lam", [0.0, 3.5])
def test_polynomial_exactness_with_dirichlet_data(N, lam):
    """For a global polynomial p of degree <= N with g = p on the boundary, all
    jumps vanish and A p + L(p) = M (-lap p + lam p), whatever tau is."""
    S = _sip(_mesh(3, rotate=N), N)
    a = N // 2
    b = N - a
    x, y = S.x, S.y
    p = 0.3 + x ** a * y ** b + 0.5 * x ** (N - 1 if N > 1 else 0) * y
    lap = np.zeros_like(x)
    if a >= 2:
        lap += a * (a - 1) * x ** (a - 2) * y ** b
    if b >= 2:
        lap += b * (b - 1) * x ** a * y ** (b - 2)
    if N - 1 >= 2:
        lap += 0.5 * (N - 1) * (N - 2) * x ** (N - 3) * y
    lhs = S.apply(p, lam=lam) + S.dirichlet_lift(p)
    rhs = S.mass_apply(-lap + lam * p)
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * max(1.0, np.linalg.norm(rhs)) * N


@pytest.mark.parametrize("N", range(1, 11))
@pytest.mark.parametrize("lam", [0.0, 3.5])
def test_polynomial_exactness_with_neumann_sides(N, lam):
    """Neumann on x = 0 and x = 1, Dirichlet (g = p) on y = 0 and y = 1: for a
    polynomial with dp/dx = 0 on x = 0, 1 the homogeneous Neumann faces carry
    exactly the right (zero) flux and no jump, so A p + L(g) = M(-lap p + lam p)
    again, with data g that equal p on the Dirichlet sides only (g - p = 5 y (1 - y)
    is not zero on the Neumann sides). A Neumann face that takes a Dirichlet block
    or boundary data fails."""
    m = rotate_local_vertices(jittered_grid(3, 3, jitter=0.1, seed=0, bc_sides=(2, 2, 1, 1)), N)
    S = _sip(m, N)
    x, y = S.x, S.y
    p = 0.3 + 0.7 * y ** N
    lap = 0.7 * N * (N - 1) * y ** (N - 2) if N >= 2 else np.zeros_like(x)
    if N >= 4:  # x^2 (1 - x)^2 has zero slope at x = 0 and x = 1
        X = x * x * (1 - x) ** 2
        Xpp = 2 - 12 * x + 12 * x * x
        p = p + X * y ** (N - 4)
        lap = lap + Xpp * y ** (N - 4)
        if N >= 6:
            lap = lap + X * (N - 4) * (N - 5) * y ** (N - 6)
    lhs = S.apply(p, lam=lam) + S.dirichlet_lift(p + 5.0 * y * (1.0 - y))
    rhs = S.mass_apply(-lap + lam * p)
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * max(1.0, np.linalg.norm(rhs)) * N


def test_helmholtz_large_lambda_tends_to_mass():
    S = _sip(_mesh(2, rotate=0), 4)
    lam = 1e9
    A = S.assemble(lam).toarray() / lam
    Mref = S.mass_matrix_ref()
    for e in range(S.K):
        blk = A[e * S.Np:(e + 1) * S.Np, e * S.Np:(e + 1) * S.Np]
        assert np.allclose(blk, S.geo.J[e] * Mref, rtol=0, atol=1e-6 * np.abs(Mref).max())


@pytest.mark.parametrize("N", [2, 5])
def test_matrix_free_equals_assembled_and_sampling(N):
    S = _sip(_mesh(4, rotate=7), N)
    u = np.random.default_rng(1).uniform(-1, 1, (S.K, S.Np))
    A = S.assemble(2.0)
    ref = (A @ u.ravel()).reshape(u.shape)
    mf = S.apply(u, lam=2.0)
    assert np.abs(ref - mf).max() < 1e-12 * np.abs(ref).max()
    elems = np.array([0, 5, 17, S.K - 1])
    assert np.abs(S.apply(u, lam=2.0, elems=elems) - ref[elems]).max() < 1e-12 * np.abs(ref).max()
    ub = np.stack([u, 2 * u])
    assert np.allclose(S.apply(ub, lam=2.0), np.stack([mf, 2 * mf]), rtol=1e-13, atol=1e-12)


def test_invariant_under_local_vertex_rotation():
    """Rotating each element's local vertex list permutes its (symmetric) node
    set; the operator must be the same up to that permutation."""
    m = _mesh(3)
    mr = rotate_local_vertices(m, 11)
    N = 4
    S, Sr = _sip(m, N), _sip(mr, N)
    u = np.random.default_rng(2).uniform(-1, 1, (S.K, S.Np))
    perm = np.empty((S.K, S.Np), dtype=int)
    for e in range(S.K):
        for i in range(S.Np):
            d = (S.x[e] - Sr.x[e, i]) ** 2 + (S.y[e] - Sr.y[e, i]) ** 2
            perm[e, i] = int(np.argmin(d))
            assert d[perm[e, i]] < 1e-24
    ur = np.take_along_axis(u, perm, axis=1)
    Au = S.apply(u)
    Aur = Sr.apply(ur)
    assert np.abs(np.take_along_axis(Au, perm, axis=1) - Aur).max() < 1e-12 * np.abs(Au).max()


@pytest.mark.parametrize("N", [1, 2, 3])
def test_h_convergence_rate(N):
    """Manufactured u = sin(pi x) sin(pi y): L2 error ~ h^{N+1} (Section 4.1)."""
    uex, fex = manufactured("sin_pi_x_sin_pi_y")
    errs = []
    for n in (4, 8, 16):
        S = _sip(_mesh(n), N)
        A = S.assemble().tocsc()
        b = S.rhs(fex(S.x, S.y), uex(S.x, S.y))
        u = spla.spsolve(A, b.ravel()).reshape(S.K, S.Np)
        errs.append(S.l2_error(u, uex))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > N + 1 - 0.35, (errs, rates)


def test_p_convergence_is_spectral():
    """Manufactured u = sin(pi x) sin(pi y) on a fixed 4x4 grid: raising N lowers
    the L2 error exponentially for a smooth solution (the paper's p-convergence
    statement in Section 4.1). Measured gains per step N -> N+1 are 11-26 up to
    N = 7; an algebraic rate p would give gains ((N+1)/N)^p that decay toward 1,
    so every gain staying above 8 and log(err) falling linearly in N pin it."""
    uex, fex = manufactured("sin_pi_x_sin_pi_y")
    errs = []
    for N in range(1, 8):
        S = _sip(_mesh(4), N)
        A = S.assemble().tocsc()
        b = S.rhs(fex(S.x, S.y), uex(S.x, S.y))
        u = spla.spsolve(A, b.ravel()).reshape(S.K, S.Np)
        errs.append(S.l2_error(u, uex))
    gains = np.array(errs[:-1]) / np.array(errs[1:])
    assert (gains > 8.0).all(), (errs, gains)
    slope = np.polyfit(np.arange(1, 8), np.log(errs), 1)[0]
    assert slope < -2.0, (errs, slope)
    assert errs[-1] < 1e-8
