"""Pins of the tetrahedral SIPDG oracle (the paper's three-dimensional extension,
Section 6, with the readings stated in oracle/tet.py)."""
from math import factorial

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from dg_inputs.tetmesh import jittered_tet_grid
from oracle.tet import TetSipdg, tet_nodes, tet_quadrature


def _sip(n, N, seed=1, bc_sides=(1,) * 6):
    m = jittered_tet_grid(n, jitter=0.1, seed=seed, bc_sides=bc_sides)
    return TetSipdg(m.VX, m.VY, m.VZ, m.EToV, m.bc, N), m


@pytest.mark.parametrize("n", [2, 3, 5])
def test_tet_quadrature_against_simplex_closed_form(n):
    """Over the unit simplex, int x^a y^b z^c = a! b! c! / (a+b+c+3)!; the
    reference tetrahedron is its image under (r, s, t) = 2 (x, y, z) - 1."""
    r, s, t, w = tet_quadrature(n)
    x, y, z = (r + 1) / 2, (s + 1) / 2, (t + 1) / 2
    for a in range(2 * n):
        for b in range(2 * n - a):
            for c in range(2 * n - a - b):
                exact = 8.0 * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
                assert abs(np.sum(w * x ** a * y ** b * z ** c) - exact) <= 1e-14, (a, b, c)


@pytest.mark.parametrize("N", range(1, 6))
def test_tet_nodes_count_and_faces(N):
    r, s, t = tet_nodes(N)
    assert len(r) == (N + 1) * (N + 2) * (N + 3) // 6
    nf = (N + 1) * (N + 2) // 2
    on = [np.isclose(t, -1), np.isclose(s, -1), np.isclose(r + s + t, -1), np.isclose(r, -1)]
    assert all(int(o.sum()) == nf for o in on)


def test_penalty_by_hand_on_the_corner_tetrahedron():
    """The tetrahedron (0,0,0), (1,0,0), (0,1,0), (0,0,1): volume 1/6, three faces
    of area 1/2 and one of area sqrt(3)/2, so 1/h = |face|/|E| = 3 and 3 sqrt(3);
    all faces on the boundary (interior side only), N = 2: (N+1)(N+3)/3 = 5."""
    S = TetSipdg([0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1], [[0, 1, 2, 3]], [[1, 1, 1, 1]], 2)
    # faces: 0 = (v0,v1,v2) on z = 0, 1 = (v0,v1,v3) on y = 0, 2 = (v1,v2,v3) slanted, 3 = (v0,v2,v3) on x = 0
    assert np.allclose(S.tau[0], [15.0, 15.0, 15.0 * np.sqrt(3.0), 15.0], rtol=1e-14)


def test_penalty_takes_the_larger_side_on_interior_faces():
    S, _ = _sip(2, 1)
    g = S.geo
    ih = g.area / g.vol[:, None]
    for e in range(S.K):
        for f in range(4):
            e2, f2 = g.EToE[e, f], g.EToF[e, f]
            want = 2 * 4 / 3 * (max(ih[e, f], ih[e2, f2]) if e2 >= 0 else ih[e, f])
            assert abs(S.tau[e, f] - want) <= 1e-12 * want


@pytest.mark.parametrize("n,N", [(1, 1), (1, 3), (2, 2), (2, 4)])
def test_tet_symmetric_positive_definite(n, N):
    S, _ = _sip(n, N)
    A = S.assemble().toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_tet_all_neumann_kills_constants():
    S, _ = _sip(2, 2, bc_sides=(2,) * 6)
    assert np.abs(S.apply(np.ones((S.K, S.Np)))).max() < 1e-12


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("lam", [0.0, 1.5])
def test_tet_polynomial_exactness_with_dirichlet_data(N, lam):
    """For p of degree <= N (here quadratic) the discrete form is consistent:
    A p + L(p) = M(-lap p + lam p) node by node."""
    S, _ = _sip(2, N, seed=3)
    p = lambda x, y, z: x * x - 2 * y * z + 0.5 * z + 0.3 * x - 0.1
    P = p(S.x, S.y, S.z)
    lhs = S.apply(P, lam=lam) + S.dirichlet_lift(P)
    rhs = S.mass_apply(-2.0 + lam * P)
    assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(rhs).max()


def test_tet_h_convergence_rate():
    """u = sin(pi x) sin(pi y) sin(pi z) on the unit cube, Dirichlet: the L2
    error of the discrete solution (by a quadrature exact to degree 2N + 6)
    falls like h^{N+1}; measured rates between n = 2 and 4 cubes a side are
    3.18 (N = 2) and 3.76 (N = 3)."""
    u = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    f = lambda x, y, z: 3 * np.pi ** 2 * u(x, y, z)
    for N, rmin in ((2, 2.8), (3, 3.5)):
        errs = []
        for n in (2, 4):
            m = jittered_tet_grid(n, jitter=0.0)
            S = TetSipdg(m.VX, m.VY, m.VZ, m.EToV, m.bc, N)
            b = S.rhs(f(S.x, S.y, S.z), u(S.x, S.y, S.z))
            x = spla.spsolve(S.assemble().tocsc(), b.ravel()).reshape(b.shape)
            rq, sq, tq, wq = tet_quadrature(N + 3)
            Lq = S._eval_basis(rq, sq, tq)[0]
            X = S.geo.to_physical(np.arange(S.K), rq[None], sq[None], tq[None])
            e = x @ Lq.T - u(X[..., 0], X[..., 1], X[..., 2])
            errs.append(np.sqrt(np.sum(e ** 2 * wq[None] * S.geo.J[:, None])))
        assert np.log2(errs[0] / errs[1]) > rmin, (N, errs)


@pytest.mark.parametrize("N", [1, 3])
def test_tet_operator_invariant_under_local_vertex_renumbering(N):
    """Renumbering each element's vertices (even permutations, face tags moved
    with them) renumbers the nodes of the element and nothing else: A u at every
    physical node is unchanged."""
    from dg_inputs.tetmesh import permute_local_vertices
    m = jittered_tet_grid(2, jitter=0.1, seed=3, bc_sides=(1, 2, 2, 1, 1, 2))
    pm = permute_local_vertices(m, 5)
    S1 = TetSipdg(m.VX, m.VY, m.VZ, m.EToV, m.bc, N)
    S2 = TetSipdg(pm.VX, pm.VY, pm.VZ, pm.EToV, pm.bc, N)
    f = lambda x, y, z: np.sin(x + 2 * y) * np.cos(z) + x * z
    A1 = S1.apply(f(S1.x, S1.y, S1.z), lam=0.5)
    A2 = S2.apply(f(S2.x, S2.y, S2.z), lam=0.5)
    X1 = np.stack([S1.x, S1.y, S1.z], -1)
    X2 = np.stack([S2.x, S2.y, S2.z], -1)
    for e in range(S1.K):
        d = np.linalg.norm(X1[e][:, None, :] - X2[e][None, :, :], axis=-1)
        perm = d.argmin(axis=1)
        assert np.all(d[np.arange(S1.Np), perm] < 1e-12)
        assert np.abs(A1[e] - A2[e][perm]).max() <= 1e-12 * np.abs(A1).max()


def test_tet_mass_integrates_volume_and_moments():
    """1^T J M p is the integral of p over the mesh: the unit cube's volume 1 and its
    first and second moments 1/2 and 1/3 (p = 1, x, y^2)."""
    S, _ = _sip(2, 2)
    for p, want in ((np.ones_like(S.x), 1.0), (S.x, 0.5), (S.y ** 2, 1.0 / 3.0)):
        assert abs(S.mass_apply(p).sum() - want) <= 1e-13


def test_tet_helmholtz_is_poisson_plus_lambda_mass():
    """A(lambda) u = A(0) u + lambda J M u: the screened term enters the element
    blocks only, at the quadrature that integrates the mass exactly."""
    S, _ = _sip(2, 3, seed=4)
    u = np.random.default_rng(2).uniform(-1, 1, (S.K, S.Np))
    lam = 7.25
    d = S.apply(u, lam=lam) - S.apply(u)
    assert np.abs(d - lam * S.mass_apply(u)).max() <= 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("N,lost", [(1, 0.1), (2, 0.25), (3, 0.25)])
def test_tet_penalty_keeps_the_form_coercive_with_margin(N, lost):
    """The interior penalty has to dominate the consistency terms: with the
    reading's tau = (N+1)(N+3)/3 max(1/h) the assembled form stays positive
    definite at half the penalty too, and loses definiteness once the penalty is
    cut to a quarter (a tenth at N = 1): the constant is of the right size, not
    merely positive."""
    S, _ = _sip(2, N)
    t0 = S.tau.copy()

    def lam_min(scale):
        S.tau = t0 * scale
        A = S.assemble().toarray()
        return np.linalg.eigvalsh(0.5 * (A + A.T)).min()

    assert lam_min(1.0) > 0 and lam_min(0.5) > 0
    assert lam_min(lost) < 0
