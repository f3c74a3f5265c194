"""Pins of the oracle's CG, Chebyshev and p-multigrid (Section 3)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from dg_inputs import jittered_grid, manufactured
from oracle import refops
from oracle.sipdg import Sipdg
from oracle.solvers import PMultigrid, cg, chebyshev, inverse_mass_prec, power_rho


def test_cg_terminates_in_number_of_distinct_eigenvalues():
    d = np.repeat([1.0, 2.0, 5.0, 11.0], 25)
    b = np.random.default_rng(0).standard_normal(d.size)
    x, it, rel = cg(lambda v: d * v, b, tol=1e-13)
    assert it <= 4 and rel < 1e-13
    assert np.allclose(x, b / d)


def test_chebyshev_degree2_matches_closed_form():
    """Scalar A = lam, D = 1: e_k = T_k((theta-lam)/delta) / T_k(theta/delta) e_0."""
    lmin, lmax = 0.4, 3.0
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    T2 = lambda t: 2 * t * t - 1
    for lam in (0.5, 1.3, 2.9):
        b = np.array([lam * 1.0])   # exact solution 1
        x = chebyshev(lambda v: lam * v, np.ones(1), b, np.zeros(1), lmin, lmax, 2)
        e_pred = T2((theta - lam) / delta) / T2(theta / delta) * (0.0 - 1.0)
        assert abs((x[0] - 1.0) - e_pred) < 1e-14


def _problem(n, N, rotate=None):
    from dg_inputs.mesh import rotate_local_vertices
    m = jittered_grid(n, n, jitter=0.1, seed=0)
    if rotate is not None:
        m = rotate_local_vertices(m, rotate)
    return Sipdg(m.VX, m.VY, m.EToV, m.bc, N)


def test_jacobi_pcg_matches_direct_solve():
    S = _problem(8, 3)
    A = S.assemble()
    uex, fex = manufactured("sin_pi_x_sin_pi_y")
    b = S.rhs(fex(S.x, S.y), uex(S.x, S.y))
    xd = spla.spsolve(A.tocsc(), b.ravel())
    dinv = 1.0 / S.diagonal()
    x, it, rel = cg(lambda v: (A @ v.ravel()).reshape(v.shape), b, tol=1e-12, prec=lambda r: dinv * r)
    assert rel <= 1e-12
    assert np.linalg.norm(x.ravel() - xd) <= 1e-9 * np.linalg.norm(xd)


def _pmg(n, degrees, coarse_exact=False, rotate=None):
    sips = [_problem(n, d, rotate) for d in degrees]
    mats = [s.assemble() for s in sips]
    ops = []
    for s, A in zip(sips, mats):
        ops.append(((lambda A_: (lambda v: (A_ @ v.reshape(-1, ).copy()).reshape(v.shape)))(A),
                    1.0 / s.diagonal()))
    P = [refops.interpolation(degrees[l], degrees[l + 1]) for l in range(len(degrees) - 1)]
    shapes = [(s.K, s.Np) for s in sips]
    cs = None
    if coarse_exact:
        Ac = mats[-1].tocsc()
        lu = spla.splu(Ac)
        cs = lambda r: lu.solve(r.ravel()).reshape(r.shape)
    return sips, mats, PMultigrid(ops, P, shapes, cheb_degree=2, coarse_tol=1e-2, coarse_solve=cs)


def test_vcycle_is_symmetric_with_exact_coarse_solve():
    sips, mats, pmg = _pmg(4, [6, 3, 1], coarse_exact=True, rotate=5)
    rng = np.random.default_rng(3)
    y = rng.standard_normal((sips[0].K, sips[0].Np))
    z = rng.standard_normal((sips[0].K, sips[0].Np))
    lhs = np.vdot(y, pmg.vcycle(z))
    rhs = np.vdot(z, pmg.vcycle(y))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_pmg_fcg_converges_to_direct_solution_and_beats_jacobi():
    sips, mats, pmg = _pmg(8, [6, 3, 1])
    S, A = sips[0], mats[0]
    uex, fex = manufactured("sin_2pi_x_cos_3pi_y")
    b = S.rhs(fex(S.x, S.y), uex(S.x, S.y))
    xd = spla.spsolve(A.tocsc(), b.ravel())
    Aop = lambda v: (A @ v.ravel()).reshape(v.shape)
    x, it, rel = cg(Aop, b, tol=1e-10, prec=pmg.vcycle, flexible=True)
    assert rel <= 1e-10
    assert np.linalg.norm(x.ravel() - xd) <= 1e-7 * np.linalg.norm(xd)
    dinv = 1.0 / S.diagonal()
    _, itj, _ = cg(Aop, b, tol=1e-10, prec=lambda r: dinv * r)
    assert it < itj / 4, (it, itj)


def test_power_estimate_bounds_spectrum():
    S = _problem(3, 3)
    A = S.assemble().toarray()
    d = np.diag(A)
    ev = np.linalg.eigvals(A / d[:, None]).real
    rho = power_rho(lambda v: (A @ v.ravel()).reshape(v.shape), 1.0 / S.diagonal(), (S.K, S.Np), steps=60)
    assert 0.9 * ev.max() <= rho <= ev.max() * (1 + 1e-9)


def test_inverse_mass_preconditioner_is_block_inverse():
    S = _problem(3, 4)
    lam = 7.0
    prec = inverse_mass_prec(S, lam)
    r = np.random.default_rng(4).standard_normal((S.K, S.Np))
    z = prec(r)
    assert np.allclose(lam * S.mass_apply(z), r, atol=1e-11)
