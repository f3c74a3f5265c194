"""Pins of the reference operators of Section 5.2 (Eq. elMass, elStiff, elLift)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import basis, refops
from tests.test_oracle_basis import _tri_monomial


@pytest.mark.parametrize("N", range(1, 11))
def test_derivatives_exact_on_monomials(N):
    ops = refops.reference_operators(N)
    r, s = ops["r"], ops["s"]
    assert np.abs(ops["Dr"] @ np.ones_like(r)).max() < 1e-12
    for a in range(N + 1):
        for b in range(N + 1 - a):
            u = r ** a * s ** b
            ur = a * r ** max(a - 1, 0) * s ** b if a > 0 else 0 * r
            us = b * r ** a * s ** max(b - 1, 0) if b > 0 else 0 * r
            assert np.abs(ops["Dr"] @ u - ur).max() < 1e-11 * max(1, N ** 2)
            assert np.abs(ops["Ds"] @ u - us).max() < 1e-11 * max(1, N ** 2)


@pytest.mark.parametrize("N", range(1, 11))
def test_mass_integrates_monomials(N):
    ops = refops.reference_operators(N)
    r, s, M = ops["r"], ops["s"], ops["M"]
    one = np.ones_like(r)
    assert abs(one @ M @ one - 2.0) < 1e-13
    for a in range(N + 1):
        for b in range(N + 1 - a):
            assert abs(one @ M @ (r ** a * s ** b) - _tri_monomial(a, b)) < 1e-12


@pytest.mark.parametrize("N", range(1, 11))
def test_lift_reproduces_face_integrals(N):
    """v^T M LIFT_f w_f = integral over face f (parameter t in [-1,1]) of v w,
    checked with an independent Gauss-Legendre rule on each edge."""
    ops = refops.reference_operators(N)
    r, s, M, LIFT = ops["r"], ops["s"], ops["M"], ops["LIFT"]
    Nfp = N + 1
    x, w = npleg.leggauss(N + 2)
    ends = [((-1, -1), (1, -1)), ((1, -1), (-1, 1)), ((-1, 1), (-1, -1))]
    rng = np.random.default_rng(N)
    for f in range(3):
        (ra, sa), (rb, sb) = ends[f]
        rq = ra + 0.5 * (x + 1) * (rb - ra)
        sq = sa + 0.5 * (x + 1) * (sb - sa)
        cv = rng.standard_normal((N + 1, N + 1))
        cw = rng.standard_normal((N + 1, N + 1))
        pv = lambda rr, ss: sum(cv[i, j] * rr ** i * ss ** j for i in range(N + 1) for j in range(N + 1 - i))
        pw = lambda rr, ss: sum(cw[i, j] * rr ** i * ss ** j for i in range(N + 1) for j in range(N + 1 - i))
        exact = np.sum(w * pv(rq, sq) * pw(rq, sq))
        fl = ops["faces"][f]
        wf = np.zeros(3 * Nfp)
        wf[f * Nfp:(f + 1) * Nfp] = pw(r[fl], s[fl])
        got = pv(r, s) @ M @ (LIFT @ wf)
        assert abs(got - exact) < 1e-10 * max(1, abs(exact))


@pytest.mark.parametrize("Nf,Nc", [(2, 1), (3, 1), (6, 3), (8, 4), (4, 2), (10, 5)])
def test_pmg_interpolation_reproduces_coarse_polynomials(Nf, Nc):
    P = refops.interpolation(Nf, Nc)
    rf, sf = basis.warp_blend_nodes(Nf)
    rc, sc = basis.warp_blend_nodes(Nc)
    for a in range(Nc + 1):
        for b in range(Nc + 1 - a):
            assert np.abs(P @ (rc ** a * sc ** b) - rf ** a * sf ** b).max() < 1e-12
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
