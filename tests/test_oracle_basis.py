"""Pins of the oracle's bases, Gauss rules and Warp & Blend nodes (Section 2.1)."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import basis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_lgl():
    out = {}
    with open(os.path.join(GOLDEN, "lgl_points.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            out[int(parts[0])] = np.array([float(v) for v in parts[1:]])
    return out


@pytest.mark.parametrize("alpha,beta", [(0, 0), (1, 0), (3, 0), (5, 0), (1, 1), (2, 2)])
def test_jacobi_orthonormal(alpha, beta):
    # integrate (1-x)^a (1+x)^b P_m P_n with a 40-point Gauss-Legendre rule (exact)
    x, w = npleg.leggauss(40)
    wt = w * (1 - x) ** alpha * (1 + x) ** beta
    P = np.stack([basis.jacobi_normalized(x, alpha, beta, n) for n in range(9)])
    G = (P * wt) @ P.T
    assert np.allclose(G, np.eye(9), atol=1e-12)


@pytest.mark.parametrize("n", range(1, 9))
def test_jacobi_derivative_matches_finite_difference(n):
    x = np.linspace(-0.9, 0.9, 7)
    h = 1e-6
    for a, b in [(0, 0), (3, 0)]:
        fd = (basis.jacobi_normalized(x + h, a, b, n) - basis.jacobi_normalized(x - h, a, b, n)) / (2 * h)
        assert np.allclose(basis.jacobi_normalized_deriv(x, a, b, n), fd, rtol=1e-6, atol=1e-6)


def test_lgl_points_golden_and_legendre_roots():
    gold = _read_lgl()
    for N, pts in gold.items():
        assert np.allclose(basis.gauss_lobatto(N), pts, atol=1e-15)
    for N in range(2, 12):
        c = np.zeros(N + 1)
        c[N] = 1.0
        inner = np.sort(npleg.legroots(npleg.legder(c)).real)
        assert np.allclose(basis.gauss_lobatto(N)[1:-1], inner, atol=1e-13)


def test_warp_blend_low_degree_nodes():
    r, s = basis.warp_blend_nodes(1)
    assert np.allclose(np.c_[r, s], [[-1, -1], [1, -1], [-1, 1]], atol=1e-15)
    r, s = basis.warp_blend_nodes(2)
    assert np.allclose(np.c_[r, s], [[-1, -1], [0, -1], [1, -1], [-1, 0], [0, 0], [-1, 1]], atol=1e-15)
    r, s = basis.warp_blend_nodes(3)
    # the one interior node of the symmetric N=3 set is the centroid
    assert np.allclose([r[5], s[5]], [-1 / 3, -1 / 3], atol=1e-14)


@pytest.mark.parametrize("N", range(1, 11))
def test_warp_blend_edges_are_lobatto_and_set_is_symmetric(N):
    r, s = basis.warp_blend_nodes(N)
    assert len(r) == (N + 1) * (N + 2) // 2
    t = basis.gauss_lobatto(N)
    fl = basis.face_node_lists(N)
    # face 0: s = -1, r = t; face 1: r + s = 0, r = -t; face 2: r = -1, s = -t
    assert np.allclose(s[fl[0]], -1) and np.allclose(r[fl[0]], t, atol=1e-13)
    assert np.allclose(r[fl[1]] + s[fl[1]], 0, atol=1e-13) and np.allclose(r[fl[1]], -t, atol=1e-13)
    assert np.allclose(r[fl[2]], -1) and np.allclose(s[fl[2]], -t, atol=1e-13)
    # invariance under the six symmetries of the triangle (barycentric permutations)
    lam = np.stack([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2], axis=1)
    key = lambda L: set(tuple(np.round(row, 10)) for row in L)
    base = key(lam)
    for perm in itertools.permutations(range(3)):
        assert key(lam[:, perm]) == base
    # all nodes in the closed triangle
    assert np.all(r >= -1 - 1e-13) and np.all(s >= -1 - 1e-13) and np.all(r + s <= 1e-13)


def _tri_monomial(a, b):
    """Exact integral of r^a s^b over the bi-unit triangle: r = 2x-1, s = 2y-1
    on the unit simplex, int x^p y^q = p! q! / (p+q+2)!."""
    tot = Fraction(0)
    for p in range(a + 1):
        for q in range(b + 1):
            c = (math.comb(a, p) * math.comb(b, q) * 2 ** (p + q) * (-1) ** (a - p + b - q))
            tot += Fraction(c * math.factorial(p) * math.factorial(q), math.factorial(p + q + 2))
    return float(4 * tot)


@pytest.mark.parametrize("n", [1, 3, 5, 9])
def test_triangle_quadrature_exact(n):
    r, s, w = basis.triangle_quadrature(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            assert abs(np.sum(w * r ** a * s ** b) - _tri_monomial(a, b)) < 1e-13 * max(1, abs(_tri_monomial(a, b))) + 1e-14


@pytest.mark.parametrize("N", [1, 4, 8])
def test_simplex_basis_orthonormal_and_gradients(N):
    r, s, w = basis.triangle_quadrature(N + 2)
    V = basis.vandermonde(N, r, s)
    assert np.allclose((V * w[:, None]).T @ V, np.eye(V.shape[1]), atol=1e-12)
    rng = np.random.default_rng(0)
    rr = rng.uniform(-0.9, 0.2, 20)
    ss = rng.uniform(-0.9, -0.1, 20)
    ok = rr + ss < -0.05
    rr, ss = rr[ok], ss[ok]
    h = 1e-6
    Vr, Vs = basis.vandermonde_grad(N, rr, ss)
    fr = (basis.vandermonde(N, rr + h, ss) - basis.vandermonde(N, rr - h, ss)) / (2 * h)
    fs = (basis.vandermonde(N, rr, ss + h) - basis.vandermonde(N, rr, ss - h)) / (2 * h)
    assert np.allclose(Vr, fr, atol=1e-6) and np.allclose(Vs, fs, atol=1e-6)
