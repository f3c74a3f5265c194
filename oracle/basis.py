"""Polynomial bases, Gauss rules and Warp & Blend nodes on the triangle (oracle).

TEST INFRASTRUCTURE ONLY.

Section 2.1 of the paper takes the nodal basis of P_N on each triangle to be
the Lagrange polynomials through the Warp & Blend nodes of Warburton (2006).
That construction is not printed in the paper; it is restated here from the
cited publication: equidistant barycentric nodes on an equilateral triangle
are displaced along each edge direction by a 1-D warp (the Gauss-Lobatto minus
equidistant displacement, interpolated) times an edge blend 4*L_a*L_b that is
enhanced in the interior by (1 + (alpha*L_c)^2), with the per-degree alpha
optimised in that publication.

Library routines used as steps: scipy.special.eval_jacobi, roots_jacobi and
gammaln (Jacobi polynomials and their Gauss rules).
"""
import numpy as np
from scipy.special import eval_jacobi, gammaln, roots_jacobi

# Optimised blend parameters alpha(N), N = 1..15 (Warburton 2006, Table 1).
ALPHA_OPT = [0.0000, 0.0000, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999, 1.2832,
             1.3648, 1.4773, 1.4959, 1.5743, 1.5770, 1.6223, 1.6258]


def jacobi_normalized(x, alpha, beta, n):
    """P_n^{(alpha,beta)}(x) scaled to unit norm w.r.t. (1-x)^alpha (1+x)^beta:
    the 1-D factors of the orthonormal basis behind the nodal basis of Section 2.1."""
    x = np.asarray(x, dtype=np.float64)
    # squared norm of the classical polynomial
    lh = ((alpha + beta + 1) * np.log(2.0) - np.log(2 * n + alpha + beta + 1)
          + gammaln(n + alpha + 1) + gammaln(n + beta + 1)
          - gammaln(n + alpha + beta + 1) - gammaln(n + 1))
    return eval_jacobi(n, alpha, beta, x) / np.exp(0.5 * lh)


def jacobi_normalized_deriv(x, alpha, beta, n):
    """d/dx of jacobi_normalized, from d/dx P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1)
    (for the derivative matrices of Section 5.2, Eq. operators1)."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return np.sqrt(n * (n + alpha + beta + 1.0)) * jacobi_normalized(x, alpha + 1, beta + 1, n - 1)


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1] (exact to degree 2n-1): the face
    integrals of Eq. ellipticOp1 and Eq. INS_CUB_N."""
    x, w = roots_jacobi(n, 0.0, 0.0)
    return np.asarray(x), np.asarray(w)


def gauss_lobatto(N):
    """N+1 Legendre-Gauss-Lobatto points on [-1, 1]: the endpoints and the
    zeros of P_N', which are the zeros of P_{N-1}^{(1,1)} (the edge nodes of the
    Warp & Blend set of Section 2.1)."""
    if N == 1:
        return np.array([-1.0, 1.0])
    xi, _ = roots_jacobi(N - 1, 1.0, 1.0)
    return np.concatenate([[-1.0], np.sort(np.asarray(xi)), [1.0]])


def warp_factor(N, rout):
    """1-D warp: the interpolant (through equispaced points) of the displacement
    from equispaced to Gauss-Lobatto points, divided by the edge blend 1-r^2
    (Warburton 2006, the node construction Section 2.1 cites)."""
    rout = np.asarray(rout, dtype=np.float64)
    r_gl = gauss_lobatto(N)
    r_eq = np.linspace(-1.0, 1.0, N + 1)
    # Lagrange basis through r_eq evaluated at rout
    warp = np.zeros_like(rout)
    for i in range(N + 1):
        li = np.ones_like(rout)
        for j in range(N + 1):
            if j != i:
                li = li * (rout - r_eq[j]) / (r_eq[i] - r_eq[j])
        warp = warp + li * (r_gl[i] - r_eq[i])
    interior = np.abs(rout) < 1.0 - 1e-10
    out = np.where(interior, warp / np.where(interior, 1.0 - rout ** 2, 1.0), 0.0)
    return out


def warp_blend_nodes(N):
    """Warp & Blend nodes on the bi-unit triangle {r,s >= -1, r+s <= 0}
    (Section 2.1; Warburton 2006 with its Table 1 blend parameters).

    Ordering: rows of constant s from s=-1 upward; within a row r increases.
    Node 0 = (-1,-1), node N = (1,-1), node Np-1 = (-1,1).
    """
    alpha = ALPHA_OPT[N - 1] if N <= 15 else 5.0 / 3.0
    L1, L3 = [], []
    for n in range(N + 1):          # row index (s direction)
        for m in range(N + 1 - n):  # position in row (r direction)
            L1.append(n / N)
            L3.append(m / N)
    L1 = np.array(L1)
    L3 = np.array(L3)
    L2 = 1.0 - L1 - L3
    # equilateral triangle with vertices (-1,-1/sqrt3), (1,-1/sqrt3), (0,2/sqrt3)
    X = -L2 + L3
    Y = (-L2 - L3 + 2.0 * L1) / np.sqrt(3.0)
    b1, b2, b3 = 4 * L2 * L3, 4 * L1 * L3, 4 * L1 * L2
    w1 = warp_factor(N, L3 - L2)
    w2 = warp_factor(N, L1 - L3)
    w3 = warp_factor(N, L2 - L1)
    d1 = b1 * w1 * (1 + (alpha * L1) ** 2)
    d2 = b2 * w2 * (1 + (alpha * L2) ** 2)
    d3 = b3 * w3 * (1 + (alpha * L3) ** 2)
    X = X + d1 + np.cos(2 * np.pi / 3) * d2 + np.cos(4 * np.pi / 3) * d3
    Y = Y + np.sin(2 * np.pi / 3) * d2 + np.sin(4 * np.pi / 3) * d3
    # back to the bi-unit right triangle through barycentric coordinates
    l1 = (np.sqrt(3.0) * Y + 1.0) / 3.0
    l2 = (-3.0 * X - np.sqrt(3.0) * Y + 2.0) / 6.0
    l3 = (3.0 * X - np.sqrt(3.0) * Y + 2.0) / 6.0
    r = -l2 + l3 - l1
    s = -l2 - l3 + l1
    return r, s


def face_node_lists(N):
    """Local node indices of the three faces, each in counter-clockwise order:
    face 0 v0->v1 (s=-1), face 1 v1->v2 (r+s=0), face 2 v2->v0 (r=-1): the
    face nodes of Section 2.1 (ordering: a reading, the paper is silent)."""
    rows = []
    k = 0
    for n in range(N + 1):
        rows.append(list(range(k, k + N + 1 - n)))
        k += N + 1 - n
    f0 = rows[0]
    f1 = [row[-1] for row in rows]
    f2 = [row[0] for row in rows][::-1]
    return [np.array(f0), np.array(f1), np.array(f2)]


def collapsed(r, s):
    """Collapsed coordinates a = 2(1+r)/(1-s) - 1, b = s (a = -1 at s = 1), in
    which the orthonormal basis of Section 2.1 factors into Jacobi polynomials."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    top = np.abs(1.0 - s) < 1e-14
    a = np.where(top, -1.0, 2.0 * (1.0 + r) / np.where(top, 1.0, 1.0 - s) - 1.0)
    return a, s


def simplex_modes(N):
    """Mode indices (i, j), i + j <= N, of P_N on the triangle (Section 2.1)."""
    return [(i, j) for i in range(N + 1) for j in range(N + 1 - i)]


def simplex_basis(r, s, i, j):
    """Orthonormal (Dubiner) basis function psi_ij on the bi-unit triangle: the
    modal basis whose Vandermonde gives M and Dr, Ds (Section 5.2, Eq. operators1)."""
    a, b = collapsed(r, s)
    return (np.sqrt(2.0) * jacobi_normalized(a, 0, 0, i)
            * jacobi_normalized(b, 2 * i + 1, 0, j) * (1.0 - b) ** i)


def simplex_basis_grad(r, s, i, j):
    """(d psi_ij / dr, d psi_ij / ds) by the chain rule through (a, b) (for Dr, Ds of
    Section 5.2, Eq. operators1)."""
    a, b = collapsed(r, s)
    fa = jacobi_normalized(a, 0, 0, i)
    dfa = jacobi_normalized_deriv(a, 0, 0, i)
    gb = jacobi_normalized(b, 2 * i + 1, 0, j)
    dgb = jacobi_normalized_deriv(b, 2 * i + 1, 0, j)
    # d/dr = 2/(1-b) d/da ; d/ds = (1+a)/(1-b) d/da + d/db
    if i == 0:
        dr = np.zeros_like(a)
        ds = fa * dgb
    else:
        omb_im1 = (1.0 - b) ** (i - 1)
        dr = 2.0 * dfa * gb * omb_im1
        ds = (1.0 + a) * dfa * gb * omb_im1 + fa * (dgb * (1.0 - b) ** i - i * gb * omb_im1)
    return np.sqrt(2.0) * dr, np.sqrt(2.0) * ds


def vandermonde(N, r, s):
    """V[q, k] = psi_k(r_q, s_q) over the modes of simplex_modes(N): the
    Vandermonde matrix of Section 5.2 (M = (V V^T)^{-1}, Eq. elMass)."""
    return np.stack([simplex_basis(r, s, i, j) for (i, j) in simplex_modes(N)], axis=-1)


def vandermonde_grad(N, r, s):
    """(Vr, Vs): derivatives of the basis at the points, so that Dr = Vr V^{-1}
    and Ds = Vs V^{-1} (Section 5.2, Eq. operators1)."""
    g = [simplex_basis_grad(r, s, i, j) for (i, j) in simplex_modes(N)]
    return np.stack([t[0] for t in g], axis=-1), np.stack([t[1] for t in g], axis=-1)


def triangle_quadrature(n):
    """Collapsed (Duffy) rule on the bi-unit triangle with n x n points: the
    volume integrals of Eq. ellipticOp1 and the cubature of Eq. INS_CUB_N.

    a: n-point Gauss-Legendre; b: n-point Gauss-Jacobi with weight (1-b);
    dr ds = (1-b)/2 da db. Exact for polynomials of total degree <= 2n-1.
    """
    xa, wa = gauss_legendre(n)
    xb, wb = roots_jacobi(n, 1.0, 0.0)
    A, Bm = np.meshgrid(xa, xb, indexing="ij")
    W = np.outer(wa, wb) * 0.5
    r = 0.5 * (1.0 + A) * (1.0 - Bm) - 1.0
    s = Bm
    return r.ravel(), s.ravel(), W.ravel()
