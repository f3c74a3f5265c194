"""Pins of the per-face penalty (Section 2.1, Eq. PenaltyParameter) and of the
Warp & Blend blend parameters the node set uses (Section 2.1, after Warburton
2006): values fixed by a hand-worked example and by the optimality that
defines the tabulated parameters, not by the oracle's own formulas."""
import os

import numpy as np
import pytest

import oracle.basis as basis
from oracle.sipdg import Sipdg

GOLD = os.path.join(os.path.dirname(__file__), "golden", "penalty_two_triangles.txt")


def _golden():
    out = {}
    with open(GOLD) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _two_triangles(tag):
    VX = np.array([0.0, 1.0, 0.0, 2.0])
    VY = np.array([0.0, 0.0, 1.0, 2.0])
    EToV = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    bc = np.array([[tag, 0, tag], [tag, tag, 0]], dtype=np.int8)
    return VX, VY, EToV, bc


def _indicator_forms(S):
    A = S.assemble().toarray()
    one = np.zeros((2, S.K * S.Np))
    one[0, :S.Np] = 1.0
    one[1, S.Np:] = 1.0
    return one[0] @ A @ one[0], one[1] @ A @ one[1], one[0] @ A @ one[1], one[1] @ A @ one[0]


def test_penalty_values_match_hand_worked_example():
    g = _golden()
    S = Sipdg(*_two_triangles(1), 2)
    want = np.array([[g["tau_A0"], g["tau_A1"], g["tau_A2"]], [g["tau_B0"], g["tau_B1"], g["tau_B2"]]])
    assert np.abs(S.tau - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("tag,prefix", [(1, "dir"), (2, "neu")])
def test_penalty_enters_operator_as_hand_worked(tag, prefix):
    """Piecewise-constant indicators see only the penalty term of Eq. ellipticOp1;
    their quadratic forms are the hand-computed sums of tau |face|."""
    g = _golden()
    aa, bb, ab, ba = _indicator_forms(Sipdg(*_two_triangles(tag), 2))
    assert abs(aa - g[prefix + "_AA"]) <= 1e-11
    assert abs(bb - g[prefix + "_BB"]) <= 1e-11
    assert abs(ab - g[prefix + "_AB"]) <= 1e-11
    assert abs(ba - g[prefix + "_AB"]) <= 1e-11


@pytest.mark.parametrize("plant", ["min", "no_half", "boundary_uses_element_0"])
def test_planted_penalty_mistakes_fail_the_example(plant):
    """A mistake planted in the oracle's penalty (on the CPU) breaks the pin."""
    g = _golden()
    S = Sipdg(*_two_triangles(1), 2)
    geo = S.geo
    c = 6.0
    inv_h = geo.face_len / geo.area[:, None]
    nb = np.where(geo.EToE >= 0, geo.EToE, 0)
    inv_h_nb = geo.face_len / geo.area[nb]
    if plant == "min":
        S.tau = c * np.where(geo.EToE >= 0, np.minimum(inv_h, inv_h_nb), inv_h)
    elif plant == "no_half":
        S.tau = 2.0 * S.tau
    else:
        S.tau = c * np.maximum(inv_h, inv_h_nb)  # neighbour index 0 used on boundary faces
    aa, bb, _, _ = _indicator_forms(S)
    assert abs(aa - g["dir_AA"]) > 1.0 or abs(bb - g["dir_BB"]) > 1.0


# --------------------------------------------------------------- blend parameters
_M = 240
_grid = np.array([(-1 + 2 * i / _M, -1 + 2 * j / _M) for j in range(_M + 1) for i in range(_M + 1 - j)])


def _nodes(N, alpha):
    saved = basis.ALPHA_OPT[N - 1]
    basis.ALPHA_OPT[N - 1] = alpha
    try:
        return basis.warp_blend_nodes(N)
    finally:
        basis.ALPHA_OPT[N - 1] = saved


def _lebesgue(N, alpha):
    """Lebesgue constant max_x sum_i |l_i(x)| of the degree-N node set: grid
    maximum, refined by a local search from the largest grid values."""
    from scipy.optimize import minimize
    r, s = _nodes(N, alpha)
    Vinv = np.linalg.inv(basis.vandermonde(N, r, s))

    def leb(x, y):
        return np.abs(basis.vandermonde(N, np.atleast_1d(x), np.atleast_1d(y)) @ Vinv).sum(-1)

    v = leb(_grid[:, 0], _grid[:, 1])
    best = v.max()
    for k in np.argsort(v)[-6:]:
        def f(z):
            x, y = z
            if x < -1 or y < -1 or x + y > 0:
                return 0.0
            return -leb(x, y)[0]
        res = minimize(f, _grid[k], method="Nelder-Mead", options=dict(xatol=1e-9, fatol=1e-12))
        best = max(best, -res.fun)
    return best


def test_blend_parameter_is_irrelevant_at_degree_3():
    """At N = 3 the only interior node is the centroid, fixed by symmetry: the
    node set must not depend on alpha (so its table entry needs no pin)."""
    r0, s0 = _nodes(3, 0.0)
    r1, s1 = _nodes(3, 1.4152)
    assert np.abs(r0 - r1).max() < 1e-14 and np.abs(s0 - s1).max() < 1e-14


@pytest.mark.parametrize("N,delta", [(5, 0.02), (6, 0.05), (7, 0.05), (8, 0.05), (9, 0.05), (10, 0.05)])
def test_tabulated_blend_parameter_minimises_lebesgue_constant(N, delta):
    """The tabulated alpha(N) is the minimiser of the node set's Lebesgue
    constant (the optimisation that defines the table): moving it either way
    raises the constant. A transposed or mistyped entry fails this."""
    a = basis.ALPHA_OPT[N - 1]
    l0 = _lebesgue(N, a)
    assert l0 < _lebesgue(N, a - delta) - 1e-4
    assert l0 < _lebesgue(N, a + delta) - 1e-4


def test_swapped_blend_parameters_fail_the_pin():
    """Planted mistake: the N = 6 entry replaced by the N = 7 one."""
    wrong = basis.ALPHA_OPT[6]
    assert _lebesgue(6, wrong) > _lebesgue(6, basis.ALPHA_OPT[5]) + 1e-3


def test_blend_parameter_at_degree_4_is_near_optimal():
    """At N = 4 the Lebesgue constant is nearly flat in alpha; the tabulated
    value lies within 1e-3 of the best constant over [0, 0.3]."""
    best = min(_lebesgue(4, a) for a in np.linspace(0.0, 0.3, 7))
    assert _lebesgue(4, basis.ALPHA_OPT[3]) <= best + 1e-3


@pytest.mark.parametrize("N", [1, 2, 4])
def test_penalty_keeps_the_form_coercive_with_margin(N):
    """Eq. PenaltyParameter's tau = (N+1)(N+2)/2 max(1/h) keeps the SIPDG form
    positive definite at half of it too, and the form loses definiteness at a
    quarter: the constant is of the size coercivity needs, not merely positive."""
    from dg_inputs import jittered_grid
    m = jittered_grid(4, 4, jitter=0.1, seed=1)
    S = Sipdg(m.VX, m.VY, m.EToV, m.bc, N)
    t0 = S.tau.copy()

    def lam_min(scale):
        S.tau = t0 * scale
        A = S.assemble().toarray()
        return np.linalg.eigvalsh(0.5 * (A + A.T)).min()

    assert lam_min(1.0) > 0 and lam_min(0.5) > 0
    assert lam_min(0.25) < 0
