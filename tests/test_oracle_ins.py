"""Pins of the oracle's INS pieces (Sections 2.1-2.3)."""
import numpy as np
import pytest

from dg_inputs import jittered_grid
from dg_inputs.fields import kovasznay
from dg_inputs.mesh import ins_pressure_tags, rotate_local_vertices
from oracle.ins import LSERK_A, LSERK_B, LSERK_C, InsOracle, lserk_integrate
from oracle.sipdg import Sipdg


def _ins(n, N, rotate=None, box=(-0.5, 1.0, -0.5, 1.5), sides=(1, 1, 1, 1)):
    m = jittered_grid(n, n, box=box, jitter=0.1, seed=0, bc_sides=sides)
    if rotate is not None:
        m = rotate_local_vertices(m, rotate)
    mp = ins_pressure_tags(m, dirichlet_sides=(1,))
    Su = Sipdg(m.VX, m.VY, m.EToV, m.bc, N)
    Sp = Sipdg(mp.VX, mp.VY, mp.EToV, mp.bc, N)
    return InsOracle(Su, Sp)


def test_lserk_fourth_order():
    """y' = i w y: the global error falls by ~2^4 per halving of the step."""
    w = 3.0
    errs = []
    for nsteps in (20, 40, 80):
        y = lserk_integrate(lambda t, y: 1j * w * y, np.array([1.0 + 0j]), 0.0, 2.0 / nsteps, nsteps)
        errs.append(abs(y[0] - np.exp(2j * w)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8), rates
    assert LSERK_C[0] == 0.0 and np.all(np.diff(LSERK_C) > 0) and LSERK_C[-1] < 1.0
    # quadrature conditions: y' = t^k integrates exactly for k <= 3 in one step
    h = 0.5
    for k in range(4):
        y = lserk_integrate(lambda t, y: np.full_like(y, t ** k), np.zeros(1), 0.0, h, 1)
        assert abs(y[0] - h ** (k + 1) / (k + 1)) < 1e-15, k
    # y' = y: one step reproduces exp(h) through the h^4 term (error ~ h^5)
    y = lserk_integrate(lambda t, y: y, np.ones(1), 0.0, 0.1, 1)
    assert abs(y[0] - np.exp(0.1)) < 2e-7
    assert len(LSERK_A) == len(LSERK_B) == 5


def _poly(N, seed):
    """Random polynomial of total degree N with its x and y derivatives."""
    c = np.random.default_rng(seed).standard_normal((N + 1, N + 1))
    terms = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    f = lambda x, y: sum(c[a, b] * x ** a * y ** b for a, b in terms)
    fx = lambda x, y: sum(c[a, b] * a * x ** (a - 1) * y ** b for a, b in terms if a > 0)
    fy = lambda x, y: sum(c[a, b] * b * x ** a * y ** (b - 1) for a, b in terms if b > 0)
    return f, fx, fy


# velocity Dirichlet everywhere, or Neumann at the outflow x = 1 (u* = u- there)
SIDES = [(1, 1, 1, 1), (1, 2, 1, 1)]


@pytest.mark.parametrize("sides", SIDES)
@pytest.mark.parametrize("N", [2, 4, 6])
def test_gradient_and_divergence_exact_on_polynomials(N, sides):
    """For continuous polynomials with matching boundary data every jump
    vanishes, so G p = grad p and D.U = div U at the nodes."""
    O = _ins(3, N, rotate=N, sides=sides)
    x, y = O.Su.x, O.Su.y
    f, fx, fy = _poly(N, 1)
    p = f(x, y)
    G = O.to_strong(O.weak_grad(p, p))
    scale = max(1.0, np.abs(fx(x, y)).max())
    assert np.abs(G[0] - fx(x, y)).max() < 1e-11 * scale * N ** 2
    assert np.abs(G[1] - fy(x, y)).max() < 1e-11 * scale * N ** 2
    g, gx, gy = _poly(N, 2)
    U = np.stack([f(x, y), g(x, y)])
    D = O.to_strong(O.weak_div(U, U))
    assert np.abs(D - (fx(x, y) + gy(x, y))).max() < 1e-11 * scale * N ** 2


@pytest.mark.parametrize("sides", SIDES)
@pytest.mark.parametrize("N", [1, 3, 5])
def test_advection_exact_on_continuous_linear_field(N, sides):
    """For a continuous linear velocity with matching boundary data the LLF
    jumps vanish and N~(U, U)_c = div(U U_c) exactly (degree <= 1 <= N)."""
    O = _ins(3, N, rotate=2, sides=sides)
    x, y = O.Su.x, O.Su.y
    U = np.stack([1.0 + x + 2 * y, 3.0 - y + 0.5 * x])
    u, v = U
    # div(U u) = u_x u + u u_x ... written out: d(u u)/dx + d(v u)/dy
    div_uu = 2 * u * 1.0 + (v * 2.0 + u * (-1.0))
    # d(u v)/dx + d(v v)/dy = u_x v + u v_x + 2 v v_y
    div_uv = 1.0 * v + u * 0.5 + 2 * v * (-1.0)
    rhs = O.advection(U, U, U)
    assert np.abs(-rhs[0] - div_uu).max() < 1e-10 * 50
    assert np.abs(-rhs[1] - div_uv).max() < 1e-10 * 50


def test_kovasznay_step_stays_near_exact():
    """One split step from the exact Kovasznay state (nu = 1/40, dt = 0.01,
    4 substeps) stays at the discretisation-error level and keeps D.U small."""
    O = _ins(8, 4, rotate=1)
    nu, fu, fv, fp = kovasznay(40.0)
    x, y = O.Su.x, O.Su.y
    U0 = np.stack([fu(x, y), fv(x, y)])
    P0 = fp(x, y)
    st = dict(U=U0.copy(), Uold=U0.copy(), P=P0.copy(), n=0)
    st, mid = O.step(st, 0.01, nu, 4, U0, P0)
    st, mid = O.step(st, 0.01, nu, 4, U0, P0)
    err_u = np.abs(st["U"] - U0).max() / np.abs(U0).max()
    err_p = np.abs(st["P"] - P0).max()
    assert err_u < 5e-3, err_u
    assert err_p < 5e-2, err_p
    div = np.linalg.norm(O.to_strong(O.weak_div(st["U"], U0)))
    div0 = np.linalg.norm(O.to_strong(O.weak_div(U0 + 0.01, U0)))
    assert div < div0


def test_second_order_in_time_self_convergence():
    """Section 4 reports second-order temporal accuracy for BDF2/EXT2 with the
    first-order pressure increment. With steady boundary data the study needs
    no closed form: from one developed state, runs with dt, dt/2, dt/4, dt/8
    to a common time differ by C dt^2, so successive differences fall by ~4.

    Flow: the Kovasznay data plus a divergence-free bump (stream function
    0.2 X^2 Y^2, vanishing with its gradient on the box), velocity Dirichlet on
    three sides and Neumann at the outflow x = 1 where the pressure is
    Dirichlet (the open boundary of the paper's Taylor-vortex set-up); 40 steps
    of dt = 0.0025 first, so that the pressure is consistent with the flow.
    Measured ratios at the finest pair: velocity 3.93 (rms), 3.72 (max),
    pressure 4.0 (rms). Planted mistakes in the step fall below the bounds: a
    constant advecting velocity 3.07, U^{n-1} advected over one step instead of
    two 2.0, beta_1 = +1/2 diverges."""
    N, Ns, T = 4, 4, 0.05
    m = jittered_grid(3, 3, box=(-0.5, 1.0, -0.5, 1.5), jitter=0.1, seed=0, bc_sides=(1, 2, 1, 1))
    mp = ins_pressure_tags(m, dirichlet_sides=(1,))
    O = InsOracle(Sipdg(m.VX, m.VY, m.EToV, m.bc, N), Sipdg(mp.VX, mp.VY, mp.EToV, mp.bc, N))
    nu, fu, fv, fp = kovasznay(40.0)
    x, y = O.Su.x, O.Su.y
    gU, gP = np.stack([fu(x, y), fv(x, y)]), fp(x, y)
    X, Xp = (x + 0.5) * (1.0 - x), 0.5 - 2.0 * x
    Y, Yp = (y + 0.5) * (1.5 - y), 1.0 - 2.0 * y
    U = gU + 0.2 * np.stack([2.0 * X ** 2 * Y * Yp, -2.0 * X * Xp * Y ** 2])
    st = dict(U=U, Uold=U.copy(), P=gP.copy(), n=0)
    for _ in range(40):
        st, _ = O.step(st, 0.0025, nu, Ns, gU, gP)
    start = st
    runs = []
    for dt in (0.005, 0.0025, 0.00125, 0.000625):
        st = dict(U=start["U"].copy(), Uold=start["U"].copy(), P=start["P"].copy(), n=0)
        for _ in range(int(round(T / dt))):
            st, _ = O.step(st, dt, nu, Ns, gU, gP)
        runs.append(st)
    rms = lambda z: np.sqrt(np.mean(z * z))
    dU = [runs[i]["U"] - runs[i + 1]["U"] for i in range(3)]
    dP = [runs[i]["P"] - runs[i + 1]["P"] for i in range(3)]
    ru = [rms(dU[i]) / rms(dU[i + 1]) for i in range(2)]
    assert np.all(np.diff([rms(d) for d in dU]) < 0) and np.all(np.diff([rms(d) for d in dP]) < 0)
    assert ru[0] > 2.8 and ru[1] > 3.5, ru
    assert np.abs(dU[1]).max() / np.abs(dU[2]).max() > 3.3
    assert rms(dP[1]) / rms(dP[2]) > 3.0


@pytest.mark.parametrize("N", [2, 3, 4])
def test_advection_converges_at_design_rate_on_smooth_field(N):
    """-N~(U, U) of the smooth divergence-free Kovasznay field (exact boundary
    data, all faces carrying jumps of the interpolant) against the closed form
    -U.grad U on 6x6, 12x12 and 24x24 grids: the L2 error of this DG
    derivative falls like h^N (measured rates at the finest pair 1.94, 2.85,
    3.97 for N = 2, 3, 4). A face term dropped, or the central average without
    its 1/2, makes the error grow under refinement."""
    Re = 40.0
    lam = Re / 2.0 - np.sqrt(Re * Re / 4.0 + 4.0 * np.pi ** 2)

    def closed_form(x, y):
        E, c, s = np.exp(lam * x), np.cos(2 * np.pi * y), np.sin(2 * np.pi * y)
        u, v = 1.0 - E * c, lam / (2 * np.pi) * E * s
        ux, uy = -lam * E * c, 2 * np.pi * E * s
        vx, vy = lam * lam / (2 * np.pi) * E * s, lam * E * c
        return np.stack([u, v]), np.stack([u * ux + v * uy, u * vx + v * vy])

    errs = []
    for n in (6, 12, 24):
        O = _ins(n, N, rotate=1)
        U, ugradu = closed_form(O.Su.x, O.Su.y)
        e = O.advection(U, U, U) + ugradu
        errs.append(np.sqrt(sum((O.Su.mass_apply(e[c]) * e[c]).sum() for c in range(2))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > N - 0.3 and rates[0] > N - 0.5, rates


def _taylor(n, N, nu):
    from dg_inputs.fields import taylor_vortex
    m = jittered_grid(n, n, box=(-1.0, 1.0, -1.0, 1.0), jitter=0.1, seed=0, bc_sides=(1, 1, 1, 1))
    mp = ins_pressure_tags(m, dirichlet_sides=(1,))
    O = InsOracle(Sipdg(m.VX, m.VY, m.EToV, m.bc, N), Sipdg(mp.VX, mp.VY, mp.EToV, mp.bc, N))
    fu, fv, fp = taylor_vortex(nu)
    x, y = O.Su.x, O.Su.y
    return O, (lambda t: np.stack([fu(x, y, t), fv(x, y, t)])), (lambda t: fp(x, y, t))


def test_time_dependent_data_path_with_constant_data_equals_steady_path():
    """Boundary data given as functions of time that do not change reproduce
    the steady-data step exactly (the increment's Dirichlet data is zero)."""
    O, gU, gP = _taylor(3, 4, 0.05)
    U0, P0 = gU(0.0), gP(0.0)
    runs = []
    for data in ((U0, P0), (lambda t: U0, lambda t: P0)):
        st = dict(U=U0.copy(), Uold=U0.copy(), P=P0.copy(), n=0)
        for _ in range(2):
            st, _ = O.step(st, 0.01, 0.05, 4, *data)
        runs.append(st)
    assert np.array_equal(runs[0]["U"], runs[1]["U"]) and np.array_equal(runs[0]["P"], runs[1]["P"])


def test_taylor_vortex_second_order_in_time():
    """Section 4.1's Taylor vortex (decaying Taylor-Green flow, exact in time):
    velocity and pressure Dirichlet data taken from the closed form at the
    times each stage needs them, N = 6 on a jittered 4x4 grid of [-1, 1]^2
    (spatial error far below the temporal one), nu = 0.05, T = 0.2 with
    dt = 0.04, 0.02, 0.01. The velocity error at T falls at second order:
    measured rates 1.65 and 1.86. Planted mistake: data one step late (the
    solves taking g(t^n) for g(t^{n+1})) gives rates 1.10 and 0.89."""
    nu, T = 0.05, 0.2
    O, gU, gP = _taylor(4, 6, nu)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        st = dict(U=gU(0.0), Uold=gU(0.0), P=gP(0.0), n=0)
        for _ in range(int(round(T / dt))):
            st, _ = O.step(st, dt, nu, 4, gU, gP)
        errs.append(np.abs(st["U"] - gU(T)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3 and rates[-1] > 1.7 and rates[0] > 1.4, (errs, rates)
