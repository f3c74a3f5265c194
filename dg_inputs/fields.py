"""Seeded vectors and closed-form data functions (inputs only)."""
import numpy as np


def uniform_field(shape, seed, lo=-1.0, hi=1.0):
    """U(lo, hi) float64 array of the given shape from default_rng(seed)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def fourier_rhs_coeffs(seed, modes=16, kmax=8):
    """Amplitudes and wavenumbers of a sum of sin(kx pi x) sin(ky pi y) modes.

    Returns (a, kx, ky): a ~ N(0,1), kx, ky ~ U{1..kmax}, `modes` of each.
    """
    rng = np.random.default_rng(seed)
    kx = rng.integers(1, kmax + 1, size=modes)
    ky = rng.integers(1, kmax + 1, size=modes)
    a = rng.standard_normal(modes)
    return a, kx, ky


def fourier_eval(coeffs, x, y):
    a, kx, ky = coeffs
    out = np.zeros_like(np.asarray(x, dtype=np.float64))
    for am, kxm, kym in zip(a, kx, ky):
        out = out + am * np.sin(kxm * np.pi * x) * np.sin(kym * np.pi * y)
    return out


def manufactured(name):
    """Closed-form solutions u and their -Laplacians f, as callables of (x, y)."""
    if name == "sin_pi_x_sin_pi_y":
        u = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
        f = lambda x, y: 2.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y)
    elif name == "sin_2pi_x_cos_3pi_y":
        u = lambda x, y: np.sin(2 * np.pi * x) * np.cos(3 * np.pi * y)
        f = lambda x, y: 13.0 * np.pi ** 2 * np.sin(2 * np.pi * x) * np.cos(3 * np.pi * y)
    else:
        raise KeyError(name)
    return u, f


def kovasznay(Re=40.0):
    """Kovasznay's steady closed-form Navier-Stokes solution (Kovasznay 1948):
    nu = 1/Re, l = Re/2 - sqrt(Re^2/4 + 4 pi^2),
    u = 1 - e^{l x} cos 2 pi y, v = l/(2 pi) e^{l x} sin 2 pi y, p = (1 - e^{2 l x})/2.
    Returns (nu, u, v, p) with u, v, p callables of (x, y)."""
    lam = Re / 2.0 - np.sqrt(Re * Re / 4.0 + 4.0 * np.pi ** 2)
    u = lambda x, y: 1.0 - np.exp(lam * x) * np.cos(2 * np.pi * y)
    v = lambda x, y: lam / (2 * np.pi) * np.exp(lam * x) * np.sin(2 * np.pi * y)
    p = lambda x, y: 0.5 * (1.0 - np.exp(2 * lam * x))
    return 1.0 / Re, u, v, p


def taylor_vortex(nu):
    """The decaying Taylor-Green vortex, a time-dependent closed-form
    Navier-Stokes solution: F(t) = exp(-2 pi^2 nu t),
    u = -cos(pi x) sin(pi y) F, v = sin(pi x) cos(pi y) F,
    p = -(cos 2 pi x + cos 2 pi y) F^2 / 4.
    Returns (u, v, p), callables of (x, y, t)."""
    F = lambda t: np.exp(-2.0 * np.pi ** 2 * nu * t)
    u = lambda x, y, t: -np.cos(np.pi * x) * np.sin(np.pi * y) * F(t)
    v = lambda x, y, t: np.sin(np.pi * x) * np.cos(np.pi * y) * F(t)
    p = lambda x, y, t: -0.25 * (np.cos(2 * np.pi * x) + np.cos(2 * np.pi * y)) * F(t) ** 2
    return u, v, p
