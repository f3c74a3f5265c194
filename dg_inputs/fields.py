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
