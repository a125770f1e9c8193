"""Linear electrostatic plasma theory used to pin the oracle's whole step.

Dielectric function of drifting Maxwellian beams (normalised units:
omega_p = 1 for unit density, charge -1, mass 1, Poisson constant 1):

    eps(omega, k) = 1 - sum_b n_b q_b^2 / (m_b 2 k^2 vth_b^2) Z'(zeta_b),
    zeta_b = (omega - k u_b) / (sqrt(2) k vth_b),   Z'(z) = -2 (1 + z Z(z)),

with Z the plasma dispersion function, Z(z) = i sqrt(pi) w(z) (Faddeeva w,
scipy.special.wofz).  Roots are found by Newton iteration in the complex plane.
"""
import numpy as np
from scipy.special import wofz


def Z(z):
    return 1j * np.sqrt(np.pi) * wofz(z)


def Zp(z):
    return -2.0 * (1.0 + z * Z(z))


def eps(omega, k, beams):
    """beams: iterable of (n, u, vth, q, m)."""
    s = 1.0 + 0j
    for n, u, vth, q, m in beams:
        zeta = (omega - k * u) / (np.sqrt(2.0) * k * vth)
        s -= n * q * q / m / (2.0 * k * k * vth * vth) * Zp(zeta)
    return s


def root(k, beams, guess, tol=1e-13, maxit=200):
    w = complex(guess)
    for _ in range(maxit):
        h = 1e-7 * max(1.0, abs(w))
        f = eps(w, k, beams)
        d = (eps(w + h, k, beams) - eps(w - h, k, beams)) / (2 * h)
        dw = f / d
        w -= dw
        if abs(dw) < tol:
            return w
    raise RuntimeError("no convergence")


def landau_root(k):
    """Least-damped Langmuir root of one Maxwellian (v_th = 1)."""
    guess = np.sqrt(1 + 3 * k * k) - 0.05j
    return root(k, [(1.0, 0.0, 1.0, -1.0, 1.0)], guess)


def two_stream_root(k, u=3.0, vth=1.0):
    """Purely growing root of two equal counter-drifting electron beams."""
    beams = [(0.5, u, vth, -1.0, 1.0), (0.5, -u, vth, -1.0, 1.0)]
    return root(k, beams, 0.0 + 0.3j)


def peaks(t, a):
    """Local maxima of a sampled positive signal (strict, interior)."""
    idx = [i for i in range(1, len(a) - 1) if a[i] > a[i - 1] and a[i] >= a[i + 1]]
    return np.asarray(idx, dtype=int)


def mode_amplitude(E, m):
    N = E.size
    i = np.arange(N)
    c = np.sum(E * np.exp(-2j * np.pi * m * i / N))
    return 2.0 * abs(c) / N
