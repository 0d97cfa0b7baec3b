"""Linear electrostatic dispersion relation for Maxwellian beams (oracle; tests only).

Not from the paper: standard kinetic plasma theory, used to pin the physics of
the dense finite-difference solver (linear Landau damping, two-stream growth).
Normalised units (Debye length, electron plasma frequency):

    eps(omega, k) = 1 + sum_b n_b / (k^2 vth_b^2) [1 + zeta_b Z(zeta_b)],
    zeta_b = (omega - k u_b) / (sqrt(2) k vth_b),

with the plasma dispersion function Z(zeta) = i sqrt(pi) w(zeta) (Faddeeva w,
valid for all Im zeta).
"""
from __future__ import annotations

import cmath
import math

from scipy.special import wofz


def Z(zeta):
    return 1j * math.sqrt(math.pi) * wofz(zeta)


def epsilon(omega, k, beams):
    """beams: iterable of (density, drift, thermal speed)."""
    out = 1.0 + 0.0j
    for (nb, ub, vth) in beams:
        zeta = (omega - k * ub) / (math.sqrt(2.0) * k * vth)
        out += nb / (k * k * vth * vth) * (1.0 + zeta * Z(zeta))
    return out


def root(k, beams, guess, tol=1e-12, maxit=200):
    """Newton iteration on eps(omega) = 0 with a centred complex derivative."""
    w = complex(guess)
    for _ in range(maxit):
        f = epsilon(w, k, beams)
        h = 1e-7 * max(1.0, abs(w))
        d = (epsilon(w + h, k, beams) - epsilon(w - h, k, beams)) / (2 * h)
        step = f / d
        w -= step
        if abs(step) < tol * max(1.0, abs(w)):
            return w
    raise RuntimeError("dispersion root did not converge")


def landau_root(k, guess=None):
    g = guess if guess is not None else cmath.sqrt(1 + 3 * k * k) - 0.1j
    return root(k, [(1.0, 0.0, 1.0)], g)


def two_stream_root(k, u=3.0, vth=1.0, guess=0.3j):
    return root(k, [(0.5, u, vth), (0.5, -u, vth)], guess)


def buneman_root(k, mass_ratio, v0, vth_i, vth_e=1.0, guess=None):
    """Electrons drifting at v0 through ions of mass mass_ratio (charge 1):
    each species enters eps with weight omega_ps^2 = n q^2 / m."""
    g = guess if guess is not None else complex(0.5 * (1.0 / mass_ratio) ** (1.0 / 3.0),
                                                0.8 * (0.5 / mass_ratio) ** (1.0 / 3.0))
    return root(k, [(1.0, v0, vth_e), (1.0 / mass_ratio, 0.0, vth_i)], g)
