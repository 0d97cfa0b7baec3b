"""Full-grid finite-difference Vlasov-Poisson solver (oracle; test infrastructure only).

The same scheme as :mod:`oracle.vp` written on the dense Nx x Nv array with
no MPS at all: second-order upwind in x (v > 0 backward, v < 0 forward),
centred v derivative with zero gradient at both v ends, RK4 in time (Methods,
"Time Evolution Procedure"; SI "Upwind time evolution").  This is the
"traditional" O(N^K) method the paper compares against (main text, "Cost
Analysis") and the ground truth for the untruncated MPS solver.
"""
from __future__ import annotations

import numpy as np

from .vp import field, grid_steps, species_params


def d_backward_x(f, dx):
    return (1.5 * f - 2.0 * np.roll(f, 1, axis=0) + 0.5 * np.roll(f, 2, axis=0)) / dx


def d_forward_x(f, dx):
    return (-1.5 * f + 2.0 * np.roll(f, -1, axis=0) - 0.5 * np.roll(f, -2, axis=0)) / dx


def d_centered_v_zero_gradient(f, dv):
    g = np.zeros_like(f)
    g[:, 1:-1] = (f[:, 2:] - f[:, :-2]) / (2.0 * dv)
    return g  # ghost node equal to the node inside the boundary: derivative 0 at both ends


def d_second_v_zero_gradient(f, dv):
    g = np.empty_like(f)
    g[:, 1:-1] = (f[:, 2:] - 2.0 * f[:, 1:-1] + f[:, :-2]) / (dv * dv)
    g[:, 0] = 2.0 * (f[:, 1] - f[:, 0]) / (dv * dv)      # ghost f_{-1} = f_1
    g[:, -1] = 2.0 * (f[:, -2] - f[:, -1]) / (dv * dv)   # ghost f_N = f_{N-2}
    return g


def dougherty(f, v, dv, nu, u, vth):
    """nu d/dv [(v - u) f + vth^2 df/dv] (Methods, "Collision Operator") with
    u, vth the species' drift and thermal speed: centred drag, three-point
    diffusion, zero-gradient ghosts on both."""
    return nu * (d_centered_v_zero_gradient((v - u)[None, :] * f, dv) + vth * vth * d_second_v_zero_gradient(f, dv))


def rhs(f, layout):
    dx, dv = grid_steps(layout)
    v = layout.v()
    vp = np.where(v > 0, v, 0.0)[None, :]
    vm = np.where(v > 0, 0.0, v)[None, :]
    rho = f.sum(axis=1) * dv
    E, we = field(rho, dx)
    out = -vp * d_backward_x(f, dx) - vm * d_forward_x(f, dx) + E[:, None] * d_centered_v_zero_gradient(f, dv)
    return out, we, rho


def rk4_step(f, layout, dt):
    k1, we, rho = rhs(f, layout)
    k2, _, _ = rhs(f + 0.5 * dt * k1, layout)
    k3, _, _ = rhs(f + 0.5 * dt * k2, layout)
    k4, _, _ = rhs(f + dt * k3, layout)
    return f + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4), we, rho


def run(f0, layout, dt, nsteps):
    """Returns (f(T), times, field energy, mass) sampled before each step."""
    f = np.array(f0, dtype=np.float64)
    dx, _ = grid_steps(layout)
    ts, wes, masses = [], [], []
    for n in range(nsteps):
        f_new, we, rho = rk4_step(f, layout, dt)
        ts.append(n * dt)
        wes.append(we)
        masses.append(float(rho.sum()) * dx)
        f = f_new
    return f, np.array(ts), np.array(wes), np.array(masses)


def boundary_flux(f, layout):
    """d/dt of the mass  sum f dx dv  for the scheme above.

    The upwind x terms telescope to zero (periodic); the centred v term
    leaves only the four end nodes: dx sum_i E_i c1 (f_{i,N-1} + f_{i,N-2}
    - f_{i,0} - f_{i,1}) with c1 = 1/2 (interior sum telescopes).  Used by
    the mass-conservation test.
    """
    dx, dv = grid_steps(layout)
    rho = f.sum(axis=1) * dv
    E, _ = field(rho, dx)
    # sum_{j=1}^{N-2} (f_{j+1} - f_{j-1}) / (2 dv) * dv = (f_{N-1} + f_{N-2} - f_0 - f_1) / 2
    s = 0.5 * (f[:, -1] + f[:, -2] - f[:, 0] - f[:, 1])
    return dx * float(np.sum(E * s))


def fit_rate(ts, wes, t0, t1):
    """Slope/2 of a line through log W_E at its local maxima in [t0, t1]."""
    ts, wes = np.asarray(ts), np.asarray(wes)
    idx = [i for i in range(1, len(wes) - 1) if wes[i] >= wes[i - 1] and wes[i] > wes[i + 1] and t0 <= ts[i] <= t1]
    if len(idx) < 2:
        raise ValueError("not enough maxima to fit")
    p = np.polyfit(ts[idx], np.log(wes[idx]), 1)
    return 0.5 * p[0]


def multi_rhs(fs, layouts, species):
    """Several species sharing E (see oracle.vp.multi_rk4_step): the field
    from -sum_s q_s rho_s, species s advanced with E scaled by -q_s / m_s."""
    dx, _ = grid_steps(layouts[0])
    rhos = []
    for f, lay in zip(fs, layouts):
        _, dv = grid_steps(lay)
        rhos.append(f.sum(axis=1) * dv)
    net = -sum(species_params(sp)[0] * r for sp, r in zip(species, rhos))
    E, we = field(net, dx)
    out = []
    for f, lay, sp in zip(fs, layouts, species):
        q, m, nu, u, vth = species_params(sp)
        _, dv = grid_steps(lay)
        v = lay.v()
        vp = np.where(v > 0, v, 0.0)[None, :]
        vm = np.where(v > 0, 0.0, v)[None, :]
        d = (-vp * d_backward_x(f, dx) - vm * d_forward_x(f, dx)
             + (-q / m) * E[:, None] * d_centered_v_zero_gradient(f, dv))
        if nu:
            d = d + dougherty(f, v, dv, nu, u, vth)
        out.append(d)
    return out, we, rhos


def multi_rk4_step(fs, layouts, species, dt):
    k1, we, rhos = multi_rhs(fs, layouts, species)
    k2, _, _ = multi_rhs([f + 0.5 * dt * k for f, k in zip(fs, k1)], layouts, species)
    k3, _, _ = multi_rhs([f + 0.5 * dt * k for f, k in zip(fs, k2)], layouts, species)
    k4, _, _ = multi_rhs([f + dt * k for f, k in zip(fs, k3)], layouts, species)
    new = [f + dt / 6.0 * (a + 2 * b + 2 * c + d) for f, a, b, c, d in zip(fs, k1, k2, k3, k4)]
    return new, we, rhos
