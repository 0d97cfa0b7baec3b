"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no arithmetic of the MPS method itself: it only samples the
initial distribution functions of the test problems on the phase-space grid and
draws seeded random numbers.  Both sides read the same grid convention:

* x is periodic with the right end excluded: ``x_i = xmin + i*dx``,
  ``dx = (xmax - xmin) / Nx``.
* v is vertex-centred and includes both ends: ``v_j = vmin + j*dv``,
  ``dv = (vmax - vmin) / (Nv - 1)`` (zero-gradient boundaries act on the end
  nodes, Methods: "Time Evolution Procedure").

Arrays are row-major ``f[ix, iv]`` with ``Nx = 2**nx`` rows and ``Nv = 2**nv``
columns.  The initial conditions follow the Methods section (Landau damping)
and the standard two-stream and bump-on-tail set-ups with one electron species
against a fixed neutralising background.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEQ = 0          # S1: x bits coarse->fine, then v bits coarse->fine
INTERLEAVED = 1  # IF: x_1, v_1, x_2, v_2, ... (coarse first)
SEQ_S2 = 2       # S2: x bits fine->coarse, then v bits coarse->fine
SEQ_S3 = 3       # S3: x bits coarse->fine, then v bits fine->coarse
GROUPED = 4      # IG: the IF site order with each (x_j, v_j) pair one d = 4 site (nx == nv)


@dataclasses.dataclass(frozen=True)
class Layout:
    nx: int
    nv: int
    xmin: float
    xmax: float
    vmin: float
    vmax: float
    mapping: int = SEQ

    @property
    def Nx(self) -> int:
        return 1 << self.nx

    @property
    def Nv(self) -> int:
        return 1 << self.nv

    @property
    def n(self) -> int:
        return self.nx + self.nv

    def x(self) -> np.ndarray:
        return self.xmin + np.arange(self.Nx) * ((self.xmax - self.xmin) / self.Nx)

    def v(self) -> np.ndarray:
        return self.vmin + np.arange(self.Nv) * ((self.vmax - self.vmin) / (self.Nv - 1))


def maxwellian(v, vth=1.0, u=0.0):
    return np.exp(-((v - u) ** 2) / (2 * vth * vth)) / math.sqrt(2 * math.pi * vth * vth)


def landau(layout: Layout, amp=0.01, k=0.5):
    """f0 = (1 + A cos kx) exp(-v^2/2)/sqrt(2 pi)."""
    x, v = layout.x(), layout.v()
    return np.outer(1.0 + amp * np.cos(k * x), maxwellian(v))


def nonlinear_landau(layout: Layout):
    """Landau initial condition at amplitude 0.5 (k = 0.5): the nonlinear case."""
    return landau(layout, amp=0.5, k=0.5)


def buneman_layouts(nx, nv_e, nv_i, k=0.1, mass_ratio=25.0, mapping=SEQ):
    """Electron and ion grids of the Buneman problem (Methods, "Buneman
    instability"): x in [-pi/k, pi/k); electron v in +-6 omega_pe / k; ion v in
    +-50 v_th,i with v_th,i = sqrt(T_i / m_i) at T_i = T_e."""
    vth_i = 1.0 / math.sqrt(mass_ratio)
    lay_e = Layout(nx, nv_e, -math.pi / k, math.pi / k, -6.0 / k, 6.0 / k, mapping)
    lay_i = Layout(nx, nv_i, -math.pi / k, math.pi / k, -50.0 * vth_i, 50.0 * vth_i, mapping)
    return lay_e, lay_i


def buneman(lay_e: Layout, lay_i: Layout, amp=1e-3, k=0.1, mass_ratio=25.0):
    """(f_e, f_i): ions a Maxwellian at rest, uniform in x; electrons a
    Maxwellian drifting at v0 = omega_pe / k, perturbed by (1 + A cos kx)."""
    vth_i = 1.0 / math.sqrt(mass_ratio)
    f_i = np.outer(np.ones(lay_i.Nx), maxwellian(lay_i.v(), vth_i))
    f_e = np.outer(1.0 + amp * np.cos(k * lay_e.x()), maxwellian(lay_e.v(), 1.0, 1.0 / k))
    return f_e, f_i


def two_stream(layout: Layout, amp=1e-3, k=0.2, v0=3.0):
    """f0 = (1 + A cos kx) [e^{-(v-v0)^2/2} + e^{-(v+v0)^2/2}] / (2 sqrt(2 pi))."""
    x, v = layout.x(), layout.v()
    h = 0.5 * (maxwellian(v, 1.0, v0) + maxwellian(v, 1.0, -v0))
    return np.outer(1.0 + amp * np.cos(k * x), h)


def bump_on_tail(layout: Layout, amp=1e-3, k=0.3, nb=0.1, vb=4.5, sb=0.5):
    x, v = layout.x(), layout.v()
    h = (1 - nb) * maxwellian(v) + nb * maxwellian(v, sb, vb)
    return np.outer(1.0 + amp * np.cos(k * x), h)


def saturated_two_stream(layout: Layout, modes=32, eps=0.05, k=0.2, v0=3.0, seed=0):
    """Two-stream background plus a seeded broadband perturbation.

    f0 = h(v) [1 + eps * sum_m a_m cos(m k x + phi_m) psi_m(v)], with psi_m a
    Hermite-Gauss shape centred on one of the beams.  With 32 modes the bond
    at the x/v cut needs 65 singular values and the interior bonds are dense,
    so a compression to chi <= 64 keeps every middle bond at the cap: the
    workload of the nonlinear (saturated) phase of the instability.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x, v = layout.x(), layout.v()
    h = 0.5 * (maxwellian(v, 1.0, v0) + maxwellian(v, 1.0, -v0))
    a = rng.uniform(0.3, 1.0, size=modes) / np.arange(1, modes + 1) ** 0.5
    phi = rng.uniform(0, 2 * math.pi, size=modes)
    centre = rng.choice([-v0, v0], size=modes)
    order = rng.integers(0, 4, size=modes)
    width = rng.uniform(0.6, 1.4, size=modes)
    pert = np.zeros((layout.Nx, layout.Nv))
    for m in range(modes):
        s = (v - centre[m]) / width[m]
        psi = np.polynomial.hermite.hermval(s, [0] * order[m] + [1]) * np.exp(-s * s / 2)
        psi = psi / np.max(np.abs(psi))
        pert += a[m] * np.outer(np.cos((m + 1) * k * x + phi[m]), psi)
    return h[None, :] * (1.0 + eps * pert)


def saturated_buneman(lay_e: Layout, lay_i: Layout, modes=32, eps=0.05, k=0.1, mass_ratio=25.0, seed=0):
    """Buneman background (drifting electrons, ions at rest) plus seeded
    broadband perturbations of both species, built like
    :func:`saturated_two_stream`: f_s = h_s(v) [1 + eps_s sum_m a_m cos(m k x +
    phi_m) psi_m(v)], psi_m a Hermite-Gauss shape around the species' drift
    (ions at a fifth of the electron amplitude).  On 512 x 512 grids with 32
    modes both species' middle bonds reach 62-63 at tol = 1e-10: the cost
    profile of the nonlinear phase of the instability at chi = 64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    vth_i = 1.0 / math.sqrt(mass_ratio)
    out = []
    for lay, u, vth, amp in ((lay_e, 1.0 / k, 1.0, eps), (lay_i, 0.0, vth_i, 0.2 * eps)):
        x, v = lay.x(), lay.v()
        a = rng.uniform(0.3, 1.0, size=modes) / np.arange(1, modes + 1) ** 0.5
        phi = rng.uniform(0, 2 * math.pi, size=modes)
        order = rng.integers(0, 4, size=modes)
        width = rng.uniform(0.6, 1.4, size=modes) * vth
        pert = np.zeros((lay.Nx, lay.Nv))
        for m in range(modes):
            s = (v - u) / width[m]
            psi = np.polynomial.hermite.hermval(s, [0] * order[m] + [1]) * np.exp(-s * s / 2)
            psi = psi / np.max(np.abs(psi))
            pert += a[m] * np.outer(np.cos((m + 1) * k * x + phi[m]), psi)
        out.append(maxwellian(v, vth, u)[None, :] * (1.0 + amp * pert))
    return out[0], out[1]


def random_cores(ranks, seed=0, d=2):
    """Random MPS cores with the given bond list ``ranks`` (length n+1, ends 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.standard_normal((ranks[k], d, ranks[k + 1])) / math.sqrt(ranks[k] * d)
            for k in range(len(ranks) - 1)]


def random_vector(n, seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(1 << n)


# Named workloads (grid, initial condition, chi, dt).  dt follows the fixed
# stability rule: CFL_x = vmax*dt/dx <= 0.6 (RK4 with the second-order upwind
# stencil is stable up to 0.696).
WORKLOADS = {
    "landau_64x64": dict(layout=Layout(6, 6, 0.0, 4 * math.pi, -6.0, 6.0, SEQ),
                         ic="landau", chi=64, dt=0.02),
    "two_stream_1024x1024_seq": dict(layout=Layout(10, 10, 0.0, 10 * math.pi, -8.0, 8.0, SEQ),
                                     ic="two_stream", chi=64, dt=0.002),
    "two_stream_1024x1024_int": dict(layout=Layout(10, 10, 0.0, 10 * math.pi, -8.0, 8.0, INTERLEAVED),
                                     ic="two_stream", chi=64, dt=0.002),
    "saturated_two_stream_1024x1024_seq": dict(layout=Layout(10, 10, 0.0, 10 * math.pi, -8.0, 8.0, SEQ),
                                               ic="saturated_two_stream", chi=64, dt=0.002),
    "saturated_two_stream_1024x1024_int": dict(layout=Layout(10, 10, 0.0, 10 * math.pi, -8.0, 8.0, INTERLEAVED),
                                               ic="saturated_two_stream", chi=64, dt=0.002),
    "saturated_two_stream_256x256_seq": dict(layout=Layout(8, 8, 0.0, 10 * math.pi, -8.0, 8.0, SEQ),
                                             ic="saturated_two_stream", chi=32, dt=0.008),
    # 4096 x 4096 (12 + 12 sites): dt = 0.6 dx / vmax
    "nonlinear_landau_4096x4096_seq": dict(layout=Layout(12, 12, 0.0, 4 * math.pi, -6.0, 6.0, SEQ),
                                           ic="nonlinear_landau", chi=128, dt=0.6 * (4 * math.pi / 4096) / 6.0),
    "saturated_two_stream_4096x4096_seq": dict(layout=Layout(12, 12, 0.0, 10 * math.pi, -8.0, 8.0, SEQ),
                                               ic="saturated_two_stream_64", chi=128,
                                               dt=0.6 * (10 * math.pi / 4096) / 8.0),
    "two_stream_4096x4096_seq": dict(layout=Layout(12, 12, 0.0, 10 * math.pi, -8.0, 8.0, SEQ),
                                     ic="two_stream", chi=128, dt=0.6 * (10 * math.pi / 4096) / 8.0),
}


# Several-species workloads (Methods, "Buneman instability": m_i/m_e = 25,
# k = 0.10, electrons drifting at omega_pe/k, collision rate ~0.007 omega_ps
# per species).  Species: (q, m, nu, u, vth); layouts from buneman_layouts.
SPECIES_WORKLOADS = {
    "saturated_buneman_512x512_s3": dict(bits=(9, 9, 9), mapping=SEQ_S3, ic="saturated_buneman", chi=64,
                                         species=[(-1.0, 1.0, 0.007, 10.0, 1.0), (1.0, 25.0, 0.0014, 0.0, 0.2)]),
    "saturated_buneman_64x64_s3": dict(bits=(6, 6, 6), mapping=SEQ_S3, ic="saturated_buneman", chi=24,
                                       species=[(-1.0, 1.0, 0.007, 10.0, 1.0), (1.0, 25.0, 0.0014, 0.0, 0.2)]),
}


def species_workload(name: str):
    """(layouts, initial grids, species, chi, dt) of a several-species
    workload; dt = 0.6 dx / max|v| of the electrons."""
    w = SPECIES_WORKLOADS[name]
    nx, nve, nvi = w["bits"]
    lay_e, lay_i = buneman_layouts(nx, nve, nvi, mapping=w["mapping"])
    fe, fi = {"saturated_buneman": saturated_buneman, "buneman": buneman}[w["ic"]](lay_e, lay_i)
    dt = 0.6 * ((lay_e.xmax - lay_e.xmin) / lay_e.Nx) / max(abs(lay_e.vmin), abs(lay_e.vmax))
    return [lay_e, lay_i], [fe, fi], w["species"], w["chi"], dt


def initial_condition(name: str, layout: Layout) -> np.ndarray:
    return {"landau": landau, "nonlinear_landau": nonlinear_landau, "two_stream": two_stream,
            "bump_on_tail": bump_on_tail, "saturated_two_stream": saturated_two_stream,
            "saturated_two_stream_64": lambda lay: saturated_two_stream(lay, modes=64)}[name](layout)
