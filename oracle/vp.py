"""One-species Vlasov-Poisson in MPS form, RK4 with compression level C1 (oracle).

Test infrastructure only.  Model (main text, "Problem Statement"; Methods,
normalised units with q_e/m_e = -1 and a uniform neutralising background):

    df/dt = -v df/dx + E df/dv,
    d2phi/dx2 = n_e - mean(n_e),   E = -dphi/dx,   n_e = int f dv.

Discretisation (Methods, "Time Evolution Procedure"; SI "Upwind time
evolution"): x advection upwind with the second-order one-sided stencils
(v > 0 backward, v < 0 forward, as the SI text states), the v derivative
centred with zero-gradient boundaries, E from the centred periodic first
derivative of phi, phi from the periodic second-order Laplacian (zero-mean
pseudo-inverse, SI "Inverse Laplacian"), n_e by the rectangle rule (SI
"Integration").

Time step (SI "Compressed time evolution algorithm", level C1): per RK4 stage
i the field E_i comes from f_i, k_i = L(E_i) f_i is never compressed, the
intermediate states f_{i+1} = f_n + a_i dt k_i (a = 1/2, 1/2, 1) and the
running sum acc_i = acc_{i-1} + b_i dt k_i (acc_0 = f_n, b = 1/6, 1/3, 1/3)
are compressed to the tolerance only, and f_{n+1} = acc_3 + dt/6 k_4 is
compressed to chi and the tolerance.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from . import mpo as M
from . import mps as S

TOL = 1e-10  # "no compression" threshold for every bond (main text, "State Compressibility")


def grid_steps(layout):
    dx = (layout.xmax - layout.xmin) / layout.Nx
    dv = (layout.vmax - layout.vmin) / (layout.Nv - 1)
    return dx, dv


def sitemap(layout):
    """Site -> (dimension, bit).  0 = x, 1 = v; bits most significant first.

    SEQ (S1): all x bits then all v bits, each coarse to fine; S2: x fine to
    coarse, then v coarse to fine; S3: x coarse to fine, then v fine to coarse
    (main text, "State Compressibility").  INTERLEAVED (IF): x_0, v_0, x_1,
    v_1, ...; when nx != nv the leftover bits of the longer dimension follow
    in their own order.
    """
    nx, nv = layout.nx, layout.nv
    if layout.mapping == 0:
        return [(0, b) for b in range(nx)] + [(1, b) for b in range(nv)]
    if layout.mapping == 2:
        return [(0, nx - 1 - b) for b in range(nx)] + [(1, b) for b in range(nv)]
    if layout.mapping == 3:
        return [(0, b) for b in range(nx)] + [(1, nv - 1 - b) for b in range(nv)]
    out = []
    for b in range(max(nx, nv)):
        if b < nx:
            out.append((0, b))
        if b < nv:
            out.append((1, b))
    return out


def dense_to_sites(f, layout):
    """f[ix, iv] -> vector indexed by the site bits (site 0 most significant)."""
    nx, nv = layout.nx, layout.nv
    axes = [b if d == 0 else nx + b for (d, b) in sitemap(layout)]
    return np.asarray(f, dtype=np.float64).reshape([2] * (nx + nv)).transpose(axes).reshape(-1)


def sites_to_dense(vec, layout):
    nx, nv = layout.nx, layout.nv
    axes = [b if d == 0 else nx + b for (d, b) in sitemap(layout)]
    inv = np.argsort(axes)
    return vec.reshape([2] * (nx + nv)).transpose(inv).reshape(layout.Nx, layout.Nv)


def descending(layout, dim):
    """True when the bits of `dim` appear fine to coarse in the site order."""
    return (layout.mapping == 2 and dim == 0) or (layout.mapping == 3 and dim == 1)


def orient(chain, layout, dim):
    """An MPO/MPS chain built coarse-to-fine, put in the site order of `dim`."""
    return M.reverse(chain) if descending(layout, dim) else chain


def bitrev(n_bits):
    idx = np.arange(1 << n_bits)
    out = np.zeros_like(idx)
    for b in range(n_bits):
        out |= ((idx >> b) & 1) << (n_bits - 1 - b)
    return out


def mps_from_f(f, layout, chi, tol=TOL):
    return S.from_dense(dense_to_sites(f, layout), layout.n, chi, tol)


def mps_to_f(cores, layout):
    return sites_to_dense(S.to_dense(cores), layout)


# ---------------------------------------------------------------- density (a3)
def density(cores, layout):
    """n_e(x_i) = sum_j f(x_i, v_j) dv: contract every v site with dv*[1,1]
    (SI "Integration"), then expand the remaining x MPS to the dense vector."""
    _, dv = grid_steps(layout)
    sm = sitemap(layout)
    vsites = {k for k, (d, _) in enumerate(sm) if d == 1}
    vecs = {k: np.ones(2) for k in vsites}
    xm = S.contract_sites(cores, vsites, vecs)
    rho = S.to_dense(xm) * dv  # indexed by the x bits in site order
    return rho[bitrev(layout.nx)] if descending(layout, 0) else rho


# ---------------------------------------------------------------- Poisson (a4)
@functools.lru_cache(maxsize=8)
def _laplacian_pinv(Nx, dx):
    D2 = M.to_dense(M.second_periodic(int(round(math.log2(Nx))), dx))
    # the smallest nonzero eigenvalue is 4 sin^2(pi/N)/dx^2, i.e. >= 1e-8 of the
    # largest for N <= 2^14: a relative cut of 1e-9 drops only the null space
    return np.linalg.pinv(D2, rtol=1e-9, hermitian=True)


def poisson_pinv(rho, dx):
    """phi = pinv(D2) (rho - mean rho): the zero-mean solution of the periodic
    second-order Poisson problem (SI "Inverse Laplacian" inverts the dense
    Laplacian)."""
    rho = np.asarray(rho, dtype=np.float64)
    return _laplacian_pinv(len(rho), dx) @ (rho - rho.mean())


def poisson_dft(rho, dx):
    """Same solution through the DFT, which diagonalises the circulant
    Laplacian: eigenvalue -4 sin^2(pi m / N) / dx^2, mode 0 set to zero."""
    rho = np.asarray(rho, dtype=np.float64)
    N = len(rho)
    s = np.fft.fft(rho - rho.mean())
    m = np.arange(N)
    lam = -4.0 * np.sin(np.pi * m / N) ** 2 / (dx * dx)
    lam[0] = 1.0
    phi_hat = s / lam
    phi_hat[0] = 0.0
    return np.real(np.fft.ifft(phi_hat))


def field(rho, dx):
    """E = -D_c phi (centred periodic), field energy W_E = 1/2 sum E^2 dx."""
    phi = poisson_pinv(rho, dx) if len(rho) <= 2048 else poisson_dft(rho, dx)
    E = -(np.roll(phi, -1) - np.roll(phi, 1)) / (2.0 * dx)
    return E, 0.5 * float(np.sum(E * E)) * dx


# ------------------------------------------------------------- operators (a2)
def _vh_mps(layout, positive):
    """MPS of v*H(v) (or v*(1-H(v))) on the v bits, found numerically by TT-SVD
    (SI "Upwind time evolution")."""
    v = layout.v()
    h = (v > 0).astype(np.float64) if positive else (v <= 0).astype(np.float64)
    return S.from_dense(v * h, layout.nv, 1 << layout.nv, 1e-14)


@functools.lru_cache(maxsize=16)
def _static_parts(layout):
    dx, dv = grid_steps(layout)
    sm = sitemap(layout)
    vp = M.diag_from_mps(_vh_mps(layout, True))
    vm = M.diag_from_mps(_vh_mps(layout, False))
    # -v+ D_b  -v- D_f  (v > 0 takes the backward stencil, v < 0 the forward one)
    bwd = orient(M.mpo_scale(M.backward_periodic(layout.nx, dx), -1.0), layout, 0)
    fwd = orient(M.mpo_scale(M.forward_periodic(layout.nx, dx), -1.0), layout, 0)
    up = M.mpo_sum(M.place([bwd, orient(vp, layout, 1)], sm), M.place([fwd, orient(vm, layout, 1)], sm))
    dvz = orient(M.centered_zero_gradient(layout.nv, dv), layout, 1)
    return up, dvz


def operator(E_cores, layout):
    """L(E) = -v+ D_b^x - v- D_f^x + diag(E) D_c^v (zero-gradient v)."""
    up, dvz = _static_parts(layout)
    et = M.place([M.diag_from_mps(E_cores), dvz], sitemap(layout))
    return M.mpo_sum(up, et)


def field_mps(E, layout, tol=TOL, e_chi=None):
    """E(x) as an MPS on the x bits in their site order, tolerance-truncated;
    e_chi caps its bond (the field compression D_F of the main text,
    "Approximation of the nonlinear term"; None: no cap)."""
    E = np.asarray(E, dtype=np.float64)
    if descending(layout, 0):
        E = E[bitrev(layout.nx)]
    return S.from_dense(E, layout.nx, e_chi if e_chi else 1 << layout.nx, tol)


# ------------------------------------------------------------------ step (a10)
A_RK = (0.5, 0.5, 1.0)
B_RK = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


def stage_field(cores, layout, e_tol=TOL):
    dx, _ = grid_steps(layout)
    rho = density(cores, layout)
    E, we = field(rho, dx)
    return E, we, rho


def rhs(cores, layout, e_tol=TOL):
    E, we, rho = stage_field(cores, layout, e_tol)
    L = operator(field_mps(E, layout, e_tol), layout)
    return S.apply_mpo(L, cores), we, rho


def _compressors(layout, modified):
    """(compress, compress_with_entropy) of a step: the plain QR + SVD sweeps,
    or, for a sequential ordering, the modified centre-bond-first scheme with
    the centre at the x / v cut (SI "Modified Compression Scheme")."""
    if not modified:
        return S.compress, S.compress_with_entropy
    if layout.mapping not in (0, 2, 3):
        raise ValueError("the modified compression needs a sequential ordering")
    split = layout.nx

    def comp(c, chi, tol):
        out, errs, _ = S.compress_modified(c, chi, tol, split)
        return out, errs

    def comp_ee(c, chi, tol):
        out, errs, sv = S.compress_modified(c, chi, tol, split)
        ee = [S.entanglement_entropy(sv[j], out[j + 1].shape[0]) for j in range(len(out) - 1)]
        return out, errs, ee

    return comp, comp_ee


def rk4_step(f, layout, dt, chi, tol=TOL, e_tol=TOL, level=1, e_chi=None, modified=False):
    """One RK4 step; returns (f_{n+1}, diagnostics).

    Compression levels (SI "Compressed time evolution algorithm"); every
    compression also applies the tolerance:
      C1  f_{n+1} to chi; intermediate states and the running sum to tol only;
      C2  C1 + the intermediate states f_n + a_i dt k_i to chi;
      C3  C2 + the sum of derivatives: D = k_1, D <- C_chi(D + w_i k_i) with
          w = (2, 2, 1), f_{n+1} = C_chi(f_n + dt/6 D);
      C4  C3 + each derivative k_i = C_chi(L f_i);
      C5  C4 + the terms of each derivative: k_i = C_chi(C_chi(U f_i) +
          C_chi(T f_i)), U the advection operator, T the field term.
    """
    comp, comp_ee = _compressors(layout, modified)
    if level != 1 or e_chi:
        return _rk4_step_levels(f, layout, dt, chi, tol, e_tol, level, e_chi, comp, comp_ee)
    acc = f
    fi = f
    diag = {}
    errs = None
    for i in range(4):
        k, we, rho = rhs(fi, layout, e_tol)
        if i == 0:
            dx, dv = grid_steps(layout)
            diag["field_energy"] = we
            diag["mass"] = float(np.sum(rho)) * dx
        if i < 3:
            fi, _ = comp(S.add(f, k, 1.0, A_RK[i] * dt), 1 << 30, tol)
            acc, _ = comp(S.add(acc, k, 1.0, B_RK[i] * dt), 1 << 30, tol)
        else:
            acc, errs, ee = comp_ee(S.add(acc, k, 1.0, B_RK[3] * dt), chi, tol)
            diag["entropy"] = ee
    diag["trunc_err"] = errs
    diag["bonds"] = S.bonds(acc)
    return acc, diag


def stable_dt(layout, dt_cfg=None, cfl=0.6):
    """Fixed step: dt_cfg divided by the smallest integer s with
    vmax*dt/dx <= cfl; without dt_cfg, dt = cfl*dx/vmax.  RK4 with the
    second-order upwind stencil is stable for vmax*dt/dx <= 0.696 (the
    adaptive 0.9*CFL rule of the Methods section exceeds that)."""
    dx, _ = grid_steps(layout)
    vmax = max(abs(layout.vmin), abs(layout.vmax))
    if dt_cfg is None:
        return cfl * dx / vmax
    s = max(1, math.ceil(vmax * dt_cfg / dx / cfl - 1e-12))
    return dt_cfg / s


def run(f0, layout, dt, nsteps, chi, tol=TOL, e_tol=TOL, every=1):
    cores = mps_from_f(f0, layout, chi, tol)
    hist = []
    for step in range(nsteps):
        cores, d = rk4_step(cores, layout, dt, chi, tol, e_tol)
        if step % every == 0:
            hist.append((step * dt, d["field_energy"], d["mass"], max(d["bonds"])))
    return cores, hist


W_RK = (1.0, 2.0, 2.0, 1.0)


def _rk4_step_levels(f, layout, dt, chi, tol, e_tol, level, e_chi, comp=S.compress, comp_ee=S.compress_with_entropy):
    big = 1 << 30
    up, dvz = _static_parts(layout)
    sm = sitemap(layout)
    acc, D, fi, k = f, None, f, None
    diag = {}
    errs = None
    for i in range(4):
        E, we, rho = stage_field(fi, layout, e_tol)
        if i == 0:
            dx, _ = grid_steps(layout)
            diag["field_energy"] = we
            diag["mass"] = float(np.sum(rho)) * dx
        Em = field_mps(E, layout, e_tol, e_chi)
        if level >= 5:
            ku, _ = comp(S.apply_mpo(up, fi), chi, tol)
            kt, _ = comp(S.apply_mpo(M.place([M.diag_from_mps(Em), dvz], sm), fi), chi, tol)
            k, _ = comp(S.add(ku, kt), chi, tol)
        else:
            k = S.apply_mpo(M.mpo_sum(up, M.place([M.diag_from_mps(Em), dvz], sm)), fi)
            if level >= 4:
                k, _ = comp(k, chi, tol)
        if level >= 3:
            D = k if i == 0 else comp(S.add(D, k, 1.0, W_RK[i]), chi, tol)[0]
        elif i < 3:
            acc, _ = comp(S.add(acc, k, 1.0, B_RK[i] * dt), big, tol)
        if i < 3:
            fi, _ = comp(S.add(f, k, 1.0, A_RK[i] * dt), chi if level >= 2 else big, tol)
    if level >= 3:
        out, errs, ee = comp_ee(S.add(f, D, 1.0, dt / 6.0), chi, tol)
    else:
        out, errs, ee = comp_ee(S.add(acc, k, 1.0, B_RK[3] * dt), chi, tol)
    diag["entropy"] = ee
    diag["trunc_err"] = errs
    diag["bonds"] = S.bonds(out)
    return out, diag


# ------------------------------------------- several species sharing E
def species_params(sp):
    """(q, m) or (q, m, nu, u, vth) -> (q, m, nu, u, vth): charge and mass in
    electron units, Dougherty collision rate, drift and thermal speed."""
    sp = tuple(sp)
    return sp + (0.0, 0.0, 1.0)[len(sp) - 2:] if len(sp) < 5 else sp


def collision_mpo(layout, nu, u, vth):
    """nu d/dv [(v - u) f + vth^2 df/dv] (Methods, "Collision Operator",
    the Dougherty operator) with u and vth the species' drift and thermal
    speed: nu [D_c^v diag(v - u) + vth^2 D_vv] on the v bits, both
    derivatives with zero-gradient ghosts, identity on the x bits."""
    _, dv = grid_steps(layout)
    drift = M.diag_from_mps(S.from_dense(layout.v() - u, layout.nv, 1 << layout.nv, 1e-14))
    cv = M.mpo_sum(M.mpo_product(M.centered_zero_gradient(layout.nv, dv), drift),
                   M.mpo_scale(M.second_zero_gradient(layout.nv, dv), vth * vth))
    cv = M.mpo_scale(cv, nu)
    return M.place([M.identity(layout.nx), orient(cv, layout, 1)], sitemap(layout))


def multi_stage_field(fs, layouts, species):
    """E from the net charge sum_s q_s n_s of all species (Problem
    Statement, every species evolved: no fixed background).  The periodic
    solve is the one of :func:`field`, fed with -sum_s q_s rho_s (for
    electrons alone that is rho_e: the one-species equation).  Returns
    (E, W_E, per-species densities)."""
    dx, _ = grid_steps(layouts[0])
    rhos = [density(c, lay) for c, lay in zip(fs, layouts)]
    net = -sum(species_params(sp)[0] * r for sp, r in zip(species, rhos))
    E, we = field(net, dx)
    return E, we, rhos


def multi_rk4_step(fs, layouts, species, dt, chi, tol=TOL, e_tol=TOL):
    """One RK4-C1 step of several species sharing the field: species s obeys
    df_s/dt = -v df_s/dx - (q_s / m_s) E df_s/dv + C[f_s], the one-species
    operator with E scaled by -q_s / m_s (electrons: +1) plus the Dougherty
    term when nu_s > 0.  The stage field is computed once from all species'
    stage states; every species then follows the C1 schedule of
    :func:`rk4_step`.  Returns (new states, diagnostics)."""
    n = len(fs)
    accs = list(fs)
    fis = list(fs)
    coll = []
    for sp, lay in zip(species, layouts):
        _, _, nu, u, vth = species_params(sp)
        coll.append(collision_mpo(lay, nu, u, vth) if nu else None)
    diag = {}
    for i in range(4):
        E, we, rhos = multi_stage_field(fis, layouts, species)
        if i == 0:
            dx, _ = grid_steps(layouts[0])
            diag["field_energy"] = we
            diag["mass"] = [float(np.sum(r)) * dx for r in rhos]
        ks = []
        for s in range(n):
            q, m = species_params(species[s])[:2]
            L = operator(field_mps(-q / m * E, layouts[s], e_tol), layouts[s])
            if coll[s] is not None:
                L = M.mpo_sum(L, coll[s])
            ks.append(S.apply_mpo(L, fis[s]))
        errs = []
        for s in range(n):
            if i < 3:
                fis[s], _ = S.compress(S.add(fs[s], ks[s], 1.0, A_RK[i] * dt), 1 << 30, tol)
                accs[s], _ = S.compress(S.add(accs[s], ks[s], 1.0, B_RK[i] * dt), 1 << 30, tol)
            else:
                accs[s], e = S.compress(S.add(accs[s], ks[s], 1.0, B_RK[3] * dt), chi, tol)
                errs.append(e)
    diag["trunc_err"] = errs
    diag["bonds"] = [S.bonds(a) for a in accs]
    return accs, diag
