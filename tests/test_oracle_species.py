"""Pins of the oracle's several-species path: shared field from the net charge,
the per-species field factor -q/m, and the Dougherty collision operator (CPU)."""
import math

import numpy as np
import pytest

from oracle import dense_fd as DF
from oracle import dispersion as DS
from oracle import mpo as M
from oracle import mps as S
from oracle import vp as V
from paper_2205_11990_gb300 import inputs as I

GOLDEN = __import__("pathlib").Path(__file__).parent / "golden" / "paper_printed_values.txt"


def golden(name):
    for line in GOLDEN.read_text().splitlines():
        if line.startswith(name + " |"):
            _, val, tol, _ = [t.strip() for t in line.split("|", 3)]
            return float(val), float(tol)
    raise KeyError(name)


def stencil_matrix(N, dv, coeffs, ghost):
    """Dense matrix of sum_s c_s f_{j+s} with out-of-range f_{j+s} replaced
    by the ghost rule (brute force, tiny N)."""
    A = np.zeros((N, N))
    for j in range(N):
        for s, c in coeffs:
            A[j, ghost(j + s, N)] += c
    return A


def mirror(jj, N):
    return 1 if jj < 0 else (N - 2 if jj > N - 1 else jj)


@pytest.mark.parametrize("L", [2, 3, 5])
def test_second_zero_gradient_is_mirrored_three_point_stencil(L):
    dv = 0.37
    ref = stencil_matrix(1 << L, dv, [(-1, 1 / dv**2), (0, -2 / dv**2), (1, 1 / dv**2)], mirror)
    np.testing.assert_allclose(M.to_dense(M.second_zero_gradient(L, dv)), ref, atol=1e-12)
    # exact on a quadratic away from the ends
    v = np.arange(1 << L) * dv
    np.testing.assert_allclose((M.to_dense(M.second_zero_gradient(L, dv)) @ v**2)[1:-1], 2.0, rtol=1e-12)


def test_mpo_product_is_matrix_product():
    a = M.centered_zero_gradient(4, 0.2)
    b = M.diag_from_mps(S.from_dense(np.linspace(-3, 5, 16), 4, 16, 0.0))
    np.testing.assert_allclose(M.to_dense(M.mpo_product(a, b)), M.to_dense(a) @ M.to_dense(b), atol=1e-12)


def test_dougherty_maxwellian_is_second_order_steady_state():
    # C[M_{u,vth}] = 0 in the continuum; the discrete residual falls as dv^2
    res = []
    for nv in (7, 8, 9):
        lay = I.Layout(1, nv, 0.0, 1.0, -9.0, 11.0)
        v = lay.v()
        _, dv = V.grid_steps(lay)
        f = I.maxwellian(v, 1.3, 1.0)[None, :]
        res.append(np.max(np.abs(DF.dougherty(f, v, dv, 0.5, 1.0, 1.3))))
    assert res[0] < 1e-3 and 3.6 < res[0] / res[1] < 4.4 and 3.6 < res[1] / res[2] < 4.4


def test_dougherty_other_temperature_closed_form():
    # u = 0, f = M_T: C[f] = nu (1 - vth^2/T) d/dv(v M_T) = nu (1 - vth^2/T) M_T (1 - v^2/T)
    nu, vth, T = 0.3, 1.0, 2.0
    errs = []
    for nv in (8, 9):
        lay = I.Layout(1, nv, 0.0, 1.0, -12.0, 12.0)
        v = lay.v()
        _, dv = V.grid_steps(lay)
        f = I.maxwellian(v, math.sqrt(T))
        exact = nu * (1 - vth**2 / T) * f * (1 - v**2 / T)
        errs.append(np.max(np.abs(DF.dougherty(f[None, :], v, dv, nu, 0.0, vth)[0] - exact)))
    assert errs[1] < 2e-4 and 3.6 < errs[0] / errs[1] < 4.4


@pytest.mark.parametrize("mapping", [I.SEQ, I.INTERLEAVED, I.SEQ_S2, I.SEQ_S3])
def test_collision_mpo_equals_dense_operator(mapping):
    lay = I.Layout(3, 5, 0.0, 2 * math.pi, -7.0, 9.0, mapping)
    f = np.random.default_rng(3).standard_normal((lay.Nx, lay.Nv))
    _, dv = V.grid_steps(lay)
    C = V.collision_mpo(lay, 0.4, 1.5, 0.8)
    got = V.sites_to_dense(M.to_dense(C) @ V.dense_to_sites(f, lay), lay)
    np.testing.assert_allclose(got, DF.dougherty(f, lay.v(), dv, 0.4, 1.5, 0.8), atol=1e-11)


def test_buneman_root_cold_limit():
    # vth -> 0: 1 = 1/(w - k v0)^2 + (1/25)/w^2, a quartic in w
    k, v0, mu = 0.1, 10.0, 1.0 / 25.0
    a = k * v0
    # (w^2)(w-a)^2 - w^2 - mu (w-a)^2 = 0
    p = np.polymul([1, 0, 0], np.polymul([1, -a], [1, -a]))
    p = np.polysub(p, np.polyadd([1, 0, 0], mu * np.polymul([1, -a], [1, -a])))
    cold = max(np.roots(p), key=lambda z: z.imag)
    # the thermal correction falls as vth^2
    d = [abs(DS.buneman_root(k, 25.0, v0, vth_i=vt, vth_e=vt, guess=cold) - cold) for vt in (0.03, 0.01)]
    assert d[1] < 1e-5 and 7.0 < d[0] / d[1] < 11.0


def test_buneman_root_matches_paper_rate():
    g, tol = golden("buneman_growth_rate")
    assert abs(DS.buneman_root(0.1, 25.0, 10.0, 0.2).imag - g) <= tol


def test_dense_two_species_buneman_growth_rate():
    le, li = I.buneman_layouts(5, 8, 6)
    fe, fi = I.buneman(le, li)
    dx, _ = V.grid_steps(le)
    dt = 0.6 * dx / 60.0
    fs, ts, wes = [fe, fi], [], []
    for n in range(int(31.0 / dt)):
        fs, we, _ = DF.multi_rk4_step(fs, [le, li], [(-1.0, 1.0), (1.0, 25.0)], dt)
        ts.append(n * dt)
        wes.append(we)
    ts, wes = np.array(ts), np.array(wes)
    sel = (ts >= 15) & (ts <= 30)
    g = 0.5 * np.polyfit(ts[sel], np.log(wes[sel]), 1)[0]
    ref = DS.buneman_root(0.1, 25.0, 10.0, 0.2).imag
    assert abs(g - ref) / ref < 0.02


@pytest.mark.parametrize("mapping", [I.SEQ, I.INTERLEAVED, I.SEQ_S3])
def test_two_species_exact_mode_matches_dense_grid(mapping):
    le, li = I.buneman_layouts(4, 5, 4, mapping=mapping)
    fe, fi = I.buneman(le, li, amp=0.1)
    sp = [(-1.0, 1.0, 0.05, 10.0, 1.0), (1.0, 25.0, 0.01, 0.0, 0.2)]
    fs = [fe, fi]
    cores = [V.mps_from_f(fe, le, 1 << 20, 0.0), V.mps_from_f(fi, li, 1 << 20, 0.0)]
    for _ in range(2):
        cores, d = V.multi_rk4_step(cores, [le, li], sp, 0.02, 1 << 20, tol=0.0, e_tol=0.0)
        fs, we, rhos = DF.multi_rk4_step(fs, [le, li], sp, 0.02)
        assert abs(d["field_energy"] - we) <= 1e-12 * we
    for c, f, lay in zip(cores, fs, [le, li]):
        np.testing.assert_allclose(V.mps_to_f(c, lay), f, atol=1e-12 * np.abs(f).max())


def test_one_species_reduces_to_single_species_step():
    lay = I.Layout(4, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    c = V.mps_from_f(I.landau(lay, 0.3, 0.5), lay, 64)
    one, d1 = V.rk4_step(c, lay, 0.05, 8)
    many, dm = V.multi_rk4_step([c], [lay], [(-1.0, 1.0)], 0.05, 8)
    np.testing.assert_array_equal(V.mps_to_f(many[0], lay), V.mps_to_f(one, lay))
    assert dm["field_energy"] == d1["field_energy"]


def test_heavy_ions_match_fixed_background():
    # the field is the superposition of the electron and ion fields
    le = I.Layout(4, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    li = I.Layout(4, 4, 0.0, 4 * math.pi, -1.0, 1.0, I.SEQ)
    fe = I.landau(le, 0.3, 0.5)
    fi = np.outer(1.0 + 0.2 * np.cos(0.5 * li.x()), I.maxwellian(li.v(), 0.2))
    ce, ci = V.mps_from_f(fe, le, 64), V.mps_from_f(fi, li, 64)
    (ne, ni), _ = V.multi_rk4_step([ce, ci], [le, li], [(-1.0, 1.0), (1.0, 1e14)], 0.05, 64)
    # ions of huge mass only stream: as a neutral species (q = 0, no field)
    (free,), _ = V.multi_rk4_step([ci], [li], [(0.0, 1.0)], 0.05, 64)
    np.testing.assert_allclose(V.mps_to_f(ni, li), V.mps_to_f(free, li), atol=1e-12)
    # the electrons feel the ion density ripple: -div E = n_e - n_i differs
    # from the fixed-background field by the ion term
    rho_i = fi.sum(axis=1) * V.grid_steps(li)[1]
    E_mix, _, _ = V.multi_stage_field([ce, ci], [le, li], [(-1.0, 1.0), (1.0, 1e14)])
    E_e, _ = V.field(V.density(ce, le), V.grid_steps(le)[0])
    E_i, _ = V.field(rho_i, V.grid_steps(li)[0])
    np.testing.assert_allclose(E_mix, E_e - E_i, atol=1e-12)
