"""Pins of the oracle's Vlasov-Poisson pieces and physics (CPU)."""
import math

import numpy as np
import pytest

from oracle import dense_fd as DF
from oracle import dispersion as DS
from oracle import mpo as M
from oracle import mps as S
from oracle import vp as V
from paper_2205_11990_gb300 import inputs as I

LAYOUTS = [I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ),
           I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.INTERLEAVED),
           I.Layout(3, 5, 0.0, 2 * math.pi, -5.0, 5.0, I.INTERLEAVED)]


@pytest.mark.parametrize("lay", LAYOUTS)
def test_site_permutation_roundtrip(lay):
    f = np.random.default_rng(0).standard_normal((lay.Nx, lay.Nv))
    np.testing.assert_array_equal(V.sites_to_dense(V.dense_to_sites(f, lay), lay), f)


@pytest.mark.parametrize("lay", LAYOUTS)
def test_density_is_rectangle_rule(lay):
    f = I.landau(lay, 0.3, 0.5)
    cores = V.mps_from_f(f, lay, 1 << 10, 0.0)
    _, dv = V.grid_steps(lay)
    np.testing.assert_allclose(V.density(cores, lay), f.sum(axis=1) * dv, atol=1e-13)


def test_poisson_single_mode_closed_form():
    N, dx, m, A = 64, 0.3, 3, 0.7
    i = np.arange(N)
    rho = 1.0 + A * np.cos(2 * np.pi * m * i / N)
    # D2 phi = rho - mean: phi = -A dx^2 cos(...) / (4 sin^2(pi m/N))
    phi_ref = -A * dx * dx * np.cos(2 * np.pi * m * i / N) / (4 * np.sin(np.pi * m / N) ** 2)
    np.testing.assert_allclose(V.poisson_pinv(rho, dx), phi_ref, atol=1e-12)
    np.testing.assert_allclose(V.poisson_dft(rho, dx), phi_ref, atol=1e-12)
    E, we = V.field(rho, dx)
    E_ref = -(np.roll(phi_ref, -1) - np.roll(phi_ref, 1)) / (2 * dx)
    np.testing.assert_allclose(E, E_ref, atol=1e-12)
    assert abs(we - 0.5 * np.sum(E_ref ** 2) * dx) < 1e-12


def test_poisson_pinv_matches_dft_random():
    rho = np.random.default_rng(1).standard_normal(256)
    np.testing.assert_allclose(V.poisson_pinv(rho, 0.05), V.poisson_dft(rho, 0.05), atol=1e-12)


@pytest.mark.parametrize("lay", LAYOUTS)
def test_vlasov_operator_equals_dense_rhs(lay):
    f = I.landau(lay, 0.4, 0.5) + 0.1 * I.random_vector(lay.n, 3).reshape(lay.Nx, lay.Nv)
    cores = V.mps_from_f(f, lay, 1 << 10, 0.0)
    E, _, _ = V.stage_field(cores, lay)
    L = V.operator(V.field_mps(E, lay, 0.0), lay)
    got = V.sites_to_dense(M.to_dense(L) @ V.dense_to_sites(f, lay), lay)
    ref, _, _ = DF.rhs(f, lay)
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("lay", LAYOUTS[:2])
def test_untruncated_mps_step_matches_dense_grid(lay):
    # untruncated MPS (chi = 2^(n/2), tol = 0): the same step as the dense FD solver
    f = I.landau(lay, 0.3, 0.5)
    cores = V.mps_from_f(f, lay, 1 << 10, 0.0)
    fd = f.copy()
    dt = 0.05
    for _ in range(6):
        fd, _, _ = DF.rk4_step(fd, lay, dt)
        cores, _ = V.rk4_step(cores, lay, dt, 1 << 10, 0.0, 0.0)
    rel = np.linalg.norm(V.mps_to_f(cores, lay) - fd) / np.linalg.norm(fd)
    assert rel < 1e-12


def test_tolerance_mode_matches_dense_grid_to_tolerance():
    lay = I.Layout(5, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f = I.landau(lay, 0.01, 0.5)
    cores = V.mps_from_f(f, lay, 64, 1e-10)
    fd = f.copy()
    for _ in range(5):
        fd, _, _ = DF.rk4_step(fd, lay, 0.02)
        cores, d = V.rk4_step(cores, lay, 0.02, 64)
    rel = np.linalg.norm(V.mps_to_f(cores, lay) - fd) / np.linalg.norm(fd)
    assert rel < 1e-8
    assert max(d["bonds"]) < 32  # compressed well below the full rank 32


def test_mass_changes_only_by_boundary_flux():
    lay = I.Layout(5, 5, 0.0, 4 * math.pi, -4.0, 4.0, I.SEQ)
    f = I.landau(lay, 0.3, 0.5) + 0.01
    dx, dv = V.grid_steps(lay)
    r, _, _ = DF.rhs(f, lay)
    np.testing.assert_allclose(float(r.sum()) * dx * dv, DF.boundary_flux(f, lay), rtol=1e-10, atol=1e-14)


def test_dispersion_function_pins():
    assert abs(DS.Z(0.0) - 1j * math.sqrt(math.pi)) < 1e-14
    z = 30.0 + 0.0j  # large-argument expansion Z ~ -1/z - 1/(2 z^3) - 3/(4 z^5)
    assert abs(DS.Z(z).real - (-1 / z - 1 / (2 * z ** 3) - 3 / (4 * z ** 5)).real) < 1e-10
    # Bohm-Gross at small k: omega^2 ~ 1 + 3 k^2
    w = DS.landau_root(0.05)
    assert abs(w.real ** 2 - (1 + 3 * 0.05 ** 2)) < 1e-4 and abs(w.imag) < 1e-20
    # cold symmetric beams: omega^2 = a^2 + 1/2 - sqrt(2 a^2 + 1/4), a = k u
    a = 0.2 * 3.0
    cold = math.sqrt(-(a * a + 0.5 - math.sqrt(2 * a * a + 0.25)))
    # (vth = 0.05: the thermal correction is O(3 k^2 vth^2 / (omega - k u)^2) ~ 1e-3)
    w = DS.two_stream_root(0.2, vth=0.05, guess=0.35j)
    assert abs(w.imag - cold) < 2e-3 * cold and abs(w.real) < 1e-8
    for root, k, beams in ((DS.landau_root(0.5), 0.5, [(1, 0, 1)]),
                           (DS.two_stream_root(0.2), 0.2, [(0.5, 3, 1), (0.5, -3, 1)])):
        assert abs(DS.epsilon(root, k, beams)) < 1e-10


def test_landau_root_matches_configured_rate():
    # configuration of the linear Landau workload: damping rate about -0.153
    w = DS.landau_root(0.5)
    assert abs(w.imag - (-0.153)) < 1e-3 and abs(w.real - 1.4157) < 1e-3


def test_dense_solver_landau_damping_rate():
    w = I.WORKLOADS["landau_64x64"]
    lay = w["layout"]
    f0 = I.landau(lay)
    _, ts, wes, _ = DF.run(f0, lay, 0.02, 1000)
    g = DF.fit_rate(ts, wes, 2.0, 18.0)
    assert abs(g - DS.landau_root(0.5).imag) < 0.01


@pytest.mark.slow
def test_dense_solver_two_stream_growth_rate():
    lay = I.Layout(7, 8, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ)
    f0 = I.two_stream(lay)
    dt = V.stable_dt(lay)
    n = int(24.0 / dt)
    _, ts, wes, _ = DF.run(f0, lay, dt, n)
    sel = (ts > 8) & (ts < 22)
    g = 0.5 * np.polyfit(ts[sel], np.log(wes[sel]), 1)[0]
    assert abs(g - DS.two_stream_root(0.2).imag) / DS.two_stream_root(0.2).imag < 0.05


@pytest.mark.parametrize("level", [1, 2, 3, 4, 5])
def test_compression_levels_exact_mode_match_dense_grid(level):
    # with chi = 2^(n/2) and tol = 0 every compression is exact, so all five
    # schedules reproduce the plain RK4 step of the dense solver
    lay = I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f = I.landau(lay, 0.3, 0.5)
    cores = V.mps_from_f(f, lay, 1 << 10, 0.0)
    fd = f.copy()
    for _ in range(3):
        fd, _, _ = DF.rk4_step(fd, lay, 0.05)
        cores, _ = V.rk4_step(cores, lay, 0.05, 1 << 10, 0.0, 0.0, level=level)
    assert np.linalg.norm(V.mps_to_f(cores, lay) - fd) / np.linalg.norm(fd) < 1e-12


@pytest.mark.parametrize("level", [2, 3, 4, 5])
def test_higher_levels_compress_more(level):
    lay = I.Layout(5, 5, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ)
    f = I.saturated_two_stream(lay, modes=6)
    c = V.mps_from_f(f, lay, 8, 1e-10)
    out, d = V.rk4_step(c, lay, 0.02, 8, level=level)
    out1, d1 = V.rk4_step(c, lay, 0.02, 8, level=1)
    assert max(d["bonds"]) <= 8
    # the extra truncations move the result by at most a small fraction
    ref = V.mps_to_f(out1, lay)
    assert np.linalg.norm(V.mps_to_f(out, lay) - ref) / np.linalg.norm(ref) < 1e-2


def test_field_bond_cap():
    lay = I.Layout(6, 5, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ)
    x = lay.x()
    E = sum(np.cos(m * 0.2 * x + m) / m for m in range(1, 12))
    for cap in (2, 4):
        em = V.field_mps(E, lay, 1e-10, cap)
        assert max(S.bonds(em)) <= cap
    # the cap is the best rank-cap approximation: error decreases with the cap
    errs = [np.linalg.norm(S.to_dense(V.field_mps(E, lay, 1e-10, c)) - E) for c in (1, 2, 4, 8)]
    assert errs == sorted(errs, reverse=True)


@pytest.mark.parametrize("mapping", [I.SEQ_S2, I.SEQ_S3])
def test_s2_s3_orderings(mapping):
    lay = I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, mapping)
    f = I.landau(lay, 0.4, 0.5) + 0.1 * I.random_vector(lay.n, 3).reshape(lay.Nx, lay.Nv)
    np.testing.assert_array_equal(V.sites_to_dense(V.dense_to_sites(f, lay), lay), f)
    cores = V.mps_from_f(f, lay, 1 << 10, 0.0)
    _, dv = V.grid_steps(lay)
    np.testing.assert_allclose(V.density(cores, lay), f.sum(axis=1) * dv, atol=1e-13)
    E, _, _ = V.stage_field(cores, lay)
    L = V.operator(V.field_mps(E, lay, 0.0), lay)
    got = V.sites_to_dense(M.to_dense(L) @ V.dense_to_sites(f, lay), lay)
    ref, _, _ = DF.rhs(f, lay)
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())
    # the untruncated step still equals the dense FD step
    fd, _, _ = DF.rk4_step(f, lay, 0.05)
    out, _ = V.rk4_step(cores, lay, 0.05, 1 << 10, 0.0, 0.0)
    assert np.linalg.norm(V.mps_to_f(out, lay) - fd) / np.linalg.norm(fd) < 1e-12


def test_reverse_chain_is_same_operator():
    X = M.forward_periodic(4, 0.3)
    D = M.to_dense(X)
    Dr = M.to_dense(M.reverse(X))
    # reversing the site order permutes the basis by bit reversal
    br = V.bitrev(4)
    np.testing.assert_allclose(Dr, D[np.ix_(br, br)], atol=1e-13)


@pytest.mark.parametrize("mapping", [I.SEQ, I.SEQ_S2, I.SEQ_S3])
def test_modified_compression_step_exact_mode(mapping):
    # the centre-bond-first compression truncates nothing at tol = 0: the MPS
    # step still equals the dense finite-difference step
    lay = I.Layout(3, 4, 0.0, 4 * math.pi, -6.0, 6.0, mapping)
    f0 = I.landau(lay, 0.3, 0.5)
    c = V.mps_from_f(f0, lay, 1 << 10, 0.0)
    c, _ = V.rk4_step(c, lay, 0.05, 1 << 10, 0.0, 0.0, modified=True)
    fd, _, _ = DF.rk4_step(f0.copy(), lay, 0.05)
    assert np.linalg.norm(V.mps_to_f(c, lay) - fd) <= 1e-12 * np.linalg.norm(fd)
    with pytest.raises(ValueError):
        V.rk4_step(c, I.Layout(3, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.INTERLEAVED), 0.05, 8, modified=True)
