"""CUDA path vs the CPU oracle, element by element (GPU).

Every call goes through the C ABI (ctypes binding); expected values come from
``oracle/`` on the same seeded inputs.  Floating-point bar: relative L2 of the
dense result <= 1e-10 (f) and 1e-9 (field energy), the FP64 tolerances of the
method's parity contract.  MPS cores are compared only through dense
contractions or gauge-invariant quantities (cores are unique only up to gauge
and sign).
"""
import math

import numpy as np
import pytest

from oracle import mpo as OM
from oracle import mps as OS
from oracle import vp as OV
from paper_2205_11990_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F_TOL = 1e-10
WE_TOL = 1e-9


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    c = vpmps.Context()
    yield c
    c.close()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


LAYS = [I.Layout(3, 4, 0.0, 2 * math.pi, -5.0, 5.0, I.SEQ),
        I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.INTERLEAVED),
        I.Layout(3, 5, 0.0, 3.0, -4.0, 4.0, I.INTERLEAVED),
        I.Layout(4, 3, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ_S2),
        I.Layout(3, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ_S3)]


# ----------------------------------------------------------------- MPOs (a2)
@pytest.mark.parametrize("lay", LAYS)
def test_mpo_builders_match_printed_operators(ctx, lay):
    from paper_2205_11990_gb300 import vpmps as V
    dx, dv = OV.grid_steps(lay)
    sm = OV.sitemap(lay)
    idx, idv = OM.identity(lay.nx), OM.identity(lay.nv)
    nx = lay.nx
    ox = lambda ch: OV.orient(ch, lay, 0)  # noqa: E731
    cases = {
        V.MPO_DX_CENTERED: OM.place([ox(OM.centered_periodic(nx, dx)), idv], sm),
        V.MPO_DX_FORWARD: OM.place([ox(OM.forward_periodic(nx, dx)), idv], sm),
        V.MPO_DX_BACKWARD: OM.place([ox(OM.backward_periodic(nx, dx)), idv], sm),
        V.MPO_DV_ZERO_GRAD: OM.place([idx, OV.orient(OM.centered_zero_gradient(lay.nv, dv), lay, 1)], sm),
        V.MPO_DXX: OM.place([ox(OM.second_periodic(nx, dx)), idv], sm),
        V.MPO_ADVECTION: OV._static_parts(lay)[0],
    }
    for kind, ref in cases.items():
        got = ctx.mpo_vp(lay, kind).to_dense()
        want = OM.to_dense(ref)
        assert rel(got, want) < 1e-13, kind


@pytest.mark.parametrize("lay", LAYS)
def test_vlasov_operator_with_field(ctx, lay):
    x = lay.x()
    E = 0.3 * np.sin(2 * np.pi * x / (lay.xmax - lay.xmin)) + 0.05 * np.cos(6 * np.pi * x / (lay.xmax - lay.xmin))
    got = ctx.mpo_vlasov(lay, E, 1e-12).to_dense()
    want = OM.to_dense(OV.operator(OV.field_mps(E, lay, 1e-12), lay))
    assert rel(got, want) < 1e-12


# ----------------------------------------------------- apply / add (a6, a7)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_apply_mpo_random(ctx, seed):
    rng = np.random.default_rng(seed)
    n = 6
    ranks = [1, 2, 3, 7, 5, 2, 1]
    w = [1, 3, 2, 5, 4, 3, 1]
    mps = I.random_cores(ranks, seed=seed)
    mpo = [rng.standard_normal((w[k], 2, 2, w[k + 1])) for k in range(n)]
    out = ctx.apply_mpo(ctx.mpo_from_cores(mpo), ctx.mps_from_cores(mps))
    assert out.bonds() == [a * b for a, b in zip(ranks, w)]
    assert rel(out.to_dense(), OS.to_dense(OS.apply_mpo(mpo, mps))) < 1e-13


def test_axpby_random(ctx):
    a = I.random_cores([1, 2, 4, 3, 1], seed=5)
    b = I.random_cores([1, 2, 2, 5, 1], seed=6)
    out = ctx.axpby(0.7, ctx.mps_from_cores(a), -1.9, ctx.mps_from_cores(b))
    assert out.bonds() == [1, 4, 6, 8, 1]
    assert rel(out.to_dense(), 0.7 * OS.to_dense(a) - 1.9 * OS.to_dense(b)) < 1e-14


# --------------------------------------------------------- compression (a8, a9)
COMPRESS_CASES = [
    # ranks, chi, tol  (ragged bonds; tall and wide SVD reshapes; several tiles)
    ([1, 2, 4, 8, 16, 8, 4, 2, 1], 1 << 10, 0.0),
    ([1, 2, 4, 8, 16, 8, 4, 2, 1], 5, 0.0),
    ([1, 2, 3, 37, 90, 41, 7, 2, 1], 1 << 10, 0.0),
    ([1, 2, 4, 8, 16, 32, 64, 130, 64, 17, 4, 2, 1], 24, 0.0),
    ([1, 2, 4, 8, 16, 32, 70, 150, 200, 75, 31, 8, 2, 1], 1 << 10, 0.0),
    # truncating compressions (the double-word Jacobi path)
    ([1, 2, 4, 8, 16, 32, 70, 150, 200, 75, 31, 8, 2, 1], 1 << 10, 1e-12),
    ([1, 2, 4, 8, 16, 32, 64, 130, 64, 17, 4, 2, 1], 24, 1e-10),
    ([1, 2, 3, 37, 90, 41, 7, 2, 1], 1 << 10, 1e-3),
    # an SVD site of 700 rows: the truncation scan runs over chunks of several
    # values per thread (more values than the block's 512 threads)
    ([1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 700, 512, 256, 128, 64, 32, 16, 8, 4, 2, 1], 1 << 10, 1e-10),
]


@pytest.mark.parametrize("ranks,chi,tol", COMPRESS_CASES)
def test_compress_random(ctx, ranks, chi, tol):
    cores = I.random_cores(ranks, seed=len(ranks) + chi)
    # graded singular values: scale core k by a decaying diagonal so cuts are unambiguous
    ref, ref_errs = OS.compress(cores, chi, tol)
    m = ctx.mps_from_cores(cores)
    errs = ctx.compress(m, chi, tol)
    assert m.bonds() == OS.bonds(ref)
    assert rel(m.to_dense(), OS.to_dense(ref)) < F_TOL
    np.testing.assert_allclose(errs, ref_errs, rtol=1e-6, atol=1e-14)


def test_compress_tolerance_on_smooth_state(ctx):
    lay = I.Layout(6, 6, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f = I.saturated_two_stream(lay, modes=6)
    v = OV.dense_to_sites(f, lay)
    exact = OS.tt_svd(v, lay.n)
    for tol, chi in ((1e-10, 1 << 10), (1e-6, 1 << 10), (1e-10, 9)):
        ref, ref_errs = OS.compress(exact, chi, tol)
        m = ctx.mps_from_cores(exact)
        errs = ctx.compress(m, chi, tol)
        assert m.bonds() == OS.bonds(ref), (tol, chi)
        assert rel(m.to_dense(), OS.to_dense(ref)) < F_TOL
        assert max(errs) <= max(tol, 1.0) and abs(max(errs) - max(ref_errs)) <= 1e-6 * max(ref_errs) + 1e-15


def test_compress_rank_deficient_sum(ctx):
    # f + f has every bond doubled with exactly dependent rows: the truncating
    # compression must find the original ranks (singular values at round-off
    # level are cut) and reproduce 2 f
    lay = I.Layout(5, 6, 0.0, 4 * math.pi, -6.0, 6.0, I.INTERLEAVED)
    f = I.landau(lay, 0.3, 0.5) + 0.05 * I.saturated_two_stream(lay, modes=4)
    a = ctx.mps_from_grid(lay, f, 1 << 10, 1e-12)
    s = ctx.axpby(1.0, a, 1.0, a)
    assert s.bonds()[1:-1] == [2 * r for r in a.bonds()[1:-1]]
    ref, _ = OS.compress(OS.add(a.cores(), a.cores(), 1.0, 1.0), 1 << 10, 1e-12)
    ctx.compress(s, 1 << 10, 1e-12)
    assert s.bonds() == OS.bonds(ref)
    assert max(s.bonds()) <= max(a.bonds())
    assert rel(s.to_grid(lay), 2 * a.to_grid(lay)) < F_TOL


def test_compress_zero_state(ctx):
    cores = [np.zeros((1, 2, 3)), np.zeros((3, 2, 2)), np.zeros((2, 2, 1))]
    m = ctx.mps_from_cores(cores)
    ctx.compress(m, 4, 1e-10)
    assert m.bonds() == [1, 1, 1, 1]
    assert np.all(m.to_dense() == 0.0)


# --------------------------------------------------------------- create (a1)
@pytest.mark.parametrize("lay", LAYS + [I.Layout(6, 6, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)])
def test_create_from_grid(ctx, lay):
    f = I.landau(lay, 0.3, 0.5) + 0.01 * I.random_vector(lay.n, 1).reshape(lay.Nx, lay.Nv)
    for chi, tol in ((1 << 10, 0.0), (1 << 10, 1e-10), (6, 1e-10)):
        ref = OV.mps_from_f(f, lay, chi, tol)
        m = ctx.mps_from_grid(lay, f, chi, tol)
        assert m.bonds() == OS.bonds(ref)
        assert rel(m.to_grid(lay), OV.mps_to_f(ref, lay)) < F_TOL


# ------------------------------------------------------- density, field (a3-a5)
@pytest.mark.parametrize("lay", LAYS)
def test_density_poisson(ctx, lay):
    f = I.landau(lay, 0.4, 0.5 * 2 * math.pi / (lay.xmax - lay.xmin) * 2)
    m = ctx.mps_from_grid(lay, f, 1 << 10, 0.0)
    rho = ctx.density(lay, m)
    ref_rho = OV.density(OV.mps_from_f(f, lay, 1 << 10, 0.0), lay)
    assert rel(rho.cpu().numpy(), ref_rho) < 1e-13
    dx, _ = OV.grid_steps(lay)
    E, we = ctx.poisson(rho, lay.nx, dx)
    ref_E, ref_we = OV.field(ref_rho, dx)
    assert rel(E.cpu().numpy(), ref_E) < 1e-11
    assert abs(we - ref_we) <= 1e-11 * ref_we


def test_poisson_large_grid(ctx):
    import torch
    rng = np.random.default_rng(3)
    for nx in (10, 12):
        rho = 1.0 + 0.1 * rng.standard_normal(1 << nx)
        E, we = ctx.poisson(torch.tensor(rho, device="cuda"), nx, 0.01)
        ref_E, ref_we = OV.field(rho, 0.01)
        assert rel(E.cpu().numpy(), ref_E) < 1e-10
        assert abs(we - ref_we) <= 1e-10 * ref_we


# --------------------------------------------------------------- step (a10)
STEP_CASES = [
    (I.Layout(5, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ), "landau", 0.02, 16, 3),
    (I.Layout(5, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ_S2), "landau", 0.02, 16, 2),
    (I.Layout(5, 5, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ_S3), "two_stream", 0.05, 16, 2),
    (I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.INTERLEAVED), "landau", 0.05, 8, 3),
    (I.Layout(5, 6, 0.0, 10 * math.pi, -8.0, 8.0, I.INTERLEAVED), "two_stream", 0.05, 12, 2),
    (I.Layout(6, 6, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ), "landau", 0.02, 64, 2),
]


@pytest.mark.parametrize("lay,ic,dt,chi,nsteps", STEP_CASES)
def test_rk4_c1_steps(ctx, lay, ic, dt, chi, nsteps):
    f0 = I.initial_condition(ic, lay)
    if ic == "landau":
        f0 = I.landau(lay, 0.3, 0.5)
    m = ctx.mps_from_grid(lay, f0, chi, 1e-10)
    sim = ctx.sim(lay, m, dt, chi)
    ref = OV.mps_from_f(f0, lay, chi, 1e-10)
    for step in range(nsteps):
        rec = sim.step(1)[0]
        ref, d = OV.rk4_step(ref, lay, dt, chi)
        assert abs(rec["field_energy"] - d["field_energy"]) <= WE_TOL * d["field_energy"]
        # mass to the f tolerance: the truncating factorisations run in
        # double-word arithmetic (~1e-12)
        assert abs(rec["mass"] - d["mass"]) <= F_TOL * abs(d["mass"])
        assert sim.state().bonds() == d["bonds"]
        assert rel(sim.state().to_grid(lay), OV.mps_to_f(ref, lay)) < F_TOL
        np.testing.assert_allclose(sim.entropy(), d["entropy"], rtol=1e-8, atol=1e-12)


def test_exact_mode_matches_dense_grid(ctx):
    # untruncated MPS (chi = 2^(n/2), tol = 0) equals the dense FD solver
    from oracle import dense_fd as DF
    lay = I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay, 0.3, 0.5)
    m = ctx.mps_from_grid(lay, f0, 16, 0.0)
    sim = ctx.sim(lay, m, 0.05, 16, tol=0.0, e_tol=0.0)
    sim.step(5)
    fd = f0.copy()
    for _ in range(5):
        fd, _, _ = DF.rk4_step(fd, lay, 0.05)
    assert rel(sim.state().to_grid(lay), fd) < 1e-12


def test_run_entry_point(ctx):
    lay = I.Layout(4, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay, 0.2, 0.5)
    fT, recs = ctx.run(lay, f0, 0.02, 2, 16)
    ref = OV.mps_from_f(f0, lay, 16, 1e-10)
    for _ in range(2):
        ref, d = OV.rk4_step(ref, lay, 0.02, 16)
    assert rel(fT, OV.mps_to_f(ref, lay)) < F_TOL
    assert len(recs) == 2 and recs[1]["t"] == pytest.approx(0.02)


def test_cfl_guard(ctx):
    from paper_2205_11990_gb300 import vpmps
    lay = I.Layout(4, 4, 0.0, 1.0, -8.0, 8.0, I.SEQ)
    m = ctx.mps_from_grid(lay, I.landau(lay), 8, 1e-10)
    with pytest.raises(vpmps.VpError) as e:
        ctx.sim(lay, m, 1.0, 8)
    assert e.value.code == 7


# ---------------------------------------------- compression levels C2-C5, D_F
@pytest.mark.parametrize("level,e_chi", [(2, 0), (3, 0), (4, 0), (5, 0), (1, 3), (4, 2)])
def test_compression_levels_and_field_cap(ctx, level, e_chi):
    lay = I.Layout(5, 5, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ)
    f0 = I.saturated_two_stream(lay, modes=6)
    chi, dt = 10, 0.02
    m = ctx.mps_from_grid(lay, f0, chi, 1e-10)
    sim = ctx.sim(lay, m, dt, chi, level=level, e_chi=e_chi)
    ref = OV.mps_from_f(f0, lay, chi, 1e-10)
    for _ in range(2):
        rec = sim.step(1)[0]
        ref, d = OV.rk4_step(ref, lay, dt, chi, level=level, e_chi=e_chi or None)
        assert abs(rec["field_energy"] - d["field_energy"]) <= WE_TOL * d["field_energy"]
        assert sim.state().bonds() == d["bonds"]
        assert rel(sim.state().to_grid(lay), OV.mps_to_f(ref, lay)) < F_TOL


# Reduced-precision contraction modes against the FP64 oracle.  Each mode
# rounds the operands of the sweeps' GEMMs (and of the density) to a unit
# roundoff u: FP32 2^-24, TF32x3 ~2^-21 (11 + 11 significant bits, FP32
# accumulation), TF32 2^-11, BF16 2^-8.  That rounding, carried through four
# RK4-C1 steps (28 compressions), moves f by a modest multiple of u: the bound
# is K_f u with one K_f for every mode, and a floor of 1e-3 u shows the mode
# is really active.  W_E is quadratic in the field of a perturbation of
# relative size eps = 0.05 of the state (saturated_two_stream's amplitude), so
# a relative change d of f moves W_E by ~2 d / eps: its bound is K_W = 2 K_f /
# eps times u.
PREC_U = {1: 2.0 ** -24, 4: 2.0 ** -21, 2: 2.0 ** -11, 3: 2.0 ** -8}
PREC_K = 200.0
PREC_KW = 2 * PREC_K / 0.05


@pytest.mark.parametrize("prec", [1, 4, 2, 3])
def test_reduced_precision_contractions_vs_oracle(ctx, prec):
    lay = I.Layout(6, 6, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ)
    f0 = I.saturated_two_stream(lay, modes=8)
    chi, dt = 24, 0.02
    m = ctx.mps_from_grid(lay, f0, chi, 1e-10)
    sim = ctx.sim(lay, m, dt, chi, precision=prec)
    recs = sim.step(4)
    fp = sim.state().to_grid(lay)
    sim.close()
    ref = OV.mps_from_f(f0, lay, chi, 1e-10)
    we_ref = []
    for _ in range(4):
        ref, d = OV.rk4_step(ref, lay, dt, chi)
        we_ref.append(d["field_energy"])
    we_ref = np.array(we_ref)
    wep = np.array([r["field_energy"] for r in recs])
    u = PREC_U[prec]
    we_err = float(np.max(np.abs(wep - we_ref) / we_ref))
    f_err = rel(fp, OV.mps_to_f(ref, lay))
    assert we_err < PREC_KW * u and 1e-3 * u < f_err < PREC_K * u, (we_err / u, f_err / u)


def test_profile_trace_records(ctx):
    # the launch trace carries one record per bracketed launch with its shape,
    # and its per-class counts agree with the class totals
    lay = I.Layout(5, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    m = ctx.mps_from_grid(lay, I.landau(lay), 16, 1e-10)
    sim = ctx.sim(lay, m, 0.02, 16, streams=1)
    ctx.profile(True)
    sim.step(1)
    tr = ctx.profile_trace()
    tot = ctx.profile_read()
    ctx.profile(False)
    sim.close()
    assert tr and all(r["ms"] >= 0 for r in tr)
    for cls, (ms, n, _) in tot.items():
        recs = [r for r in tr if r["class"] == cls]
        assert len(recs) == n
        assert abs(sum(r["ms"] for r in recs) - ms) <= 1e-6 * max(1.0, ms)
    qr = [r for r in tr if r["class"] == "qr_factor"]
    assert qr and all(r["m"] >= 1 and r["n"] >= 1 for r in qr)
    jac = [r for r in tr if r["class"] == "jacobi"]
    assert jac and all(r["m"] == r["n"] and r["k"] >= 1 for r in jac)


# ------------------------------------ modified compression (SI scheme, f1)
@pytest.mark.parametrize("ranks,split,chi,tol", [
    ([1, 2, 4, 8, 16, 32, 16, 8, 4, 2, 1], 5, 1 << 10, 0.0),
    ([1, 2, 4, 8, 16, 32, 16, 8, 4, 2, 1], 5, 6, 1e-10),
    ([1, 2, 4, 8, 16, 32, 70, 64, 31, 8, 2, 1], 6, 24, 1e-12),
    ([1, 2, 3, 37, 90, 41, 7, 2, 1], 3, 1 << 10, 1e-3),
])
def test_compress_modified_random(ctx, ranks, split, chi, tol):
    cores = I.random_cores(ranks, seed=len(ranks) + split)
    ref, ref_errs, _ = OS.compress_modified(cores, chi, tol, split)
    m = ctx.mps_from_cores(cores)
    errs = ctx.compress_modified(m, split, chi, tol)
    assert m.bonds() == OS.bonds(ref)
    assert rel(m.to_dense(), OS.to_dense(ref)) < F_TOL
    np.testing.assert_allclose(errs, ref_errs, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("mapping", [I.SEQ, I.SEQ_S2, I.SEQ_S3])
def test_rk4_steps_modified_compression(ctx, mapping):
    lay = I.Layout(5, 5, 0.0, 10 * math.pi, -8.0, 8.0, mapping)
    f0 = I.saturated_two_stream(lay, modes=6)
    dt, chi = 0.05, 12
    m = ctx.mps_from_grid(lay, f0, chi, 1e-10)
    sim = ctx.sim(lay, m, dt, chi, compression=1)
    ref = OV.mps_from_f(f0, lay, chi, 1e-10)
    for _ in range(2):
        rec = sim.step(1)[0]
        ref, d = OV.rk4_step(ref, lay, dt, chi, modified=True)
        assert abs(rec["field_energy"] - d["field_energy"]) <= WE_TOL * d["field_energy"]
        assert sim.state().bonds() == d["bonds"]
        assert rel(sim.state().to_grid(lay), OV.mps_to_f(ref, lay)) < F_TOL
        np.testing.assert_allclose(sim.entropy(), d["entropy"], rtol=1e-8, atol=1e-12)
    sim.close()
    from paper_2205_11990_gb300.vpmps import VpError
    lay_i = I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.INTERLEAVED)
    with pytest.raises(VpError):
        ctx.sim(lay_i, ctx.mps_from_grid(lay_i, I.landau(lay_i), 8, 1e-10), 0.05, 8, compression=1)


def test_compression_error_vs_oracle(ctx):
    # rms compression error against the bond dimension (State Compressibility)
    lay = I.Layout(6, 6, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ)
    f0 = I.saturated_two_stream(lay, modes=12)
    m = ctx.mps_from_grid(lay, f0, 64, 0.0)
    ref = OV.mps_from_f(f0, lay, 64, 0.0)
    chis = [2, 4, 8, 16, 32, 64]
    got = ctx.compression_error(m, chis, 0.0)
    want = OS.compression_error(ref, chis, 0.0)
    scale = float(np.sqrt(np.mean(f0 * f0)))
    assert np.all(np.abs(got - want) <= 1e-10 * scale + 1e-6 * want)
    assert got[-1] <= 1e-12 * scale and np.all(np.diff(got) <= 1e-12 * scale)
