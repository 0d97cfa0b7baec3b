"""Several species sharing one field (vp_multi_*), GPU vs oracle.

The Buneman set-up (Methods, "Buneman instability": drifting electrons through
ions of mass ratio 25, each species on its own v grid), collisionless and with
Dougherty collisions, on every ordering; f per species to 1e-10 relative L2,
the field energy to 1e-9, masses and bonds exactly as the oracle's.
"""
import math

import numpy as np
import pytest

from oracle import vp as OV
from paper_2205_11990_gb300 import inputs as I

pytestmark = pytest.mark.gpu

COLL = [(-1.0, 1.0, 0.05, 10.0, 1.0), (1.0, 25.0, 0.01, 0.0, 0.2)]
FREE = [(-1.0, 1.0), (1.0, 25.0)]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    c = vpmps.Context()
    yield c
    c.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_pair(ctx, lays, fs, species, dt, chi, nsteps, tol=1e-10, streams=2):
    ms = [ctx.mps_from_grid(l, f, 1 << 20, tol) for l, f in zip(lays, fs)]
    refs = [OV.mps_from_f(f, l, 1 << 20, tol) for l, f in zip(lays, fs)]
    run = ctx.multi(lays, species, ms, dt, chi, tol=tol, streams=streams)
    for _ in range(nsteps):
        rec = run.step(1)[0]
        refs, d = OV.multi_rk4_step(refs, lays, species, dt, chi, tol=tol)
        assert abs(rec["field_energy"] - d["field_energy"]) <= 1e-9 * d["field_energy"]
        np.testing.assert_allclose(rec["mass"], d["mass"], rtol=1e-10)  # f itself agrees to 1e-10
        for s in range(len(lays)):
            assert run.state(s).bonds() == d["bonds"][s]
    for s, (l, r) in enumerate(zip(lays, refs)):
        assert rel(run.state(s).to_grid(l), OV.mps_to_f(r, l)) < 1e-10, s
    run.close()


@pytest.mark.parametrize("mapping", [I.SEQ, I.INTERLEAVED, I.SEQ_S2, I.SEQ_S3])
@pytest.mark.parametrize("species", [FREE, COLL], ids=["collisionless", "dougherty"])
def test_buneman_steps_match_oracle(ctx, mapping, species):
    le, li = I.buneman_layouts(5, 6, 5, mapping=mapping)
    fe, fi = I.buneman(le, li, amp=0.05)
    dt = 0.5 * V_dt(le)
    run_pair(ctx, [le, li], [fe, fi], species, dt, 12, 3)


def V_dt(lay):
    dx, _ = OV.grid_steps(lay)
    return 0.6 * dx / max(abs(lay.vmin), abs(lay.vmax))


def test_buneman_one_stream(ctx):
    le, li = I.buneman_layouts(5, 7, 5)
    fe, fi = I.buneman(le, li, amp=0.05)
    run_pair(ctx, [le, li], [fe, fi], COLL, V_dt(le), 16, 2, streams=1)


def test_one_species_equals_single_species_sim(ctx):
    lay = I.Layout(5, 6, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay, 0.3, 0.5)
    a = ctx.sim(lay, ctx.mps_from_grid(lay, f0, 64, 1e-10), 0.04, 12)
    b = ctx.multi([lay], [(-1.0, 1.0)], [ctx.mps_from_grid(lay, f0, 64, 1e-10)], 0.04, 12)
    ra, rb = a.step(3), b.step(3)
    assert [r["field_energy"] for r in ra] == [r["field_energy"] for r in rb]
    for x, y in zip(a.state().cores(), b.state(0).cores()):
        np.testing.assert_array_equal(x, y)


def test_three_species(ctx):
    # electrons, ions and a positron-like light species of charge +1, mass 1
    lx = dict(nx=4, xmin=-math.pi / 0.1, xmax=math.pi / 0.1)
    lays = [I.Layout(lx["nx"], 6, lx["xmin"], lx["xmax"], -60.0, 60.0),
            I.Layout(lx["nx"], 5, lx["xmin"], lx["xmax"], -10.0, 10.0),
            I.Layout(lx["nx"], 5, lx["xmin"], lx["xmax"], -8.0, 8.0, I.INTERLEAVED)]
    x = lays[0].x()
    fs = [np.outer(1 + 0.05 * np.cos(0.1 * x), I.maxwellian(lays[0].v(), 1.0, 10.0)),
          np.outer(np.ones_like(x), I.maxwellian(lays[1].v(), 0.2)) * 0.5,
          np.outer(1 - 0.05 * np.cos(0.1 * x), I.maxwellian(lays[2].v(), 1.0)) * 0.5]
    run_pair(ctx, lays, fs, [(-1.0, 1.0), (1.0, 25.0, 0.02, 0.0, 0.2), (1.0, 1.0)], V_dt(lays[0]), 16, 2)


def test_invalid_arguments(ctx):
    from paper_2205_11990_gb300.vpmps import VpError
    le, li = I.buneman_layouts(4, 5, 4)
    fe, fi = I.buneman(le, li)
    ms = [ctx.mps_from_grid(le, fe, 16, 1e-10), ctx.mps_from_grid(li, fi, 16, 1e-10)]
    dt = V_dt(le)
    bad_x = I.Layout(4, 4, -math.pi / 0.1, 2 * math.pi / 0.1, li.vmin, li.vmax)
    cases = [([le, bad_x], FREE, dt, 1),                       # x grids differ
             ([le, li], [(-1.0, 1.0), (1.0, 0.0)], dt, 1),     # zero mass
             ([le, li], [(-1.0, 1.0, 0.1, 0.0, 0.0), (1.0, 25.0)], dt, 1),  # collisions without vth
             ([le, li], FREE, 2.0 * dt / 0.6, 7)]              # above the CFL limit of the electrons
    for lays, sp, step, code in cases:
        with pytest.raises(VpError) as e:
            ctx.multi(lays, sp, ms, step, 16)
        assert e.value.code == code
