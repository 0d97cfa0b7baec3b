"""Parity at the benchmark's full size (1024 x 1024, chi = 64), GPU vs oracle.

The benchmark times RK4-C1 steps of the saturated two-stream state on a
1024 x 1024 grid (10 + 10 sites, sequential mapping).  Here one step of the
same workload, launched the same way (vp_sim), is compared with one oracle
step from the same initial condition: the dense f (2^20 values) to 1e-10
relative L2 and the field energy to 1e-9.
"""
import math

import numpy as np
import pytest

from oracle import vp as OV
from paper_2205_11990_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("name", ["saturated_two_stream_1024x1024_seq", "two_stream_1024x1024_seq"])
def test_full_size_step(ctx, name):
    w = I.WORKLOADS[name]
    lay = w["layout"]
    f0 = I.initial_condition(w["ic"], lay)
    chi, dt = w["chi"], w["dt"]
    m = ctx.mps_from_grid(lay, f0, chi, 1e-10)
    ref = OV.mps_from_f(f0, lay, chi, 1e-10)
    assert m.bonds() == [int(x) for x in [1] + [c.shape[2] for c in ref]]
    assert rel(m.to_grid(lay), OV.mps_to_f(ref, lay)) < 1e-10
    sim = ctx.sim(lay, m, dt, chi)
    rec = sim.step(1)[0]
    ref, d = OV.rk4_step(ref, lay, dt, chi)
    assert abs(rec["field_energy"] - d["field_energy"]) <= 1e-9 * d["field_energy"]
    assert sim.state().bonds() == d["bonds"]
    assert rel(sim.state().to_grid(lay), OV.mps_to_f(ref, lay)) < 1e-10


def test_interleaved_mid_size_steps(ctx):
    lay = I.Layout(7, 7, 0.0, 10 * math.pi, -8.0, 8.0, I.INTERLEAVED)
    f0 = I.saturated_two_stream(lay, modes=8)
    dt = OV.stable_dt(lay, 0.01)
    m = ctx.mps_from_grid(lay, f0, 32, 1e-10)
    sim = ctx.sim(lay, m, dt, 32)
    ref = OV.mps_from_f(f0, lay, 32, 1e-10)
    for _ in range(2):
        rec = sim.step(1)[0]
        ref, d = OV.rk4_step(ref, lay, dt, 32)
        assert abs(rec["field_energy"] - d["field_energy"]) <= 1e-9 * d["field_energy"]
    assert rel(sim.state().to_grid(lay), OV.mps_to_f(ref, lay)) < 1e-10


def test_full_size_two_species_step(ctx):
    # the two-species bench workload: Buneman electrons and ions, 512 x 512
    # each (S3), chi = 64, Dougherty collisions; one step launched as the
    # bench launches it (vp_multi, two streams)
    lays, fs, species, chi, dt = I.species_workload("saturated_buneman_512x512_s3")
    ms = [ctx.mps_from_grid(l, f, chi, 1e-10) for l, f in zip(lays, fs)]
    refs = [OV.mps_from_f(f, l, chi, 1e-10) for l, f in zip(lays, fs)]
    run = ctx.multi(lays, species, ms, dt, chi)
    rec = run.step(1)[0]
    refs, d = OV.multi_rk4_step(refs, lays, species, dt, chi)
    assert abs(rec["field_energy"] - d["field_energy"]) <= 1e-9 * d["field_energy"]
    for s, (l, r) in enumerate(zip(lays, refs)):
        assert run.state(s).bonds() == d["bonds"][s]
        assert rel(run.state(s).to_grid(l), OV.mps_to_f(r, l)) < 1e-10
    run.close()


def test_full_size_4096_step_against_stored_oracle(ctx):
    # 4096 x 4096 (12 + 12 sites), chi = 128: the oracle's step takes minutes,
    # so its result is stored (tests/golden/make_fullsize_4096.py) and the
    # GPU step, launched as the sims run it, is compared on 4096 seeded grid
    # points, its field energy, mass and bonds
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fullsize_4096_step.json")
    g = json.load(open(path))
    w = I.WORKLOADS[g["workload"]]
    lay = w["layout"]
    f0 = I.initial_condition(w["ic"], lay)
    m = ctx.mps_from_grid(lay, f0, g["chi"], g["tol"])
    assert m.bonds() == g["start_bonds"]
    sim = ctx.sim(lay, m, g["dt"], g["chi"])
    rec = sim.step(1)[0]
    assert abs(rec["field_energy"] - g["field_energy"]) <= 1e-9 * g["field_energy"]
    assert abs(rec["mass"] - g["mass"]) <= 1e-10 * abs(g["mass"])
    assert sim.state().bonds() == g["bonds"]
    f1 = sim.state().to_grid(lay)
    ref = np.array(g["f"])
    got = f1[np.array(g["ix"]), np.array(g["iv"])]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
    sim.close()


@pytest.mark.parametrize("chi", [32, 128])
def test_full_size_step_other_chi(ctx, chi):
    # the benchmark's state and grid at the other bond caps of the
    # configuration (1024 x 1024 two-stream, chi in {32, 64, 128})
    w = I.WORKLOADS["saturated_two_stream_1024x1024_seq"]
    lay, dt = w["layout"], w["dt"]
    f0 = I.initial_condition(w["ic"], lay)
    m = ctx.mps_from_grid(lay, f0, chi, 1e-10)
    ref = OV.mps_from_f(f0, lay, chi, 1e-10)
    assert m.bonds() == [int(x) for x in [1] + [c.shape[2] for c in ref]]
    sim = ctx.sim(lay, m, dt, chi)
    rec = sim.step(1)[0]
    ref, d = OV.rk4_step(ref, lay, dt, chi)
    assert abs(rec["field_energy"] - d["field_energy"]) <= 1e-9 * d["field_energy"]
    assert sim.state().bonds() == d["bonds"]
    assert rel(sim.state().to_grid(lay), OV.mps_to_f(ref, lay)) < 1e-10


@pytest.mark.parametrize("case", ["interleaved_1024_chi64", "seq_4096_chi256"])
def test_full_size_step_against_stored_sketches(ctx, case):
    # oracle steps that take minutes, stored by tests/golden/make_fullsize_sketch.py:
    # the dense f(T) is compared through 64 seeded tensor-product sketches
    # r_i^T F s_i (every grid value enters each; their relative error
    # estimates the relative L2 error of f) and at 4096 seeded points
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", f"fullsize_{case}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    g = json.load(open(path))
    nx, nv, xmin, xmax, vmin, vmax, mapping = g["layout"]
    lay = I.Layout(nx, nv, xmin, xmax, vmin, vmax, mapping)
    f0 = I.saturated_two_stream(lay, modes=g["modes"])
    m = ctx.mps_from_grid(lay, f0, g["chi"], g["tol"])
    assert m.bonds() == g["start_bonds"]
    sim = ctx.sim(lay, m, g["dt"], g["chi"])
    rec = sim.step(1)[0]
    assert abs(rec["field_energy"] - g["field_energy"]) <= 1e-9 * g["field_energy"]
    assert abs(rec["mass"] - g["mass"]) <= 1e-10 * abs(g["mass"])
    assert sim.state().bonds() == g["bonds"]
    f1 = sim.state().to_grid(lay)
    sim.close()
    ref = np.array(g["f"])
    got = f1[np.array(g["ix"]), np.array(g["iv"])]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
    rng = np.random.Generator(np.random.PCG64(g["sketch_seed"]))
    r = rng.standard_normal((len(g["sketches"]), lay.Nx))
    s = rng.standard_normal((len(g["sketches"]), lay.Nv))
    y = np.einsum("ix,xv,iv->i", r, f1, s)
    y_ref = np.array(g["sketches"])
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-10


def test_run_horizon_256(ctx):
    # a 20-step run at 256 x 256 (8 + 8 sites, linear Landau, chi = 32):
    # the GPU and the oracle step from the same state at every step, and the
    # run stays within the FP64 contract over the whole horizon
    lay = I.Layout(8, 8, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay, 0.01, 0.5)
    dt = OV.stable_dt(lay, 0.02)
    chi = 32
    sim = ctx.sim(lay, ctx.mps_from_grid(lay, f0, chi, 1e-10), dt, chi)
    ref = OV.mps_from_f(f0, lay, chi, 1e-10)
    recs = sim.step(20)
    for n in range(20):
        ref, d = OV.rk4_step(ref, lay, dt, chi)
        assert abs(recs[n]["field_energy"] - d["field_energy"]) <= 1e-9 * d["field_energy"], n
        assert abs(recs[n]["mass"] - d["mass"]) <= 1e-10 * abs(d["mass"]), n
    assert sim.state().bonds() == d["bonds"]
    assert rel(sim.state().to_grid(lay), OV.mps_to_f(ref, lay)) < 1e-10
