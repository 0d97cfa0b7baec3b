"""Lockstep groups of simulations (vp_group_*) through the C ABI (GPU).

A group step runs every member's RK4-C1 step with batched launches (one
launch per sweep position for all members).  Each member must come out bit
for bit as the same sim stepped alone with vp_step, whatever the other
members are (grid bits, mapping, chi, dt, contraction mode), and the group's
result must match the oracle within the FP64 contract.  A member that fails
(a NaN in its state) stops alone.
"""
import math

import numpy as np
import pytest

from oracle import vp as OV
from paper_2205_11990_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F_TOL = 1e-10
WE_TOL = 1e-9
VP_EINVAL, VP_ENUMERIC = 1, 6


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


def member_cases():
    """A mix of members: grid bits 4..7, all five orderings, chi 8..32,
    Landau / two-stream / bump-on-tail, FP64 and FP32 contractions."""
    cases = []
    rng = np.random.Generator(np.random.PCG64(5))
    maps = [I.SEQ, I.INTERLEAVED, I.SEQ_S2, I.SEQ_S3, I.GROUPED, I.SEQ, I.INTERLEAVED]
    for i, mp in enumerate(maps):
        nb = int(rng.integers(4, 8))
        if i % 3 == 0:
            lay = I.Layout(nb, nb, 0.0, 4 * math.pi, -6.0, 6.0, mp)
            f0 = I.landau(lay, float(rng.uniform(0.01, 0.3)), 0.5)
        elif i % 3 == 1:
            lay = I.Layout(nb, nb, 0.0, 10 * math.pi, -8.0, 8.0, mp)
            f0 = I.two_stream(lay)
        else:
            lay = I.Layout(nb, nb, 0.0, 2 * math.pi / 0.3, -8.0, 8.0, mp)
            f0 = I.bump_on_tail(lay, 1e-2, 0.3)
        dt = 0.5 * (lay.xmax - lay.xmin) / lay.Nx / lay.vmax
        chi = int(rng.choice([8, 16, 32]))
        prec = 1 if i == 5 else 0  # one member with FP32 contractions
        cases.append((lay, f0, dt, chi, prec))
    return cases


def test_group_equals_alone(ctx):
    cases = member_cases()
    grp = ctx.group(len(cases))
    gsims, alone = [], []
    for lay, f0, dt, chi, prec in cases:
        s = ctx.sim(lay, ctx.mps_from_grid(lay, f0, chi, 1e-10), dt, chi, streams=1, precision=prec)
        grp.add(s)
        gsims.append(s)
        alone.append(ctx.sim(lay, ctx.mps_from_grid(lay, f0, chi, 1e-10), dt, chi, precision=prec))
    for step in range(3):
        recs, status = grp.step()
        assert status == [0] * len(cases)
        for i, (lay, *_rest) in enumerate(cases):
            ra = alone[i].step(1)[0]
            assert recs[i] == ra, (step, i)
            assert gsims[i].state().bonds() == alone[i].state().bonds()
            assert np.array_equal(gsims[i].state().to_grid(lay), alone[i].state().to_grid(lay)), (step, i)
            assert np.array_equal(gsims[i].entropy(), alone[i].entropy())
    grp.close()


def test_group_matches_oracle(ctx):
    cases = [
        (I.Layout(5, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ), "landau", 0.02, 16),
        (I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.INTERLEAVED), "landau", 0.05, 8),
        (I.Layout(5, 6, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ_S3), "two_stream", 0.05, 12),
    ]
    grp = ctx.group(4)
    sims, refs = [], []
    for lay, ic, dt, chi in cases:
        f0 = I.landau(lay, 0.3, 0.5) if ic == "landau" else I.initial_condition(ic, lay)
        s = ctx.sim(lay, ctx.mps_from_grid(lay, f0, chi, 1e-10), dt, chi, streams=1)
        grp.add(s)
        sims.append(s)
        refs.append(OV.mps_from_f(f0, lay, chi, 1e-10))
    for step in range(2):
        recs, status = grp.step()
        assert status == [0, 0, 0]
        for i, (lay, ic, dt, chi) in enumerate(cases):
            refs[i], d = OV.rk4_step(refs[i], lay, dt, chi)
            assert abs(recs[i]["field_energy"] - d["field_energy"]) <= WE_TOL * d["field_energy"]
            assert abs(recs[i]["mass"] - d["mass"]) <= F_TOL * abs(d["mass"])
            assert sims[i].state().bonds() == d["bonds"]
            assert rel(sims[i].state().to_grid(lay), OV.mps_to_f(refs[i], lay)) < F_TOL
            np.testing.assert_allclose(sims[i].entropy(), d["entropy"], rtol=1e-8, atol=1e-12)
    grp.close()


def test_member_failure_is_isolated(ctx):
    lay = I.Layout(5, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay, 0.1, 0.5)
    dt = 0.02
    good = ctx.mps_from_grid(lay, f0, 16, 1e-10)
    # poison one member's state: its cores are built from a NaN-bearing grid
    cores = good.cores()
    cores[3] = cores[3].copy()
    cores[3][0, 0, 0] = np.nan
    bad = ctx.mps_from_cores(cores)
    grp = ctx.group(3)
    sa = ctx.sim(lay, good, dt, 16, streams=1)
    sb = ctx.sim(lay, bad, dt, 16, streams=1)
    sc = ctx.sim(lay, ctx.mps_from_grid(lay, f0, 16, 1e-10), dt, 16, streams=1)
    for s in (sa, sb, sc):
        grp.add(s)
    ref = ctx.sim(lay, ctx.mps_from_grid(lay, f0, 16, 1e-10), dt, 16)
    for _ in range(2):
        recs, status = grp.step()
        ra = ref.step(1)[0]
        assert status[1] == VP_ENUMERIC
        assert status[0] == status[2] == 0
        assert recs[0] == ra and recs[2] == ra
    assert np.array_equal(sa.state().to_grid(lay), ref.state().to_grid(lay))
    grp.remove(sb)
    assert len(grp) == 2
    recs, status = grp.step()
    assert status == [0, 0]
    grp.close()


def test_many_members_span_several_launch_packs(ctx):
    # 40 members (two compressions each: 80 problems per sweep position,
    # three parameter packs of at most 32 per batched launch)
    grp = ctx.group(40)
    sims, alone, lays = [], [], []
    for i in range(40):
        nb = 4 + i % 2
        lay = I.Layout(nb, nb, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ if i % 3 else I.INTERLEAVED)
        f0 = I.landau(lay, 0.01 + 0.005 * i, 0.5)
        s = ctx.sim(lay, ctx.mps_from_grid(lay, f0, 8, 1e-10), 0.02, 8, streams=1)
        grp.add(s)
        sims.append(s)
        alone.append(ctx.sim(lay, ctx.mps_from_grid(lay, f0, 8, 1e-10), 0.02, 8))
        lays.append(lay)
    recs, status = grp.step()
    assert status == [0] * 40
    for i in range(40):
        assert recs[i] == alone[i].step(1)[0], i
        assert np.array_equal(sims[i].state().to_grid(lays[i]), alone[i].state().to_grid(lays[i])), i
    grp.close()


def test_ineligible_members_refused(ctx):
    from paper_2205_11990_gb300.vpmps import VpError
    lay = I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay)
    grp = ctx.group(1)
    for kw in (dict(streams=2), dict(streams=1, level=2), dict(streams=1, precision=2), dict(streams=1, tol=0.0),
               dict(streams=1, compression=1)):
        s = ctx.sim(lay, ctx.mps_from_grid(lay, f0, 8, 1e-10), 0.05, 8, **kw)
        with pytest.raises(VpError) as e:
            grp.add(s)
        assert e.value.code == VP_EINVAL, kw
        s.close()
    s = ctx.sim(lay, ctx.mps_from_grid(lay, f0, 8, 1e-10), 0.05, 8, streams=1)
    grp.add(s)
    with pytest.raises(VpError):
        grp.add(ctx.sim(lay, ctx.mps_from_grid(lay, f0, 8, 1e-10), 0.05, 8, streams=1))  # full
    grp.close()


def test_batched_creation_equals_mps_create(ctx):
    cases = member_cases()
    items = [(lay, f0, chi, 1e-10) for lay, f0, dt, chi, prec in cases]
    bad = cases[0][1].copy()
    bad[1, 2] = np.nan
    items.append((cases[0][0], bad, 8, 1e-10))             # NaN grid: fails alone
    items.append((cases[1][0], cases[1][1], 8, 0.0))       # exact mode: not batched
    grp = ctx.group(8)
    ms, status = grp.create_mps(items)
    assert status[:-2] == [0] * len(cases) and status[-2] == VP_ENUMERIC and status[-1] == VP_EINVAL
    assert ms[-1] is None and ms[-2] is None
    for (lay, f0, chi, tol), m in zip(items[:-2], ms[:-2]):
        ref = ctx.mps_from_grid(lay, f0, chi, tol)
        assert m.bonds() == ref.bonds()
        assert all(np.array_equal(a, b) for a, b in zip(m.cores(), ref.cores()))
    grp.close()


def test_group_equals_alone_with_grid_factors(ctx):
    # 9 + 9 interleaved members: the tolerance-only stage compressions carry
    # bonds of r W (W ~ 12 + 3 D_F) whose factors exceed a cluster's shared
    # memory and run on the cooperative grid kernel, several problems per launch
    cases = []
    for amp, chi, ic in ((0.3, 16, "landau"), (0.05, 32, "bump"), (0.2, 24, "landau")):
        if ic == "landau":
            lay = I.Layout(9, 9, 0.0, 4 * math.pi, -6.0, 6.0, I.INTERLEAVED)
            f0 = I.landau(lay, amp, 0.5)
        else:
            lay = I.Layout(9, 9, 0.0, 2 * math.pi / 0.3, -8.0, 8.0, I.INTERLEAVED)
            f0 = I.bump_on_tail(lay, amp, 0.3)
        cases.append((lay, f0, 0.6 * (lay.xmax - lay.xmin) / lay.Nx / lay.vmax, chi))
    grp = ctx.group(len(cases))
    gs, al = [], []
    for lay, f0, dt, chi in cases:
        s = ctx.sim(lay, ctx.mps_from_grid(lay, f0, chi, 1e-10), dt, chi, streams=1)
        grp.add(s)
        gs.append(s)
        al.append(ctx.sim(lay, ctx.mps_from_grid(lay, f0, chi, 1e-10), dt, chi))
    recs, status = grp.step()
    assert status == [0] * len(cases)
    for i, (lay, *_r) in enumerate(cases):
        assert recs[i] == al[i].step(1)[0], i
        assert np.array_equal(gs[i].state().to_grid(lay), al[i].state().to_grid(lay)), i
    grp.close()


def test_lockstep_stepping_mode_equals_two_streams(ctx):
    # vp_step with streams = 0 runs a one-member lockstep group: the same
    # records, state and entropies as the two-stream path, and the flop count
    cases = member_cases()[:4]
    for lay, f0, dt, chi, prec in cases:
        a = ctx.sim(lay, ctx.mps_from_grid(lay, f0, chi, 1e-10), dt, chi, streams=0, precision=prec)
        b = ctx.sim(lay, ctx.mps_from_grid(lay, f0, chi, 1e-10), dt, chi, streams=2, precision=prec)
        assert a.step(2) == b.step(2)
        assert np.array_equal(a.state().to_grid(lay), b.state().to_grid(lay))
        assert np.array_equal(a.entropy(), b.entropy())
        assert abs(a.flops - b.flops) <= 1e-9 * b.flops
        a.close()
        b.close()
