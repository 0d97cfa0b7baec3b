"""Batched / served runs (vp_batch_*) on one GPU (GPU).

Each run in a mix must give the same result as the same run alone (its own
buffers, stream and deterministic arithmetic), admission must respect the
memory budget, and oversized requests are refused.
"""
import math

import numpy as np
import pytest

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


def mixed_requests():
    reqs = []
    rng = np.random.Generator(np.random.PCG64(0))
    for i in range(6):
        nb = int(rng.integers(5, 8))
        mapping = I.SEQ if i % 2 == 0 else I.INTERLEAVED
        if i % 3 == 0:
            k = float(rng.uniform(0.3, 0.6))
            lay = I.Layout(nb, nb, 0.0, 2 * math.pi / k, -6.0, 6.0, mapping)
            f0 = I.landau(lay, float(rng.uniform(1e-3, 0.3)), k)
        else:
            k = 0.3
            lay = I.Layout(nb, nb, 0.0, 2 * math.pi / k, -8.0, 8.0, mapping)
            f0 = I.bump_on_tail(lay, 1e-2, k)
        dx = (lay.xmax - lay.xmin) / lay.Nx
        dt = 0.5 * dx / lay.vmax
        chi = int(rng.choice([8, 16, 32]))
        reqs.append((lay, f0, dt, int(rng.integers(3, 7)), chi))
    return reqs


def test_mix_equals_alone_and_admission(ctx):
    from paper_2205_11990_gb300 import vpmps
    reqs = mixed_requests()
    budget = 64 << 30
    mixed = vpmps.Batch(ctx, 4, budget)
    ids = [mixed.submit(lay, f0, dt, n, chi, keep_f=True) for (lay, f0, dt, n, chi) in reqs]
    mixed.start()
    mixed.wait()
    res = {r["id"]: r for r in mixed.poll()}
    assert sorted(res) == sorted(ids) and all(r["status"] == 0 for r in res.values())
    # the runs stepped on the workers' contexts, whose launches the batch counts
    assert mixed.kernel_launches > 0
    for rid, (lay, f0, dt, n, chi) in zip(ids, reqs):
        recs_mix, step_ms, f_mix = mixed.records(rid, want_f=True)
        alone = vpmps.Batch(ctx, 1, budget)
        aid = alone.submit(lay, f0, dt, n, chi, keep_f=True)
        alone.start()
        alone.wait()
        recs_alone, _, f_alone = alone.records(aid, want_f=True)
        alone.close()
        assert np.linalg.norm(f_mix - f_alone) <= 1e-12 * np.linalg.norm(f_alone)
        assert [r["max_bond"] for r in recs_mix] == [r["max_bond"] for r in recs_alone]
        assert len(step_ms) == n and np.all(step_ms > 0)
    mixed.close()


def test_budget_serialises_and_rejects(ctx):
    from paper_2205_11990_gb300 import vpmps
    lay = I.Layout(5, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay, 0.1, 0.5)
    fp = vpmps.footprint_bytes(lay, 16)
    b = vpmps.Batch(ctx, 4, int(1.5 * fp))  # room for one run at a time
    ids = [b.submit(lay, f0, 0.02, 3, 16) for _ in range(3)]
    b.start()
    b.wait()
    res = sorted(b.poll(), key=lambda r: r["id"])
    assert [r["id"] for r in res] == ids
    # one at a time: each run starts after the previous one ended
    assert res[1]["queue_ms"] >= res[0]["run_ms"] * 0.9
    big = I.Layout(10, 10, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    with pytest.raises(vpmps.VpError) as e:
        b.submit(big, np.zeros((big.Nx, big.Nv)), 0.002, 1, 64)
    assert e.value.code == 3
    b.close()


def test_lockstep_mix_equals_alone(ctx):
    # continuous batching in lockstep: the same mix through one group
    from paper_2205_11990_gb300 import vpmps
    reqs = mixed_requests()
    budget = 64 << 30
    mixed = vpmps.Batch(ctx, 8, budget, lockstep=True)
    ids = [mixed.submit(lay, f0, dt, n, chi, keep_f=True) for (lay, f0, dt, n, chi) in reqs]
    mixed.start()
    mixed.wait()
    res = {r["id"]: r for r in mixed.poll()}
    assert sorted(res) == sorted(ids) and all(r["status"] == 0 for r in res.values())
    for rid, (lay, f0, dt, n, chi) in zip(ids, reqs):
        recs_mix, step_ms, f_mix = mixed.records(rid, want_f=True)
        alone = vpmps.Batch(ctx, 1, budget)
        aid = alone.submit(lay, f0, dt, n, chi, keep_f=True)
        alone.start()
        alone.wait()
        recs_alone, _, f_alone = alone.records(aid, want_f=True)
        alone.close()
        assert np.array_equal(f_mix, f_alone)
        assert recs_mix == recs_alone
        assert len(step_ms) == n and np.all(step_ms > 0)
    mixed.close()


def test_lockstep_admission_respects_budget(ctx):
    # runs that overlap in time never hold more than the budget, and a
    # request submitted while others run joins the group as room frees up
    import time
    from paper_2205_11990_gb300 import vpmps
    lays = [I.Layout(nb, nb, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ) for nb in (4, 5, 5, 4, 5, 4)]
    fps = [vpmps.footprint_bytes(l, 16) for l in lays]
    budget = int(2.2 * max(fps))  # about two runs at a time
    b = vpmps.Batch(ctx, 8, budget, lockstep=True)
    ids = [b.submit(l, I.landau(l, 0.1, 0.5), 0.02, 4, 16) for l in lays[:5]]
    t_submit = time.perf_counter()
    b.start()
    time.sleep(0.05)
    late = b.submit(lays[5], I.landau(lays[5], 0.1, 0.5), 0.02, 4, 16)
    t_late = (time.perf_counter() - t_submit) * 1e3
    b.wait()
    res = {r["id"]: r for r in b.poll()}
    assert all(r["status"] == 0 for r in res.values()) and len(res) == 6
    iv = []
    for rid, fp in zip(ids + [late], fps):
        r = res[rid]
        t0 = (t_late if rid == late else 0.0) + r["queue_ms"]
        iv.append((t0, t0 + r["run_ms"], fp))
    for t0, _, _ in iv:  # held memory at each start
        held = sum(fp for a, e, fp in iv if a <= t0 < e)
        assert held <= budget
    b.close()


def test_lockstep_nan_request_fails_alone(ctx):
    from paper_2205_11990_gb300 import vpmps
    lay = I.Layout(5, 5, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay, 0.1, 0.5)
    bad = f0.copy()
    bad[5, 9] = np.nan
    b = vpmps.Batch(ctx, 4, 8 << 30, lockstep=True)
    ids = [b.submit(lay, x, 0.02, 3, 16, keep_f=True) for x in (f0, bad, f0)]
    b.start()
    b.wait()
    res = {r["id"]: r for r in b.poll()}
    assert res[ids[1]]["status"] == 6
    assert res[ids[0]]["status"] == res[ids[2]]["status"] == 0
    assert np.array_equal(b.records(ids[0], want_f=True)[2], b.records(ids[2], want_f=True)[2])
    b.close()
