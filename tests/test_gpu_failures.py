"""Failure detection in host-side forms (GPU): nothing here faults, traps or
hangs the device.

* A device-side wait that runs out: the context's wait limit is set to one
  clock, so the first wait of the grid QR (a published reflector that is not
  there yet) gives up at once; the call returns VP_ETIMEOUT and the context
  keeps working once the default limit is back.
* An allocator that fails: the context's allocator hook returns NULL, the
  step returns VP_ENOMEM, and the same context runs a new sim correctly once
  allocation works again.
* A poisoned request: a batch run whose initial state holds a NaN ends with
  VP_ENUMERIC while the runs beside it finish with their normal results.
"""
import math

import numpy as np
import pytest

from paper_2205_11990_gb300 import inputs as I

pytestmark = pytest.mark.gpu

VP_ENOMEM, VP_ETIMEOUT, VP_ENUMERIC = 2, 5, 6


@pytest.fixture(scope="module")
def vp():
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    return vpmps


def test_wait_limit_gives_timeout_and_context_recovers(vp):
    # 10 + 10 sites: the exact decomposition factors a 1024 x 1024 reshape,
    # too large for a cluster's shared memory, on the cooperative grid kernel
    lay = I.Layout(10, 10, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ)
    f0 = I.two_stream(lay)
    ctx = vp.Context()
    ref = ctx.mps_from_grid(lay, f0, 64, 1e-10).to_grid(lay)
    ctx.set_wait_limit(1)
    with pytest.raises(vp.VpError) as e:
        ctx.mps_from_grid(lay, f0, 64, 1e-10)
    assert e.value.code == VP_ETIMEOUT
    ctx.set_wait_limit(0)  # default limit again
    again = ctx.mps_from_grid(lay, f0, 64, 1e-10).to_grid(lay)
    assert np.array_equal(again, ref)
    ctx.close()


def test_allocation_failure_gives_enomem_and_context_recovers(vp):
    lay = I.Layout(6, 6, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    f0 = I.landau(lay)
    dt = 0.5 * (lay.xmax - lay.xmin) / lay.Nx / lay.vmax
    ref_ctx = vp.Context()
    ref = ref_ctx.sim(lay, ref_ctx.mps_from_grid(lay, f0, 16, 1e-10), dt, 16, streams=1)
    ref.step(2)
    f_ref = ref.state().to_grid(lay)
    ref_ctx.close()

    ctx = vp.Context()
    sim = ctx.sim(lay, ctx.mps_from_grid(lay, f0, 16, 1e-10), dt, 16, streams=1)
    ctx.set_alloc_budget(0)  # every further device allocation of this context fails
    with pytest.raises(vp.VpError) as e:
        sim.step(1)
    assert e.value.code == VP_ENOMEM
    sim.close()
    ctx.set_alloc_budget(None)
    sim2 = ctx.sim(lay, ctx.mps_from_grid(lay, f0, 16, 1e-10), dt, 16, streams=1)
    sim2.step(2)
    assert np.array_equal(sim2.state().to_grid(lay), f_ref)
    ctx.close()


def test_nan_request_fails_alone_in_a_batch(vp):
    ctx = vp.Context()
    reqs = []
    for i, nb in enumerate((5, 6, 5)):
        lay = I.Layout(nb, nb, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ if i % 2 == 0 else I.INTERLEAVED)
        dt = 0.5 * (lay.xmax - lay.xmin) / lay.Nx / lay.vmax
        reqs.append((lay, I.landau(lay, 0.05, 0.5), dt))
    bad = reqs[1][1].copy()
    bad[3, 7] = np.nan
    b = vp.Batch(ctx, 3, 8 << 30)
    ids = [b.submit(lay, f0 if i != 1 else bad, dt, 3, 16, keep_f=True) for i, (lay, f0, dt) in enumerate(reqs)]
    b.start()
    b.wait()
    res = {r["id"]: r for r in b.poll()}
    assert res[ids[1]]["status"] == VP_ENUMERIC
    for i in (0, 2):
        assert res[ids[i]]["status"] == 0
        lay, f0, dt = reqs[i]
        alone = vp.Batch(ctx, 1, 8 << 30)
        aid = alone.submit(lay, f0, dt, 3, 16, keep_f=True)
        alone.start()
        alone.wait()
        alone.poll()
        assert np.array_equal(b.records(ids[i], want_f=True)[2], alone.records(aid, want_f=True)[2])
        alone.close()
    b.close()
    ctx.close()
