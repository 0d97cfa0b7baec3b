"""Grouped interleaved (IG) ordering through the C ABI, GPU vs the oracle's
d = 4 implementation: f to 1e-10 relative L2, field energy to 1e-9, and the
bonds between pairs equal to the oracle's bonds."""
import math

import numpy as np
import pytest

from oracle import grouped as G
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


def pair_bonds(bonds):
    return bonds[0::2]


@pytest.mark.parametrize("chi,tol", [(1 << 20, 1e-10), (8, 1e-10), (16, 1e-6)])
def test_grouped_create(ctx, chi, tol):
    lay = I.Layout(5, 5, 0.0, 10 * math.pi, -8.0, 8.0, I.GROUPED)
    f = I.saturated_two_stream(lay, modes=8)
    m = ctx.mps_from_grid(lay, f, chi, tol)
    ref = G.mps_from_f(f, lay, chi, tol)
    assert pair_bonds(m.bonds()) == G.bonds(ref)
    assert rel(m.to_grid(lay), G.mps_to_f(ref, lay)) < 1e-10


@pytest.mark.parametrize("chi", [12, 64])
def test_grouped_steps_match_oracle(ctx, chi):
    lay = I.Layout(5, 5, 0.0, 10 * math.pi, -8.0, 8.0, I.GROUPED)
    f = I.saturated_two_stream(lay, modes=8)
    dt = 0.02
    sim = ctx.sim(lay, ctx.mps_from_grid(lay, f, chi, 1e-10), dt, chi)
    ref = G.mps_from_f(f, lay, chi)
    for _ in range(3):
        rec = sim.step(1)[0]
        ref, d = G.rk4_step(ref, lay, dt, chi)
        assert abs(rec["field_energy"] - d["field_energy"]) <= 1e-9 * d["field_energy"]
        assert pair_bonds(sim.state().bonds()) == d["bonds"]
    assert rel(sim.state().to_grid(lay), G.mps_to_f(ref, lay)) < 1e-10


def test_grouped_needs_equal_bits(ctx):
    from paper_2205_11990_gb300.vpmps import VpError
    lay = I.Layout(5, 4, 0.0, 10 * math.pi, -8.0, 8.0, I.GROUPED)
    with pytest.raises(VpError) as e:
        ctx.mps_from_grid(lay, np.ones((lay.Nx, lay.Nv)), 8, 1e-10)
    assert e.value.code == 1
