"""MPS checkpoint files (mps_save / mps_load) through the C ABI (GPU).

The file is parsed here with numpy alone, independently of the library, so
the documented layout is checked, not just the round trip.
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


def parse(path):
    raw = open(path, "rb").read()
    assert raw[:8] == b"VPMPS01\0"
    n, reserved = np.frombuffer(raw[8:16], dtype="<i4")
    assert reserved == 0
    ranks = np.frombuffer(raw[16:16 + 4 * (n + 1)], dtype="<i4")
    off = (16 + 4 * (n + 1) + 7) // 8 * 8
    assert raw[16 + 4 * (n + 1):off] == b"\0" * (off - 16 - 4 * (n + 1))
    flat = np.frombuffer(raw[off:], dtype="<f8")
    sizes = [ranks[k] * 2 * ranks[k + 1] for k in range(n)]
    assert flat.size == sum(sizes)
    cores, o = [], 0
    for k, s in enumerate(sizes):
        cores.append(flat[o:o + s].reshape(ranks[k], 2, ranks[k + 1]))
        o += s
    return int(n), [int(r) for r in ranks], cores


def test_save_layout_and_round_trip(ctx, tmp_path):
    lay = I.Layout(6, 7, 0.0, 10 * math.pi, -8.0, 8.0, I.INTERLEAVED)
    m = ctx.mps_from_grid(lay, I.saturated_two_stream(lay, modes=8), 24, 1e-10)
    path = str(tmp_path / "f.mps")
    m.save(path)
    n, ranks, cores = parse(path)
    assert n == m.n and ranks == m.bonds()
    for a, b in zip(cores, m.cores()):
        assert np.array_equal(a, b)
    m2 = ctx.mps_load(path)
    assert m2.bonds() == m.bonds()
    for a, b in zip(m2.cores(), m.cores()):
        assert np.array_equal(a, b)
    assert np.array_equal(m2.to_grid(lay), m.to_grid(lay))


def test_resume_from_checkpoint(ctx, tmp_path):
    # 3 steps, checkpoint, reload, 2 more steps == 5 steps without a break
    lay = I.Layout(6, 6, 0.0, 10 * math.pi, -8.0, 8.0, I.SEQ)
    f0 = I.saturated_two_stream(lay, modes=8)
    chi, dt = 24, 0.02
    m = ctx.mps_from_grid(lay, f0, chi, 1e-10)
    sim = ctx.sim(lay, m, dt, chi)
    ref = sim.step(5)
    f_ref = sim.state().to_grid(lay)
    sim.close()
    m = ctx.mps_from_grid(lay, f0, chi, 1e-10)
    sim = ctx.sim(lay, m, dt, chi)
    first = sim.step(3)
    path = str(tmp_path / "ckpt.mps")
    sim.state().save(path)
    sim.close()
    sim = ctx.sim(lay, ctx.mps_load(path), dt, chi)
    rest = sim.step(2)
    f_res = sim.state().to_grid(lay)
    sim.close()
    we = np.array([r["field_energy"] for r in first + rest])
    we_ref = np.array([r["field_energy"] for r in ref])
    assert np.max(np.abs(we - we_ref) / we_ref) < 1e-12
    assert np.linalg.norm(f_res - f_ref) / np.linalg.norm(f_ref) < 1e-12


def test_malformed_files_rejected(ctx, tmp_path):
    from paper_2205_11990_gb300.vpmps import VpError
    lay = I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
    m = ctx.mps_from_grid(lay, I.landau(lay), 8, 1e-10)
    good = str(tmp_path / "good.mps")
    m.save(good)
    raw = open(good, "rb").read()
    cases = {
        "missing": None,
        "magic": b"XPMPS01\0" + raw[8:],
        "truncated": raw[:-8],
        "trailing": raw + b"\0" * 8,
        "rank": raw[:16] + np.array([2], dtype="<i4").tobytes() + raw[20:],
        "inflated": raw[:20] + np.array([1 << 20], dtype="<i4").tobytes() + raw[24:],
    }
    for name, data in cases.items():
        p = str(tmp_path / f"{name}.mps")
        if data is not None:
            open(p, "wb").write(data)
        with pytest.raises(VpError) as e:
            ctx.mps_load(p)
        assert e.value.code == 9, name
