"""Checkpoint headers are validated on the host before anything is allocated
(mps_file_info through the C ABI; no device needed)."""
import os

import numpy as np
import pytest

MAGIC = b"VPMPS01\0"


def _lib_or_skip():
    from paper_2205_11990_gb300 import build as B
    try:
        B.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))
    from paper_2205_11990_gb300 import vpmps
    return vpmps


def _file(path, n, ranks, payload_elems, reserved=0):
    head = MAGIC + np.array([n, reserved], dtype="<i4").tobytes() + np.array(ranks, dtype="<i4").tobytes()
    head += b"\0" * ((-len(head)) % 8)
    with open(path, "wb") as f:
        f.write(head + np.arange(payload_elems, dtype="<f8").tobytes())
    return str(path)


def test_valid_header(tmp_path):
    vp = _lib_or_skip()
    ranks = [1, 2, 4, 2, 1]
    elems = sum(ranks[k] * 2 * ranks[k + 1] for k in range(4))
    n, r, e = vp.mps_file_info(_file(tmp_path / "ok.mps", 4, ranks, elems))
    assert (n, r, e) == (4, ranks, elems)


def test_inflated_ranks_rejected_before_allocation(tmp_path):
    # ranks claiming ~2^41 doubles per core in a file of a few hundred bytes:
    # the size check rejects it (VP_EIO), nothing of that size is allocated
    vp = _lib_or_skip()
    p = _file(tmp_path / "big.mps", 4, [1, 2, 1 << 20, 1 << 20, 1], 8)
    with pytest.raises(vp.VpError) as e:
        vp.mps_file_info(p)
    assert e.value.code == 9


@pytest.mark.parametrize("case", ["magic", "n", "reserved", "boundary", "rank0", "truncated", "trailing", "missing"])
def test_malformed_headers(tmp_path, case):
    vp = _lib_or_skip()
    ranks = [1, 2, 2, 1]
    elems = sum(ranks[k] * 2 * ranks[k + 1] for k in range(3))
    p = str(tmp_path / f"{case}.mps")
    if case == "missing":
        pass
    elif case == "n":
        _file(p, 70, ranks, elems)
    elif case == "reserved":
        _file(p, 3, ranks, elems, reserved=1)
    elif case == "boundary":
        _file(p, 3, [2, 2, 2, 1], elems)
    elif case == "rank0":
        _file(p, 3, [1, 0, 2, 1], elems)
    elif case == "truncated":
        _file(p, 3, ranks, elems - 1)
    elif case == "trailing":
        _file(p, 3, ranks, elems + 1)
    else:
        _file(p, 3, ranks, elems)
        raw = open(p, "rb").read()
        open(p, "wb").write(b"X" + raw[1:])
    with pytest.raises(vp.VpError) as e:
        vp.mps_file_info(p)
    assert e.value.code == 9
    assert not os.path.exists(p) or os.path.getsize(p) < 4096
