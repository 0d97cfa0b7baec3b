"""Host-side entry points of the C ABI that need no device (CPU).

The argument checks that include/vpmps.h documents for NULL handles, and the
admission footprint of vp_footprint_bytes (pure host arithmetic): positive
and growing with the bond cap and the grid.
"""
import math

import pytest

VP_EINVAL = 1


@pytest.fixture(scope="module")
def lib():
    from paper_2205_11990_gb300 import build as B
    from paper_2205_11990_gb300 import vpmps
    try:
        B.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))
    return vpmps.load()


def test_null_handles(lib):
    assert lib.vp_kernel_launches(None) == 0
    assert lib.vp_batch_kernel_launches(None) == 0
    assert lib.vp_group_size(None) == -1
    assert lib.vp_batch_set_lockstep(None, 1) == VP_EINVAL
    assert lib.vp_ctx_destroy(None) == VP_EINVAL
    assert lib.vp_group_destroy(None) == VP_EINVAL
    assert lib.vp_batch_destroy(None) == VP_EINVAL
    assert lib.vp_last_error(None) == b"null context"
    assert lib.vp_footprint_bytes(None, None) == 0
    assert lib.mps_file_info(None, None, None, None) == VP_EINVAL


def test_footprint_grows_with_chi_and_grid(lib):
    from paper_2205_11990_gb300 import inputs as I
    from paper_2205_11990_gb300 import vpmps

    def fp(bits, chi):
        lay = I.Layout(bits, bits, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
        return vpmps.footprint_bytes(lay, chi)

    for bits in (6, 9, 12):
        by_chi = [fp(bits, chi) for chi in (16, 32, 64, 128)]
        assert all(b > 0 for b in by_chi)
        assert by_chi == sorted(by_chi), (bits, by_chi)
    for chi in (16, 64):
        by_grid = [fp(bits, chi) for bits in (6, 8, 10, 12)]
        assert by_grid == sorted(by_grid) and by_grid[0] < by_grid[-1], (chi, by_grid)
