"""vp_poisson_noalloc against vp_poisson (GPU).

vp_poisson_noalloc serves callers that cannot allocate device memory (and so
cannot create a context): it keeps its scratch in a static device array.  It
must give the same field and field energy as the context-based vp_poisson,
call after call, since the shared scratch keeps the previous call's data.
This file sorts last so that a run stopping at its first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_poisson_matches_context_poisson_twice():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    ctx = vpmps.Context()
    lib = vpmps.load()
    rng = np.random.default_rng(11)
    # N below the kernel's block size (nx = 1, 3, 7: most threads get empty
    # scan chunks), the step's sizes, and the capacity edge nx = 14 (the
    # field fills the whole static array, next to the energy and mass slots);
    # every size twice in a row (the shared scratch keeps the last call's data)
    sizes = [(1, 0.5), (3, 0.2), (7, 0.05), (10, 0.03), (12, 0.011), (14, 0.004)]
    for call, (nx, dx) in enumerate([s for s in sizes for _ in range(2)]):
        rho = torch.tensor(1.0 + 0.2 * rng.standard_normal(1 << nx), device="cuda", dtype=torch.float64)
        E_ref, we_ref = ctx.poisson(rho, nx, dx)
        E = torch.full((1 << nx,), float("nan"), device="cuda", dtype=torch.float64)
        we, mass = ctypes.c_double(), ctypes.c_double()
        code = lib.vp_poisson_noalloc(ctypes.c_void_p(ctx.stream.cuda_stream), ctypes.c_void_p(rho.data_ptr()), nx, dx,
                                      ctypes.c_void_p(E.data_ptr()), ctypes.byref(we), ctypes.byref(mass))
        assert code == 0, call
        got, ref = E.cpu().numpy(), E_ref.cpu().numpy()
        # nx = 1 has E = 0 up to rounding: an absolute floor at the scale of
        # the rounding of the prefix sums (dx N max|rho|) times 1e-14
        floor = 1e-14 * dx * (1 << nx) * float(rho.abs().max())
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref) + floor * np.sqrt(1 << nx), call
        assert abs(we.value - we_ref) <= 1e-12 * we_ref + floor * floor * (1 << nx) * dx, call
        assert abs(mass.value - float(rho.sum()) * dx) <= 1e-12 * abs(mass.value), call
    # sizes beyond the static scratch are refused
    rho = torch.ones(1 << 15, device="cuda", dtype=torch.float64)
    assert lib.vp_poisson_noalloc(ctypes.c_void_p(ctx.stream.cuda_stream), ctypes.c_void_p(rho.data_ptr()), 15, 0.1,
                                  ctypes.c_void_p(rho.data_ptr()), None, None) == 3
    ctx.close()
