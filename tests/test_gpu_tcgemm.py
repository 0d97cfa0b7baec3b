"""Dense contractions through vp_gemm in every precision mode (GPU).

The tensor-core modes (TF32, BF16, split TF32x3: tcgen05 MMA with FP32
accumulation in tensor memory, operands staged by TMA) are checked two ways:
small-integer operands, which every mode represents exactly and whose FP32
sums are exact, must give the FP64 product bit for bit (any tile, swizzle or
descriptor mistake breaks this); random operands must stay within the
rounding bound of the mode.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (128, 64, 32), (200, 77, 45), (300, 130, 300), (129, 129, 257), (64, 200, 96),
          # the FP64 plan's other branches: 64 x 64 tiles without a split (>= one
          # tile per SM), K <= 16 (no split), K just above a slice multiple, and a
          # narrow output split into many K slices
          (1024, 1000, 40), (7, 9, 16), (50, 60, 17), (33, 31, 500)]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    c = vpmps.Context()
    yield c
    c.close()


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("shape", SHAPES)
def test_integer_operands_exact(ctx, prec, shape):
    M, N, K = shape
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float64)
    B = rng.integers(-8, 9, size=(K, N)).astype(np.float64)
    for alpha in (1.0, -0.5):
        C = ctx.gemm(dev(A), dev(B), alpha, precision=prec).cpu().numpy()
        assert np.array_equal(C, alpha * (A @ B)), (prec, shape, alpha)


# elementwise bound |C - AB| <= tol * (|A| |B|): input rounding of the mode
# (2 u per product) plus FP32 accumulation over K <= 300
TOL = {0: 1e-14, 1: 4e-5, 2: 1.2e-3, 3: 5e-3, 4: 5e-5}


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_random_operands_within_rounding_bound(ctx, prec):
    for M, N, K in SHAPES:
        rng = np.random.default_rng(7 + M + N + K)
        A = rng.standard_normal((M, K))
        B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, size=(1, N)))
        C = ctx.gemm(dev(A), dev(B), 1.0, precision=prec).cpu().numpy()
        scale = np.abs(A) @ np.abs(B)
        e = np.abs(C - A @ B) / scale
        assert np.max(e) < TOL[prec], (prec, (M, N, K), np.max(e))
    if prec == 4:
        # the split recovers what plain TF32 loses
        M, N, K = SHAPES[3]
        rng = np.random.default_rng(11)
        A = rng.standard_normal((M, K))
        B = rng.standard_normal((K, N))
        e3 = np.mean(np.abs(ctx.gemm(dev(A), dev(B), 1.0, precision=4).cpu().numpy() - A @ B))
        e1 = np.mean(np.abs(ctx.gemm(dev(A), dev(B), 1.0, precision=2).cpu().numpy() - A @ B))
        assert e3 < e1 / 50, (e3, e1)


def test_empty_and_zero_k(ctx):
    import torch
    for prec in (0, 2, 4):
        A = torch.zeros((5, 0), dtype=torch.float64, device="cuda")
        B = torch.zeros((0, 7), dtype=torch.float64, device="cuda")
        C = ctx.gemm(A, B, 1.0, precision=prec).cpu().numpy()
        assert C.shape == (5, 7) and np.all(C == 0)
