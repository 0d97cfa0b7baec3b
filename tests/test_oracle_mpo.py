"""Pins of the oracle's MPOs against the stencils they stand for (CPU)."""
import itertools

import numpy as np
import pytest

from oracle import mpo as M
from oracle import mps as S
from oracle import vp as V
from paper_2205_11990_gb300 import inputs as I


def stencil(N, coefs, dx, periodic=True):
    D = np.zeros((N, N))
    for s, c in coefs.items():
        for n in range(N):
            m = n + s
            if periodic:
                D[n, m % N] += c
            elif 0 <= m < N:
                D[n, m] += c
    return D / dx


@pytest.mark.parametrize("L", [3, 4, 5, 7])
def test_printed_derivative_mpos_equal_stencils(L):
    N, dx = 1 << L, 0.37
    cases = [
        (M.centered_periodic(L, dx), stencil(N, {1: 0.5, -1: -0.5}, dx)),
        (M.forward_periodic(L, dx), stencil(N, {0: -1.5, 1: 2.0, 2: -0.5}, dx)),
        (M.backward_periodic(L, dx), stencil(N, {0: 1.5, -1: -2.0, -2: 0.5}, dx)),
        (M.second_periodic(L, dx), stencil(N, {0: -2.0, 1: 1.0, -1: 1.0}, dx) / dx),
    ]
    for op, ref in cases:
        np.testing.assert_allclose(M.to_dense(op), ref, atol=1e-13 / dx ** 2)


@pytest.mark.parametrize("L", [3, 5, 6])
def test_zero_gradient_mpo_has_zero_rows_at_both_ends(L):
    N, dv = 1 << L, 0.21
    D = M.to_dense(M.centered_zero_gradient(L, dv))
    ref = stencil(N, {1: 0.5, -1: -0.5}, dv, periodic=False)
    ref[0, :] = 0.0
    ref[-1, :] = 0.0
    np.testing.assert_allclose(D, ref, atol=1e-13)
    # ghost node equal to the node inside the boundary: a function constant
    # near the ends has zero derivative there; a linear one keeps slope inside
    j = np.arange(N, dtype=float)
    np.testing.assert_allclose((D @ (3.0 * j))[1:-1], 3.0 / dv, rtol=1e-12)


def test_fd_mpo_bonds_within_printed_range():
    # main text "Cost Analysis": FD MPO bonds around 2 to 5
    for op in (M.centered_periodic(6, 1.0), M.forward_periodic(6, 1.0), M.second_periodic(6, 1.0),
               M.centered_zero_gradient(6, 1.0)):
        assert 2 <= max(c.shape[3] for c in op[:-1]) <= 5


def test_inverse_laplacian_mpo_bond_about_five():
    # SI "Inverse Laplacian": bond ~5 at 1e-10 (golden: paper_printed_values.txt)
    L = 8
    N, dx = 1 << L, 0.1
    Dinv = np.linalg.pinv(M.to_dense(M.second_periodic(L, dx)), rtol=1e-9, hermitian=True)
    # operator as a 2L-site d=2 tensor ordered (o_1, i_1, o_2, i_2, ...)
    t = Dinv.reshape([2] * (2 * L)).transpose([a for k in range(L) for a in (k, L + k)]).reshape(-1)
    cores = S.tt_svd(t, 2 * L, tol=1e-10)
    mpo_bonds = [c.shape[2] for c in cores[1:-1:2]]
    assert abs(max(mpo_bonds) - 5) <= 1, mpo_bonds


def test_mpo_sum_and_diag():
    rng = np.random.default_rng(0)
    a = [rng.standard_normal((1 if k == 0 else 2, 2, 2, 1 if k == 3 else 2)) for k in range(4)]
    b = [rng.standard_normal((1 if k == 0 else 3, 2, 2, 1 if k == 3 else 3)) for k in range(4)]
    np.testing.assert_allclose(M.to_dense(M.mpo_sum(a, b)), M.to_dense(a) + M.to_dense(b), atol=1e-12)
    cores = I.random_cores([1, 2, 3, 2, 1], seed=3)
    np.testing.assert_allclose(M.to_dense(M.diag_from_mps(cores)), np.diag(S.to_dense(cores)), atol=1e-14)


@pytest.mark.parametrize("mapping", [I.SEQ, I.INTERLEAVED])
def test_place_is_kron_with_site_permutation(mapping):
    lay = I.Layout(3, 3, 0, 1, -1, 1, mapping)
    X = M.forward_periodic(3, 0.5)
    Vv = M.centered_zero_gradient(3, 0.25)
    op = M.place([X, Vv], V.sitemap(lay))
    dense = M.to_dense(op)
    ref = np.kron(M.to_dense(X), M.to_dense(Vv))  # on f[ix, iv] flattened row-major
    # map site-ordered indices to (ix, iv) ordered ones
    perm = np.array([int(V.sites_to_dense(np.eye(64)[k], lay).reshape(-1).argmax()) for k in range(64)])
    np.testing.assert_allclose(dense, ref[np.ix_(perm, perm)], atol=1e-13)


def test_heaviside_velocity_mps_is_exact():
    lay = I.Layout(4, 5, 0, 1, -6, 6, I.SEQ)
    v = lay.v()
    for pos in (True, False):
        cores = V._vh_mps(lay, pos)
        ref = np.where(v > 0, v, 0) if pos else np.where(v > 0, 0, v)
        np.testing.assert_allclose(S.to_dense(cores), ref, atol=1e-12)
        assert max(S.bonds(cores)) <= 2
