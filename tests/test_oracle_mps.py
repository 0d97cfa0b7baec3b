"""Pins of the oracle's MPS algebra and compression (CPU)."""
import numpy as np
import pytest

from oracle import mpo as M
from oracle import mps as S
from paper_2205_11990_gb300 import inputs as I


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_tt_svd_exact_and_full_rank_profile(n):
    x = I.random_vector(n, seed=n)
    cores = S.tt_svd(x, n)
    np.testing.assert_allclose(S.to_dense(cores), x, atol=1e-12)
    # main text: exact full-rank bonds r_j = d^min(j, KL-j)
    assert S.bonds(cores) == [2 ** min(j, n - j) for j in range(n + 1)]


def test_apply_mpo_is_matvec_and_bonds_multiply():
    rng = np.random.default_rng(1)
    n = 5
    mps = I.random_cores([1, 2, 4, 3, 2, 1], seed=2)
    w = [1, 3, 2, 4, 2, 1]
    mpo = [rng.standard_normal((w[k], 2, 2, w[k + 1])) for k in range(n)]
    out = S.apply_mpo(mpo, mps)
    np.testing.assert_allclose(S.to_dense(out), M.to_dense(mpo) @ S.to_dense(mps), atol=1e-12)
    assert S.bonds(out) == [a * b for a, b in zip(S.bonds(mps), w)]


def test_add_is_dense_add_and_bonds_add():
    a = I.random_cores([1, 2, 3, 2, 1], seed=4)
    b = I.random_cores([1, 2, 2, 2, 1], seed=5)
    out = S.add(a, b, 0.7, -1.3)
    np.testing.assert_allclose(S.to_dense(out), 0.7 * S.to_dense(a) - 1.3 * S.to_dense(b), atol=1e-13)
    assert S.bonds(out)[1:-1] == [x + y for x, y in zip(S.bonds(a)[1:-1], S.bonds(b)[1:-1])]


def test_qr_sweep_left_canonical():
    cores = I.random_cores([1, 2, 4, 8, 4, 2, 1], seed=6)
    q = S.qr_sweep(cores)
    np.testing.assert_allclose(S.to_dense(q), S.to_dense(cores), atol=1e-12)
    for c in q[:-1]:  # sum_{l,u} L_{l,r}(u) L_{l,r'}(u) = delta
        m = c.reshape(-1, c.shape[2])
        np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)


def test_svd_sweep_right_canonical_and_exact_without_truncation():
    cores = I.random_cores([1, 2, 4, 8, 4, 2, 1], seed=7)
    out, errs = S.compress(cores, 1 << 10, 0.0)
    np.testing.assert_allclose(S.to_dense(out), S.to_dense(cores), atol=1e-12)
    for c in out[1:]:
        m = c.reshape(c.shape[0], -1)
        np.testing.assert_allclose(m @ m.T, np.eye(m.shape[0]), atol=1e-12)
    assert max(errs) == 0.0


def test_two_site_compression_is_eckart_young():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((2, 2)) @ np.diag([3.0, 0.01]) @ rng.standard_normal((2, 2))
    cores = S.tt_svd(A.reshape(-1), 2)
    out, errs = S.compress(cores, 1, 0.0)
    u, s, vt = np.linalg.svd(A)
    np.testing.assert_allclose(S.to_dense(out).reshape(2, 2), s[0] * np.outer(u[:, 0], vt[0]), atol=1e-12)
    np.testing.assert_allclose(errs[0], s[1] / np.linalg.norm(s), rtol=1e-10)


def test_truncation_error_identity_single_bond():
    # main text, truncation-error equation: in canonical form, cutting one
    # bond gives ||f - f_D|| / ||f|| = sqrt(sum of discarded normalised s^2)
    cores = I.random_cores([1, 2, 3, 3, 8, 3, 3, 2, 1], seed=9)
    x = S.to_dense(cores)
    out, errs = S.compress(cores, 3, 0.0)  # only bond 4 (rank 8) exceeds 3
    assert S.bonds(out) == [1, 2, 3, 3, 3, 3, 3, 2, 1]
    assert [e > 0 for e in errs] == [False, False, False, True, False, False, False]
    err = np.linalg.norm(S.to_dense(out) - x) / np.linalg.norm(x)
    np.testing.assert_allclose(err, errs[3], rtol=1e-9)
    # and it equals the best rank-3 approximation of the 16 x 16 unfolding
    u, sv, vt = np.linalg.svd(x.reshape(16, 16))
    np.testing.assert_allclose(S.to_dense(out), ((u[:, :3] * sv[:3]) @ vt[:3]).reshape(-1), atol=1e-12)


def test_choose_rank_rules():
    s = np.array([1.0, 0.5, 1e-6, 1e-11, 1e-12])
    assert S.choose_rank(s, 10, 0.0)[0] == 5
    assert S.choose_rank(s, 10, 1e-10)[0] == 3
    assert S.choose_rank(s, 2, 1e-10)[0] == 2
    assert S.choose_rank(s, 10, 1e-5)[0] == 2
    # a degenerate pair at the cut is dropped as a whole
    assert S.choose_rank(np.array([1.0, 0.3, 0.3, 0.1]), 2, 0.0)[0] == 1
    assert S.choose_rank(np.zeros(4), 3, 1e-10)[0] == 1
    r, e = S.choose_rank(np.array([3.0, 4.0 * 0 + 1e-3]), 1, 0.0)
    assert r == 1 and abs(e - 1e-3 / np.hypot(3.0, 1e-3)) < 1e-15


def test_tie_window_edges():
    # the tie window is a relative gap of TIE_REL between the last kept and
    # the first dropped value: just outside it the chi cut stands, just
    # inside it the pair is dropped as one cluster
    w = S.TIE_REL
    for chi in (2, 3):
        top = [1.0, 0.7, 0.5][:chi - 1]
        outside = np.array(top + [0.25, 0.25 * (1 - 2 * w), 0.01])
        inside = np.array(top + [0.25, 0.25 * (1 - 0.5 * w), 0.01])
        assert S.choose_rank(outside, chi, 0.0)[0] == chi
        assert S.choose_rank(inside, chi, 0.0)[0] == chi - 1
    # a cluster of three within the window moves the cut to its start
    s = np.array([1.0, 0.5, 0.5 * (1 - 0.3 * w), 0.5 * (1 - 0.6 * w), 0.1])
    assert S.choose_rank(s, 3, 0.0)[0] == 1
    # the tolerance cut obeys the same rule: tol lands between a near-equal
    # pair (tail of the pair above tol, the last value alone below it)
    s = np.array([1.0, 1e-3, 1e-3 * (1 - 0.5 * w), 1e-12])
    assert S.choose_rank(s, 10, 1e-9)[0] == 3
    s2 = np.array([1.0, 1e-3, 1e-3 * (1 - 0.5 * w)])
    assert S.choose_rank(s2, 2, 0.0)[0] == 1
    assert S.choose_rank(s2, 2, 0.0)[1] > 1e-3


def test_tie_stats_count_the_rule():
    S.TIE_STATS.update(cuts=0, fired=0, min_gap=float("inf"))
    S.choose_rank(np.array([1.0, 0.3, 0.3, 0.1]), 2, 0.0)       # fires
    S.choose_rank(np.array([1.0, 0.5, 0.25, 0.1]), 2, 0.0)      # cut with gap 0.5
    S.choose_rank(np.array([1.0, 0.5]), 5, 0.0)                # keeps all: no cut
    assert S.TIE_STATS["cuts"] == 2 and S.TIE_STATS["fired"] == 1
    assert S.TIE_STATS["min_gap"] == 0.5


def test_entanglement_entropy_closed_forms():
    # maximally entangled: r equal values -> log2 r; product state -> 0
    assert abs(S.entanglement_entropy(np.ones(8), 8) - 3.0) < 1e-14
    assert S.entanglement_entropy(np.array([2.0, 0.0]), 1) == 0.0
    # a Bell-like two-site state (|00> + |11>)/sqrt2 has EE 1 at its bond
    v = np.array([1.0, 0.0, 0.0, 1.0]) / np.sqrt(2)
    _, _, ee = S.compress_with_entropy(S.tt_svd(v, 2), 4, 0.0)
    assert abs(ee[0] - 1.0) < 1e-12


# ------------------------------------------- modified compression (SI scheme)
def test_modified_compression_exact_and_centre_schmidt_values():
    # nothing truncated: the state is reproduced; the centre bond's values are
    # the singular values of the dense state reshaped at the x / v cut
    cores = I.random_cores([1, 2, 4, 8, 16, 8, 4, 2, 1], seed=3)
    d = S.to_dense(cores)
    out, errs, sv = S.compress_modified(cores, 1 << 10, 0.0, 4)
    assert np.linalg.norm(S.to_dense(out) - d) <= 1e-13 * np.linalg.norm(d)
    ref = np.linalg.svd(d.reshape(16, 16), compute_uv=False)
    np.testing.assert_allclose(sv[3][:len(ref)], ref, rtol=1e-12, atol=1e-14 * ref[0])
    assert max(errs) == 0.0


def test_modified_compression_centre_cut_is_eckart_young():
    # a state whose only bond above chi is the centre: the result is the best
    # rank-chi approximation across the cut (the half sweeps cut nothing)
    rng = np.random.default_rng(11)
    nx = nv = 3
    X = rng.standard_normal((8, 6))
    V = rng.standard_normal((6, 8)) * np.exp(-np.arange(6))[:, None]
    d = (X @ V).reshape(-1)
    cores = S.tt_svd(d, nx + nv)
    # bonds of a 3 + 3 site chain are at most 2, 4, (6 at the centre), 4, 2
    out, errs, _ = S.compress_modified(cores, 4, 0.0, nx)
    u, s, vt = np.linalg.svd(d.reshape(8, 8))
    best = (u[:, :4] * s[:4]) @ vt[:4]
    assert np.linalg.norm(S.to_dense(out) - best.reshape(-1)) <= 1e-12 * np.linalg.norm(d)
    assert abs(errs[nx - 1] - np.sqrt(np.sum(s[4:] ** 2)) / np.linalg.norm(s)) <= 1e-12
    assert [e for j, e in enumerate(errs) if j != nx - 1] == [0.0] * 4


def test_modified_compression_error_bound():
    # every truncation removes an orthogonal piece: the total relative error
    # is at most the root sum of the per-bond truncation errors
    cores = I.random_cores([1, 2, 4, 8, 16, 32, 16, 8, 4, 2, 1], seed=9)
    d = S.to_dense(cores)
    for chi, tol in ((6, 0.0), (1 << 10, 0.05), (4, 0.01)):
        out, errs, _ = S.compress_modified(cores, chi, tol, 5)
        e = np.linalg.norm(S.to_dense(out) - d) / np.linalg.norm(d)
        assert e <= np.sqrt(np.sum(np.square(errs))) * (1 + 1e-9) + 1e-14
        assert max(c.shape[2] for c in out) <= chi


def test_compression_error_pins():
    # one bond (two sites of dimension 2^3 each): Eckart-Young, the rms error
    # of the best rank-D approximation is sqrt(sum_{i>D} s_i^2 / N)
    rng = np.random.default_rng(12)
    M = rng.standard_normal((8, 8))
    U, s, Vt = np.linalg.svd(M)
    s = 2.0 ** -np.arange(8)
    M = (U * s) @ Vt
    cores = S.tt_svd(M.reshape(-1), 6, None, 0.0)  # bonds 1, 2, 4, 8, 4, 2, 1: the middle one is M
    errs = S.compression_error(cores, [8, 4, 2], 0.0)
    assert errs[0] < 1e-15
    # at D = 4 and D = 2 only the middle bond (rank 8) is cut; bonds 1-2 and
    # 4-5 have rank <= 4 and are exact
    assert abs(errs[1] - np.sqrt(np.sum(s[4:] ** 2) / 64)) < 1e-14
    exact2 = S.compression_error(S.tt_svd(M.reshape(-1), 6, None, 0.0), [2], 0.0)[0]
    assert exact2 >= np.sqrt(np.sum(s[2:] ** 2) / 64) - 1e-14  # no rank-2 MPS beats Eckart-Young at that cut
    # a state of bond 1 everywhere (a product) has no compression error at D = 1
    prod = [np.array([1.0, 2.0]).reshape(1, 2, 1) for _ in range(5)]
    f = S.to_dense(prod)
    assert S.compression_error(prod, [1], 0.0)[0] < 1e-14 * np.sqrt(np.mean(f * f))
