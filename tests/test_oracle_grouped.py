"""Pins of the oracle's grouped interleaved (IG, d = 4) ordering (CPU)."""
import math

import numpy as np
import pytest

from oracle import dense_fd as DF
from oracle import grouped as G
from oracle import mps as S
from oracle import vp as V
from paper_2205_11990_gb300 import inputs as I


def test_group_ungroup_round_trip():
    c = I.random_cores([1, 2, 4, 5, 3, 2, 1], seed=4)
    g = G.group(c)
    assert [x.shape[1] for x in g] == [4, 4, 4]
    np.testing.assert_allclose(G.to_dense(g), S.to_dense(c), atol=1e-14)
    np.testing.assert_allclose(S.to_dense(G.ungroup(g)), S.to_dense(c), atol=1e-14)


def test_exact_bonds_are_unfolding_ranks():
    rng = np.random.default_rng(1)
    lay = I.Layout(3, 3, 0.0, 1.0, -1.0, 1.0, I.GROUPED)
    # a sum of three separable functions: each unfolding has rank <= 3
    f = sum(np.outer(rng.standard_normal(8), rng.standard_normal(8)) for _ in range(3))
    c = G.mps_from_f(f, lay, 1 << 20, 1e-13)
    vec = V.dense_to_sites(f, lay)
    ranks = [1] + [np.linalg.matrix_rank(vec.reshape(4 ** j, -1), tol=1e-10) for j in (1, 2)] + [1]
    assert G.bonds(c) == ranks


def test_single_cut_truncation_is_eckart_young():
    rng = np.random.default_rng(2)
    vec = rng.standard_normal(16)  # two pairs: one cut, a 4 x 4 unfolding
    c = G.compress(G.group(S.tt_svd(vec, 4)), 2, 0.0)[0]
    u, s, vt = np.linalg.svd(vec.reshape(4, 4))
    best = (u[:, :2] * s[:2]) @ vt[:2]
    np.testing.assert_allclose(G.to_dense(c).reshape(4, 4), best, atol=1e-13)


def test_grouped_mpo_is_the_same_operator():
    lay = I.Layout(3, 3, 0.0, 2 * math.pi, -5.0, 5.0, I.GROUPED)
    c = V.mps_from_f(I.landau(lay, 0.2, 1.0), lay, 64, 0.0)
    E, _, _ = V.stage_field(c, lay)
    L = V.operator(V.field_mps(E, lay), lay)
    np.testing.assert_allclose(G.to_dense(G.apply_mpo(G.group_mpo(L), G.group(c))),
                               S.to_dense(S.apply_mpo(L, c)), atol=1e-11)


def test_exact_mode_step_matches_dense_grid():
    lay = I.Layout(4, 4, 0.0, 4 * math.pi, -6.0, 6.0, I.GROUPED)
    f = I.landau(lay, 0.3, 0.5)
    c = G.mps_from_f(f, lay, 1 << 20, 0.0)
    ref = f
    for _ in range(2):
        c, d = G.rk4_step(c, lay, 0.05, 1 << 20, 0.0, 0.0)
        ref, we, _ = DF.rk4_step(ref, lay, 0.05)
        assert abs(d["field_energy"] - we) <= 1e-12 * we
    np.testing.assert_allclose(G.mps_to_f(c, lay), ref, atol=1e-13)


def test_truncated_step_close_to_dense_grid_and_capped():
    lay = I.Layout(5, 5, 0.0, 10 * math.pi, -8.0, 8.0, I.GROUPED)
    f = I.saturated_two_stream(lay, modes=8)
    c = G.mps_from_f(f, lay, 1 << 20)
    c2, d = G.rk4_step(c, lay, 0.01, 1 << 20)
    ref, _, _ = DF.rk4_step(f, lay, 0.01)
    assert np.linalg.norm(G.mps_to_f(c2, lay) - ref) / np.linalg.norm(ref) < 1e-8
    c3, d3 = G.rk4_step(c, lay, 0.01, 6)
    assert max(d3["bonds"]) <= 6
