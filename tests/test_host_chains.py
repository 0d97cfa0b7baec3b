"""Host-built operator chains of the library (mpo_build.cpp) against the
oracle's dense operators (CPU: the chains are compiled with g++ here)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import dense_fd as DF

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_11990_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("chains") / "chain_dense")
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CSRC}", os.path.join(ROOT, "tests", "host", "chain_dense.cpp"),
                    os.path.join(CSRC, "mpo_build.cpp"), "-o", exe], check=True)
    return exe


def dense(driver, kind, L, vmin, dv, nu=0.0, u=0.0, vth=1.0, extra=()):
    out = subprocess.run([driver, kind, str(L), repr(vmin), repr(dv), repr(nu), repr(u), repr(vth)]
                         + [str(x) for x in extra], check=True, capture_output=True, text=True).stdout.splitlines()
    bonds = [int(x) for x in out[0].split()[1:]]
    return bonds, np.array([[float(x) for x in line.split()] for line in out[1:]])


def oracle_matrix(L, vmin, dv, nu, u, vth):
    v = vmin + dv * np.arange(1 << L)
    eye = np.eye(1 << L)
    return np.stack([DF.dougherty(eye[j][None, :], v, dv, nu, u, vth)[0] for j in range(1 << L)], axis=1)


@pytest.mark.parametrize("L", [1, 2, 5])
def test_second_derivative_chain(driver, L):
    dv = 0.3
    _, D = dense(driver, "d2", L, 0.0, dv)
    f = np.eye(1 << L)
    ref = np.stack([DF.d_second_v_zero_gradient(f[j][None, :], dv)[0] for j in range(1 << L)], axis=1)
    np.testing.assert_allclose(D, ref, atol=1e-12 / dv**2)


@pytest.mark.parametrize("L", [2, 4, 6])
def test_collision_chain_and_its_reduction(driver, L):
    vmin, dv, nu, u, vth = -60.0, 120.0 / ((1 << L) - 1), 0.3, 10.0, 1.0
    ref = oracle_matrix(L, vmin, dv, nu, u, vth)
    b0, C = dense(driver, "coll", L, vmin, dv, nu, u, vth)
    b1, R = dense(driver, "coll_reduced", L, vmin, dv, nu, u, vth)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(C, ref, atol=1e-13 * scale)
    np.testing.assert_allclose(R, ref, atol=1e-13 * scale)
    # the reduction keeps the numerical rank (at most 6 here) and never grows a bond
    assert all(r <= s for r, s in zip(b1, b0)) and max(b1) <= 6


@pytest.mark.parametrize("mapping", [0, 1, 2, 3])
def test_collisional_static_operator_equals_oracle(driver, mapping):
    # the static part of a collisional species' operator as the sim builds it
    # (upwind + placed Dougherty chain, reduced to its numerical rank) against
    # the oracle's printed-MPO upwind operator plus its collision MPO
    import math

    from oracle import mpo as M
    from oracle import vp as V
    from paper_2205_11990_gb300 import inputs as I
    lay = I.Layout(3, 4, 0.0, 2 * math.pi, -7.0, 7.0, mapping)
    dx, dv = V.grid_steps(lay)
    nu, u, vth = 0.3, 1.5, 0.8
    bonds, got = dense(driver, "static", lay.nv, lay.vmin, dv, nu, u, vth, (lay.nx, repr(dx), mapping))
    up, _ = V._static_parts(lay)
    ref = M.to_dense(M.mpo_sum(up, V.collision_mpo(lay, nu, u, vth)))
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())
