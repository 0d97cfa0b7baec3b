"""Writes fullsize_4096_step.json: the oracle's result of one RK4-C1 step of
the 4096 x 4096 saturated two-stream workload (12 + 12 sites, sequential,
chi = 128, tol = 1e-10), for the GPU full-size test, which cannot run the
oracle at this size within its time budget.

Calls only oracle/ and the seeded input generators.  The initial MPS is the
exact TT-SVD of the sampled f0 with singular values below 1e-14 of each
bond's spectrum dropped (the exact decomposition keeps numerically zero
values and would reach rank 4096 at the middle bond), then the compression
to chi and tol: a change of f0 of order 1e-14, far inside the 1e-10 the test
holds.  Stored: the field energy and mass of the start state, the bonds
after the step, and the values of f(T) at 4096 seeded grid points.

Run from the repository root:  python tests/golden/make_fullsize_4096.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import mps as S  # noqa: E402
from oracle import vp as V  # noqa: E402
from paper_2205_11990_gb300 import inputs as I  # noqa: E402

NAME = "saturated_two_stream_4096x4096_seq"
NSAMPLES = 4096


def main():
    w = I.WORKLOADS[NAME]
    lay, chi, dt = w["layout"], w["chi"], w["dt"]
    t0 = time.time()
    f0 = I.initial_condition(w["ic"], lay)
    cores = S.compress(S.tt_svd(V.dense_to_sites(f0, lay), lay.n, None, 1e-14), chi, V.TOL)[0]
    t1 = time.time()
    out, d = V.rk4_step(cores, lay, dt, chi)
    t2 = time.time()
    f1 = V.mps_to_f(out, lay)
    rng = np.random.Generator(np.random.PCG64(4096))
    ix = rng.integers(0, lay.Nx, size=NSAMPLES)
    iv = rng.integers(0, lay.Nv, size=NSAMPLES)
    res = {
        "workload": NAME, "chi": chi, "dt": dt, "tol": V.TOL,
        "field_energy": d["field_energy"], "mass": d["mass"], "bonds": [int(b) for b in d["bonds"]],
        "start_bonds": [int(b) for b in S.bonds(cores)],
        "ix": ix.tolist(), "iv": iv.tolist(), "f": f1[ix, iv].tolist(),
        "f_rms": float(np.sqrt(np.mean(f1 * f1))),
        "note": f"oracle step, {t2 - t1:.0f} s (start state {t1 - t0:.0f} s)",
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_4096_step.json")
    with open(path, "w") as fh:
        json.dump(res, fh)
    print(path, res["note"], "max bond", max(res["bonds"]))


if __name__ == "__main__":
    main()
