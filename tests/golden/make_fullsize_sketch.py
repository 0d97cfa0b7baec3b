"""Writes fullsize_<case>.json: the oracle's result of one RK4-C1 step of a
full-size workload whose oracle step takes minutes, for the GPU tests.

Cases (saturated two-stream state, tol = 1e-10):
  interleaved_1024_chi64  1024 x 1024 (10 + 10 sites, IF ordering), chi = 64,
                          32 seeded modes
  seq_4096_chi256         4096 x 4096 (12 + 12 sites, sequential), chi = 256,
                          400 seeded modes: the x / v cut needs ~2 x 400 + 1
                          singular values, so the middle bonds sit at the cap

Stored, besides the field energy and mass of the start state and the bonds
before and after the step: the values of f(T) at 4096 seeded grid points and
64 sketches y_i = r_i^T F s_i of the whole dense f(T) (F[ix, iv]) with seeded
standard normal r_i (length Nx) and s_i (length Nv).  Every grid value enters
every sketch; for an error E, E|r^T E s|^2 = |E|_F^2, so the relative error of
the sketch vector estimates the relative L2 error of the dense f.

The start MPS is the exact TT-SVD of the sampled f0 with singular values
below 1e-14 of each bond's spectrum dropped, compressed to chi and tol (a
change of f0 of order 1e-14, far inside the 1e-10 the tests hold).  Calls
only oracle/ and the seeded input generators.

Run from the repository root:  python tests/golden/make_fullsize_sketch.py [case ...]
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import mps as S  # noqa: E402
from oracle import vp as V  # noqa: E402
from paper_2205_11990_gb300 import inputs as I  # noqa: E402

NSAMPLES = 4096
NSKETCH = 64


CASES = {
    # name: (nx, nv, xmax / pi, vmax, mapping, chi, modes)
    "interleaved_1024_chi64": (10, 10, 10, 8.0, I.INTERLEAVED, 64, 32),
    "seq_4096_chi256": (12, 12, 10, 8.0, I.SEQ, 256, 400),
}


def case(name):
    nx, nv, xm, vm, mapping, chi, modes = CASES[name]
    lay = I.Layout(nx, nv, 0.0, xm * math.pi, -vm, vm, mapping)
    return lay, I.saturated_two_stream(lay, modes=modes), chi, V.stable_dt(lay, 0.01), modes


def sketch_vectors(lay, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((NSKETCH, lay.Nx)), rng.standard_normal((NSKETCH, lay.Nv))


def sketches(f, r, s):
    return np.einsum("ix,xv,iv->i", r, f, s)


def main(names):
    for name in names:
        lay, f0, chi, dt, modes = case(name)
        t0 = time.time()
        cores = S.compress(S.tt_svd(V.dense_to_sites(f0, lay), lay.n, None, 1e-14), chi, V.TOL)[0]
        t1 = time.time()
        out, d = V.rk4_step(cores, lay, dt, chi)
        t2 = time.time()
        f1 = V.mps_to_f(out, lay)
        rng = np.random.Generator(np.random.PCG64(lay.n))
        ix = rng.integers(0, lay.Nx, size=NSAMPLES)
        iv = rng.integers(0, lay.Nv, size=NSAMPLES)
        r, s = sketch_vectors(lay, 1000 + lay.n)
        res = {
            "case": name, "layout": [lay.nx, lay.nv, lay.xmin, lay.xmax, lay.vmin, lay.vmax, lay.mapping],
            "chi": chi, "dt": dt, "tol": V.TOL, "modes": modes,
            "field_energy": d["field_energy"], "mass": d["mass"], "bonds": [int(b) for b in d["bonds"]],
            "start_bonds": [int(b) for b in S.bonds(cores)],
            "ix": ix.tolist(), "iv": iv.tolist(), "f": f1[ix, iv].tolist(),
            "sketch_seed": 1000 + lay.n, "sketches": sketches(f1, r, s).tolist(),
            "note": f"oracle step {t2 - t1:.0f} s (start state {t1 - t0:.0f} s)",
        }
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fullsize_{name}.json")
        with open(path, "w") as fh:
            json.dump(res, fh)
        print(path, res["note"], "max bond", max(res["bonds"]), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["interleaved_1024_chi64", "seq_4096_chi256"])
