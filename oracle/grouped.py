"""Grouped interleaved (IG) ordering (oracle; test infrastructure only).

Main text, "State Compressibility": besides the sequential orderings and the
flat interleaved one (IF: x_0, v_0, x_1, v_1, ... one bit per site) the paper
groups each pair (x_j, v_j) into one site of physical dimension d = 4.  The
state is then an MPS of n/2 cores (r, 4, r'); it has bonds only between pairs,
and only those bonds are truncated.  Operators act through the IF MPO with
each pair of cores merged into one (w, 4, 4, w') core.  The physical index of
a pair is 2 i_x + i_v (x bit first, as in the IF site order).

Everything here is written for a general physical dimension d and follows
the same definitions as :mod:`oracle.mps` (QR sweep left to right, truncated
SVD sweep right to left, the rank rule of :func:`oracle.mps.choose_rank`).
Requires nx == nv.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import mps as S
from . import vp as V


def group(cores):
    """IF MPS (n cores (r, 2, r')) -> IG MPS (n/2 cores (r, 4, r'))."""
    if len(cores) % 2:
        raise ValueError("IG needs an even number of sites (nx == nv)")
    return [np.einsum("aib,bjc->aijc", cores[2 * j], cores[2 * j + 1]).reshape(cores[2 * j].shape[0], 4, -1)
            for j in range(len(cores) // 2)]


def ungroup(cores):
    """IG -> IF by an exact SVD split of every pair core (nothing dropped
    but exact zeros)."""
    out = []
    for c in cores:
        rl, _, rr = c.shape
        u, s, vt = sla.svd(c.reshape(rl * 2, 2 * rr), full_matrices=False, lapack_driver="gesvd")
        k = max(1, int(np.sum(s > 0)))
        out.append(u[:, :k].reshape(rl, 2, k))
        out.append((s[:k, None] * vt[:k]).reshape(k, 2, rr))
    return out


def group_mpo(mpo):
    """Pairs of IF MPO cores (w, 2, 2, w') -> one (w, 4, 4, w'') core, out
    index 2 o_x + o_v, in index 2 i_x + i_v."""
    out = []
    for j in range(len(mpo) // 2):
        a, b = mpo[2 * j], mpo[2 * j + 1]
        c = np.einsum("aoib,bpjc->aopijc", a, b)
        s = c.shape
        out.append(c.reshape(s[0], 4, 4, s[5]))
    return out


def to_dense(cores):
    t = cores[0].reshape(cores[0].shape[1], -1)
    for c in cores[1:]:
        t = (t @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
    return t.reshape(-1)


def apply_mpo(mpo, mps):
    """SI "Matrix-vector multiplication" for any d: bonds multiply."""
    out = []
    for B, A in zip(mpo, mps):
        C = np.einsum("boic,aid->abodc", B, A)
        s = C.shape
        out.append(C.reshape(s[0] * s[1], s[2], s[3] * s[4]))
    return out


def add(a, b, alpha=1.0, beta=1.0):
    """SI "Addition" for any d: block-diagonal cores."""
    n = len(a)
    out = []
    for k in range(n):
        A, B = a[k], b[k]
        if k == 0:
            A, B = alpha * A, beta * B
        if n == 1:
            out.append(A + B)
        elif k == 0:
            out.append(np.concatenate([A, B], axis=2))
        elif k == n - 1:
            out.append(np.concatenate([A, B], axis=0))
        else:
            c = np.zeros((A.shape[0] + B.shape[0], A.shape[1], A.shape[2] + B.shape[2]))
            c[:A.shape[0], :, :A.shape[2]] = A
            c[A.shape[0]:, :, A.shape[2]:] = B
            out.append(c)
    return out


def qr_sweep(cores):
    out = [c.copy() for c in cores]
    for k in range(len(out) - 1):
        rl, d, rr = out[k].shape
        q, r = sla.qr(out[k].reshape(rl * d, rr), mode="economic")
        p = q.shape[1]
        out[k] = q.reshape(rl, d, p)
        nxt = out[k + 1]
        out[k + 1] = (r @ nxt.reshape(rr, -1)).reshape(p, nxt.shape[1], nxt.shape[2])
    return out


def svd_sweep(cores, chi, tol):
    out = [c.copy() for c in cores]
    n = len(out)
    errs, svals = [0.0] * (n - 1), [None] * (n - 1)
    for k in range(n - 1, 0, -1):
        rl, d, rr = out[k].shape
        u, s, vt = sla.svd(out[k].reshape(rl, d * rr), full_matrices=False, lapack_driver="gesvd")
        r, e = S.choose_rank(s, chi, tol)
        errs[k - 1], svals[k - 1] = e, s
        out[k] = vt[:r].reshape(r, d, rr)
        prev = out[k - 1]
        out[k - 1] = (prev.reshape(-1, rl) @ (u[:, :r] * s[:r])).reshape(prev.shape[0], prev.shape[1], r)
    return out, errs, svals


def compress(cores, chi, tol):
    out, errs, _ = svd_sweep(qr_sweep(cores), chi, tol)
    return out, errs


def bonds(cores):
    return [1] + [c.shape[2] for c in cores]


def mps_from_f(f, layout, chi, tol=V.TOL):
    """f on an IF-ordered layout -> IG MPS: exact TT-SVD, grouped, compressed."""
    return compress(group(S.tt_svd(V.dense_to_sites(f, layout), layout.n)), chi, tol)[0]


def mps_to_f(cores, layout):
    return V.sites_to_dense(to_dense(cores), layout)


def rk4_step(f, layout, dt, chi, tol=V.TOL, e_tol=V.TOL):
    """One RK4-C1 step in the IG ordering: the schedule of
    :func:`oracle.vp.rk4_step` with the state held as d = 4 pair cores.  The
    stage field comes from the density of the stage state (read through the
    exact IF split), the operator is the IF operator with its pairs merged."""
    acc, fi, diag = f, f, {}
    for i in range(4):
        E, we, rho = V.stage_field(ungroup(fi), layout, e_tol)
        if i == 0:
            dx, _ = V.grid_steps(layout)
            diag["field_energy"] = we
            diag["mass"] = float(np.sum(rho)) * dx
        L = group_mpo(V.operator(V.field_mps(E, layout, e_tol), layout))
        k = apply_mpo(L, fi)
        if i < 3:
            fi, _ = compress(add(f, k, 1.0, V.A_RK[i] * dt), 1 << 30, tol)
            acc, _ = compress(add(acc, k, 1.0, V.B_RK[i] * dt), 1 << 30, tol)
        else:
            acc, errs = compress(add(acc, k, 1.0, V.B_RK[3] * dt), chi, tol)
            diag["trunc_err"] = errs
    diag["bonds"] = bonds(acc)
    return acc, diag
