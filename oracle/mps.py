"""MPS algebra, TT-SVD and compression (oracle; test infrastructure only).

An MPS is a list of cores ``A[k]`` of shape ``(r_{k-1}, 2, r_k)`` with
``r_{-1} = r_{n-1} = 1``; site 0 is the most significant bit.  Every function
follows the paper's own definitions:

* TT-SVD: iterated SVDs of reshapes (main text, "MPS Representation of
  Classical Data", MPS decomposition equation, Fig. 1a).
* MPO x MPS: ``C(o) = sum_i B(o,i) A(i)`` with gamma = (alpha, beta)
  (SI "Matrix-vector multiplication").
* MPS + MPS: block-diagonal cores, row/column concatenation at the ends
  (SI "Addition").
* QR canonicalisation left to right, R absorbed into the next core (SI
  "Canonicalization and Compression").
* Truncated-SVD sweep keeping the D largest singular values, with the
  truncation error of the epsilon_j equation (main text) as tolerance.

LAPACK does the factorisations (``scipy.linalg.qr`` Householder,
``scipy.linalg.svd`` with ``gesvd``).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

# Two singular values closer than this fraction of the smaller kept one are
# treated as one degenerate cluster that is kept or dropped as a whole, so the
# kept subspace (and hence f) is unique up to rounding.  The width follows
# from Wedin's sin-theta bound: if two computations of the same bond matrix
# differ in their singular values by delta ~ c u sigma_1 (u the unit roundoff
# of the arithmetic), a cut inside a relative gap g = (s_r - s_{r+1}) / s_r
# mixes the kept and discarded vectors by an angle up to delta / (g s_r), so
# f moves by up to ~2 delta / g relative to sigma_1.  With the double-word
# factorisations of the GPU path (u ~ 2^-48 ~ 3.6e-15, c of order 1-10) and
# the 1e-10 parity contract on f, gaps below ~1e-5 .. 1e-4 are not resolved
# identically by two correct implementations.
TIE_REL = 1e-5

# Counters of the rank choices (instrumentation for reports; no effect on
# the result): cuts made, cuts moved down by the tie rule, and the smallest
# relative gap s_{r-1} - s_r seen at a cut that the rule did not move.
TIE_STATS = {"cuts": 0, "fired": 0, "min_gap": float("inf")}


def to_dense(cores):
    """Contract the MPS into the 2^n vector (index bits: site 0 = MSB)."""
    t = cores[0].reshape(2, -1)
    for c in cores[1:]:
        t = (t @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
    return t.reshape(-1)


def bonds(cores):
    return [1] + [c.shape[2] for c in cores]


def choose_rank(s, chi, tol):
    """Number of singular values kept at one bond.

    ``s`` sorted descending.  The normalised values s/||s|| give the
    truncation error sqrt(sum_{i>=r} s_i^2)/||s|| of the epsilon_j equation
    when the first r are kept.  Keep r = min(chi, r_tol), where r_tol is the
    smallest r >= 1 with that error <= tol (tol = 0 keeps every value).  Tail
    sums run smallest-first.  A cut that would split a cluster of nearly equal
    values (relative gap <= TIE_REL) moves down to the cluster start.  Returns
    (r, truncation error).
    """
    s = np.asarray(s, dtype=np.float64)
    m = len(s)
    nrm2 = float(np.sum(s[::-1] ** 2))
    if nrm2 == 0.0:
        return 1, 0.0
    tail2 = np.zeros(m + 1)
    acc = 0.0
    for i in range(m - 1, -1, -1):  # tail2[r] = sum_{i>=r} s_i^2, smallest first
        acc += s[i] * s[i]
        tail2[i] = acc
    if tol > 0.0:
        thr2 = tol * tol * nrm2
        r_tol = m
        for r in range(1, m + 1):
            if tail2[r] <= thr2:
                r_tol = r
                break
    else:
        r_tol = m
    r = min(chi, r_tol, m)
    r0 = r
    while 1 < r < m and (s[r - 1] - s[r]) <= TIE_REL * s[r - 1]:
        r -= 1
    r = max(r, 1)
    if 1 <= r0 < m:
        TIE_STATS["cuts"] += 1
        if r != r0:
            TIE_STATS["fired"] += 1
        elif s[r - 1] > 0.0:
            TIE_STATS["min_gap"] = min(TIE_STATS["min_gap"], float((s[r - 1] - s[r]) / s[r - 1]))
    return r, math.sqrt(tail2[r] / nrm2)


def tt_svd(vec, n, chi=None, tol=0.0):
    """TT-SVD by iterated SVDs of reshapes, left to right (A1).

    With tol = 0 and chi = None nothing is truncated (exact decomposition).
    """
    chi = chi if chi is not None else 1 << n
    cores = []
    r = 1
    rest = np.asarray(vec, dtype=np.float64).reshape(1, -1)
    for k in range(n - 1):
        mat = rest.reshape(r * 2, -1)
        u, s, vt = sla.svd(mat, full_matrices=False, lapack_driver="gesvd")
        rk, _ = choose_rank(s, chi, tol)
        cores.append(u[:, :rk].reshape(r, 2, rk))
        rest = s[:rk, None] * vt[:rk]
        r = rk
    cores.append(rest.reshape(r, 2, 1))
    return cores


def apply_mpo(mpo, mps):
    """C^{(n)}_{(a,b),(a',b')}(o) = sum_i B_{b,b'}(o,i) A_{a,a'}(i); bonds multiply."""
    out = []
    for B, A in zip(mpo, mps):
        C = np.einsum("boic,aid->abodc", B, A)  # bond index = (alpha, beta)
        s = C.shape
        out.append(C.reshape(s[0] * s[1], 2, s[3] * s[4]))
    return out


def add(a, b, alpha=1.0, beta=1.0):
    """alpha*a + beta*b with block-diagonal cores; bonds add (SI "Addition")."""
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
            c = np.zeros((A.shape[0] + B.shape[0], 2, A.shape[2] + B.shape[2]))
            c[:A.shape[0], :, :A.shape[2]] = A
            c[A.shape[0]:, :, A.shape[2]:] = B
            out.append(c)
    return out


def qr_sweep(cores):
    """Left-canonicalise: QR of each (2 r_{k-1} x r_k) reshape, R into core k+1."""
    out = [c.copy() for c in cores]
    n = len(out)
    for k in range(n - 1):
        c = out[k]
        rl, _, rr = c.shape
        q, r = sla.qr(c.reshape(rl * 2, rr), mode="economic")
        p = q.shape[1]
        out[k] = q.reshape(rl, 2, p)
        nxt = out[k + 1]
        out[k + 1] = (r @ nxt.reshape(rr, -1)).reshape(p, 2, nxt.shape[2])
    return out


def svd_sweep(cores, chi, tol):
    """Right-to-left truncated SVD sweep on a left-canonical MPS.

    At site k: SVD of the (r_{k-1} x 2 r_k) reshape, keep r per
    :func:`choose_rank`, core k <- V^T (right-canonical), core k-1 <- core
    k-1 * U S.  Returns (cores, truncation error per bond, singular values
    per bond).
    """
    out = [c.copy() for c in cores]
    n = len(out)
    errs = [0.0] * (n - 1)
    svals = [None] * (n - 1)
    for k in range(n - 1, 0, -1):
        c = out[k]
        rl, _, rr = c.shape
        u, s, vt = sla.svd(c.reshape(rl, 2 * rr), full_matrices=False, lapack_driver="gesvd")
        r, e = choose_rank(s, chi, tol)
        errs[k - 1] = e
        svals[k - 1] = s
        out[k] = vt[:r].reshape(r, 2, rr)
        prev = out[k - 1]
        out[k - 1] = (prev.reshape(-1, rl) @ (u[:, :r] * s[:r])).reshape(prev.shape[0], 2, r)
    return out, errs, svals


def compress(cores, chi, tol):
    """QR sweep left to right, then truncated-SVD sweep right to left."""
    out, errs, _ = svd_sweep(qr_sweep(cores), chi, tol)
    return out, errs


def entanglement_entropy(s, r):
    """Main text, EE equation: -sum p log2 p, p_i = s_i^2 / sum_{i<r} s^2 over
    the r kept singular values of one bond."""
    p = np.asarray(s[:r], dtype=np.float64) ** 2
    tot = p.sum()
    if tot <= 0:
        return 0.0
    p = p[p > 0] / tot
    return float(-np.sum(p * np.log2(p)))


def compress_with_entropy(cores, chi, tol):
    """compress() that also returns the entropy of the kept values per bond."""
    out, errs, svals = svd_sweep(qr_sweep(cores), chi, tol)
    ee = [entanglement_entropy(svals[j], out[j + 1].shape[0]) for j in range(len(out) - 1)]
    return out, errs, ee


def compression_error(cores, chis, tol=0.0):
    """rms compression error against the bond dimension (main text, "State
    Compressibility", the rms error figure): for each D in chis,
    sqrt(mean((f - f_D)^2)) over all 2^n grid points, f_D the state
    compressed with bond cap D and tolerance tol."""
    f = to_dense(cores)
    out = []
    for chi in chis:
        fd = to_dense(compress(cores, chi, tol)[0])
        out.append(float(np.sqrt(np.mean((f - fd) ** 2))))
    return np.array(out)


def from_dense(vec, n, chi, tol):
    """Exact TT-SVD followed by :func:`compress` (used for f0 and for E)."""
    return compress(tt_svd(vec, n), chi, tol)[0]


def contract_sites(cores, sites, vectors):
    """Contract the physical leg of ``sites`` with ``vectors[k]`` (length 2).

    Returns the MPS on the remaining sites; the contracted sites' matrices are
    absorbed into the next remaining site on the right (or the left neighbour
    at the end).  Used for integration (SI "Integration").
    """
    keep = []
    pending = None
    for k, c in enumerate(cores):
        if k in sites:
            m = np.einsum("aib,i->ab", c, vectors[k])
            pending = m if pending is None else pending @ m
        else:
            if pending is not None:
                c = np.einsum("ab,bic->aic", pending, c)
                pending = None
            keep.append(c)
    if pending is not None:
        keep[-1] = np.einsum("aib,bc->aic", keep[-1], pending)
    return keep


def _lq(m):
    """m = L Q with Q having orthonormal rows (QR of the transpose)."""
    q, r = sla.qr(m.T, mode="economic")
    return r.T, q.T


def compress_modified(cores, chi, tol, split):
    """Modified centre-bond-first compression (SI "Modified Compression
    Scheme") of a sequentially ordered MPS whose first ``split`` sites hold
    one dimension (x) and the rest the other (v).

    1. Mixed canonical form about the centre bond: the v sites right of the
       first v site are right-canonicalised (LQ, factor pushed left), the x
       sites left-canonicalised (QR, R pushed right), and the first v site is
       split as C Q by one more LQ: C is the matrix of the centre bond.
    2. C = U S V^T, truncated by :func:`choose_rank`.
    3. S^{-1} S is inserted between S and V^T: the last x site takes U S, the
       first v site S V^T Q, and S^{-1} waits on the bond.  Each half then
       sees an orthonormal other half.
    4. Truncated-SVD sweep through the x sites, from the centre to the left
       end (the usual right-to-left step).
    5. The same through the v sites, from the centre to the right end
       (left-to-right steps: SVD of the (2 r_{k-1} x r_k) reshape, U kept,
       S V^T pushed right).
    6. S^{-1} is absorbed into the first v site (zero where S is zero).
    Returns (cores, truncation error per bond, singular values per bond).
    """
    out = [np.asarray(c, dtype=np.float64).copy() for c in cores]
    n = len(out)
    if not 0 < split < n:
        raise ValueError("split must leave sites on both sides")
    errs = [0.0] * (n - 1)
    svals = [None] * (n - 1)
    # 1. right-canonical v sites split+1 .. n-1
    for k in range(n - 1, split, -1):
        c = out[k]
        rl, _, rr = c.shape
        lm, q = _lq(c.reshape(rl, 2 * rr))
        p = q.shape[0]
        out[k] = q.reshape(p, 2, rr)
        prev = out[k - 1]
        out[k - 1] = (prev.reshape(-1, rl) @ lm).reshape(prev.shape[0], 2, p)
    # left-canonical x sites 0 .. split-1
    for k in range(split):
        c = out[k]
        rl, _, rr = c.shape
        q, r = sla.qr(c.reshape(rl * 2, rr), mode="economic")
        p = q.shape[1]
        out[k] = q.reshape(rl, 2, p)
        nxt = out[k + 1]
        out[k + 1] = (r @ nxt.reshape(rr, -1)).reshape(p, 2, nxt.shape[2])
    # the centre bond matrix
    c = out[split]
    rl, _, rr = c.shape
    cm, q = _lq(c.reshape(rl, 2 * rr))
    # 2. its SVD, truncated
    u, s, vt = sla.svd(cm, full_matrices=False, lapack_driver="gesvd")
    r, e = choose_rank(s, chi, tol)
    errs[split - 1], svals[split - 1] = e, s
    u, s, vt = u[:, :r], s[:r], vt[:r]
    # 3. U S to the left half, S V^T to the right half, S^{-1} on the bond
    prev = out[split - 1]
    out[split - 1] = (prev.reshape(-1, rl) @ (u * s)).reshape(prev.shape[0], 2, r)
    out[split] = ((s[:, None] * vt) @ q).reshape(r, 2, rr)
    # 4. x half, centre to left end
    for k in range(split - 1, 0, -1):
        c = out[k]
        a, _, b = c.shape
        uu, ss, vv = sla.svd(c.reshape(a, 2 * b), full_matrices=False, lapack_driver="gesvd")
        rk, ek = choose_rank(ss, chi, tol)
        errs[k - 1], svals[k - 1] = ek, ss
        out[k] = vv[:rk].reshape(rk, 2, b)
        prev = out[k - 1]
        out[k - 1] = (prev.reshape(-1, a) @ (uu[:, :rk] * ss[:rk])).reshape(prev.shape[0], 2, rk)
    # 5. v half, centre to right end
    for k in range(split, n - 1):
        c = out[k]
        a, _, b = c.shape
        uu, ss, vv = sla.svd(c.reshape(2 * a, b), full_matrices=False, lapack_driver="gesvd")
        rk, ek = choose_rank(ss, chi, tol)
        errs[k], svals[k] = ek, ss
        out[k] = uu[:, :rk].reshape(a, 2, rk)
        nxt = out[k + 1]
        out[k + 1] = ((ss[:rk, None] * vv[:rk]) @ nxt.reshape(b, -1)).reshape(rk, 2, nxt.shape[2])
    # 6. S^{-1} into the first v site
    inv = np.where(s > 0.0, 1.0 / np.where(s > 0.0, s, 1.0), 0.0)
    c = out[split]
    out[split] = (inv[:, None] * c.reshape(c.shape[0], -1)).reshape(c.shape)
    return out, errs, svals
