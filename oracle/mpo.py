"""MPOs of the SI, written out as printed (oracle; test infrastructure only).

An MPO is a list of cores ``B[k]`` with shape ``(w_left, 2_out, 2_in, w_right)``
(SI "Matrix-vector multiplication": ``B^{(n)}_{beta_{n-1}, beta_n}(o_n, i_n)``).
Site 0 is the most significant bit (the coarse grid, main text "MPS
Representation": the n-th point is indexed by the binary digits of n).

The single-bit operators are ``S+ = [[0,0],[1,0]]`` and ``S- = [[0,1],[0,0]]``
as [out, in] matrices (SI "First Derivative, Centered, Periodic").
A chain printed as ``row * M * M ... * M * col`` places the row on site 0,
M on the interior sites and the column on the last site.
"""
from __future__ import annotations

import numpy as np

I2 = np.eye(2)
Z2 = np.zeros((2, 2))
SP = np.array([[0.0, 0.0], [1.0, 0.0]])
SM = np.array([[0.0, 1.0], [0.0, 0.0]])
P0 = np.array([[1.0, 0.0], [0.0, 0.0]])
P1 = np.array([[0.0, 0.0], [0.0, 1.0]])


def _core(blocks):
    """Operator-valued matrix (list of lists of 2x2) -> core (wl, 2, 2, wr)."""
    wl, wr = len(blocks), len(blocks[0])
    c = np.zeros((wl, 2, 2, wr))
    for a in range(wl):
        for b in range(wr):
            c[a, :, :, b] = blocks[a][b]
    return c


def _chain(L, row, mid, col, before_last=None, scale=1.0):
    """Cores of ``row * mid^(L-2) * col`` (``before_last`` replaces site L-2)."""
    if L < 2:
        raise ValueError("the printed chains need at least two sites")
    cores = [_core([row])]
    for k in range(1, L - 1):
        m = before_last if (before_last is not None and k == L - 2) else mid
        cores.append(_core(m))
    cores.append(_core([[c] for c in col]))
    cores[0] = cores[0] * scale
    return cores


def centered_periodic(L, dx):
    """SI "First Derivative, Centered, Periodic Boundary Conditions", c1 = 1/2."""
    c1 = 0.5
    row = [I2, SP + SM, SP + SM]
    mid = [[I2, SM, SP], [Z2, SP, Z2], [Z2, Z2, SM]]
    col = [c1 * (SM - SP), c1 * SP, -c1 * SM]
    return _chain(L, row, mid, col, scale=1.0 / dx)


def _forward_like(L, dx, c0, c1, c2, plus, minus):
    # SI "First Derivative, Forward, Periodic": c3 appears in the printed last
    # core but is never given a value; c3 = 0 reproduces the forward stencil.
    c3 = 0.0
    row = [I2, minus, plus]
    mid = [[I2, minus, Z2], [Z2, plus, Z2], [Z2, Z2, plus]]
    blast = [[I2, minus, Z2], [Z2, plus, Z2], [Z2, plus, I2]]
    col = [c0 * I2 + c1 * minus, c1 * plus + c2 * I2 + c3 * minus, c3 * plus]
    if L < 3:
        raise ValueError("the printed forward/backward chain needs at least three sites")
    return _chain(L, row, mid, col, before_last=blast, scale=1.0 / dx)


def forward_periodic(L, dx):
    """SI "First Derivative, Forward": c0=-3/2, c1=2, c2=-1/2."""
    return _forward_like(L, dx, -1.5, 2.0, -0.5, SP, SM)


def backward_periodic(L, dx):
    """SI "First Derivative, Backward": forward with S+ <-> S-, c0=3/2, c1=-2, c2=1/2."""
    return _forward_like(L, dx, 1.5, -2.0, 0.5, SM, SP)


def centered_zero_gradient(L, dx):
    """SI "First Derivative, Centered, Zero Gradient Boundary Conditions".

    Backbone (non-periodic centred chain) plus the two ghost-cell corrections.
    M_right is used as printed (row N-1 gains +c1 f_{N-2}, so the derivative at
    the last node is zero).  The printed M_left places its 2x2 block on the
    first site with P1 on the others, which lands on row N/2-1; read as the
    mirror image of M_right: row 0 gains -c1 f_1 (P0 on every site but the
    last, whose block is ``[[0,-c1],[0,0]]``), so the derivative at the first
    node is zero as well.
    """
    c1 = 0.5
    row = [I2, SM, SP]
    mid = [[I2, SM, SP], [Z2, SP, Z2], [Z2, Z2, SM]]
    col = [c1 * (SM - SP), c1 * SP, -c1 * SM]
    backbone = _chain(L, row, mid, col)
    m_left = [P0[None, :, :, None].copy() for _ in range(L - 1)]
    m_left.append(np.array([[0.0, -c1], [0.0, 0.0]])[None, :, :, None])
    m_right = [P1[None, :, :, None].copy() for _ in range(L - 1)]
    m_right.append(np.array([[0.0, 0.0], [c1, 0.0]])[None, :, :, None])
    op = mpo_sum(mpo_sum(backbone, m_left), m_right)
    op[0] = op[0] / dx
    return op


def second_periodic(L, dx):
    """SI "Second Derivative, Centered, Periodic": c0=-2, c1=1."""
    c0, c1 = -2.0, 1.0
    row = [I2, SP + SM, SP + SM]
    mid = [[I2, SP, SM], [Z2, SM, Z2], [Z2, Z2, SP]]
    col = [c0 * I2 + c1 * (SM + SP), c1 * SM, c1 * SP]
    return _chain(L, row, mid, col, scale=1.0 / (dx * dx))


def second_zero_gradient(L, dx):
    """Second derivative with the zero-gradient ghosts of
    :func:`centered_zero_gradient` (f_{-1} = f_1, f_N = f_{N-2}): the
    non-periodic backbone of "Second Derivative, Centered" (the carry that
    would wrap around is absorbed at the first site) plus row 0 += c1 f_1 and
    row N-1 += c1 f_{N-2}.  Used by the Dougherty diffusion term (Methods,
    "Collision Operator"); the SI prints no zero-gradient second derivative."""
    c0, c1 = -2.0, 1.0
    row = [I2, SP, SM]
    mid = [[I2, SP, SM], [Z2, SM, Z2], [Z2, Z2, SP]]
    col = [c0 * I2 + c1 * (SM + SP), c1 * SM, c1 * SP]
    backbone = _chain(L, row, mid, col)
    m_left = [P0[None, :, :, None].copy() for _ in range(L - 1)]
    m_left.append(np.array([[0.0, c1], [0.0, 0.0]])[None, :, :, None])
    m_right = [P1[None, :, :, None].copy() for _ in range(L - 1)]
    m_right.append(np.array([[0.0, 0.0], [c1, 0.0]])[None, :, :, None])
    op = mpo_sum(mpo_sum(backbone, m_left), m_right)
    op[0] = op[0] / (dx * dx)
    return op


def mpo_product(a, b):
    """The MPO of a @ b (b acts first): per site C[(l,m), o, i, (r,s)] =
    sum_j a[l, o, j, r] b[m, j, i, s]."""
    out = []
    for A, B in zip(a, b):
        c = np.einsum("lojr,mjis->lmoirs", A, B)
        s = c.shape
        out.append(c.reshape(s[0] * s[1], 2, 2, s[4] * s[5]))
    return out


def identity(L):
    return [I2[None, :, :, None].copy() for _ in range(L)]


def mpo_sum(a, b):
    """Sum of two MPOs: block-diagonal cores (SI "Addition", applied to MPOs)."""
    L = len(a)
    out = []
    for k in range(L):
        A, B = a[k], b[k]
        if L == 1:
            out.append(A + B)
        elif k == 0:
            out.append(np.concatenate([A, B], axis=3))
        elif k == L - 1:
            out.append(np.concatenate([A, B], axis=0))
        else:
            c = np.zeros((A.shape[0] + B.shape[0], 2, 2, A.shape[3] + B.shape[3]))
            c[:A.shape[0], :, :, :A.shape[3]] = A
            c[A.shape[0]:, :, :, A.shape[3]:] = B
            out.append(c)
    return out


def mpo_scale(a, s):
    out = [c.copy() for c in a]
    out[0] = out[0] * s
    return out


def diag_from_mps(cores):
    """SI "Dot Product": M(o, i) = M(i) delta_{i,o}."""
    out = []
    for c in cores:
        d = np.zeros((c.shape[0], 2, 2, c.shape[2]))
        d[:, 0, 0, :] = c[:, 0, :]
        d[:, 1, 1, :] = c[:, 1, :]
        out.append(d)
    return out


def reverse(chain):
    """The same operator (or MPS) with its sites in the opposite order: core k
    of the result is core L-1-k with its two bonds exchanged."""
    if chain[0].ndim == 3:
        return [c.transpose(2, 1, 0).copy() for c in chain[::-1]]
    return [c.transpose(3, 1, 2, 0).copy() for c in chain[::-1]]


def place(factors, sitemap):
    """Tensor product of per-dimension MPOs placed on an MPS site ordering.

    ``factors[d]`` is the MPO acting on the bits of dimension d, its cores in
    the order in which the site map meets that dimension's bits
    (``sitemap[k] = (d, b)``: site k carries bit b of dimension d).  A
    dimension that is not yet entered or already left carries its bond
    through the site unchanged, so the bond at a cut is the product of the
    per-dimension bonds there.
    """
    ndim = len(factors)
    pos = [0] * ndim
    out = []
    for (d, b) in sitemap:
        left = [factors[e][pos[e]].shape[0] if pos[e] < len(factors[e]) else factors[e][-1].shape[3]
                for e in range(ndim)]
        core = factors[d][pos[d]]
        # dimensions other than d contribute an identity on their bond
        c = core
        before = int(np.prod(left[:d])) if d > 0 else 1
        after = int(np.prod(left[d + 1:])) if d + 1 < ndim else 1
        wl, wr = core.shape[0], core.shape[3]
        # full[p,a,r,o,i,q,b,s] = delta_pq * core[a,o,i,b] * delta_rs; the bond
        # index flattens the per-dimension channels in dimension order.
        full = np.einsum("pq,aoib,rs->paroiqbs", np.eye(before), c, np.eye(after))
        full = full.reshape(before * wl * after, 2, 2, before * wr * after)
        out.append(full)
        pos[d] += 1
    return out


def to_dense(cores):
    """Contract an MPO into the dense 2^L x 2^L matrix [out, in] (tests, small L)."""
    t = cores[0]  # (1, o, i, w)
    for c in cores[1:]:
        t = np.einsum("aoiw,wpjb->aopijb", t, c)
        s = t.shape
        t = t.reshape(s[0], s[1] * s[2], s[3] * s[4], s[5])
    return t[0, :, :, 0]
