"""Index bookkeeping of the documented block layouts (include/tantrg.h,
kernel-level entry points): conversions between the library's block-sparse
arrays and dense arrays, for element-wise comparisons in the tests.

Site tensor: blocks (a_l sector l, pair charge p, a_r sector r) with
charge(r) = charge(l) + p, ordered by r, then l, then p (p in increasing
(n, 2Sz)); every block row-major [a_l][pair][a_r], the pairs (sigma, sigma')
of charge p in increasing 4 sigma + sigma'.  All blocks of one right sector
are therefore one contiguous row-major matrix.
Environment of a bond with MPO channel charges c_w: per ket sector b (bond
order) a row-major matrix of rows (w ascending, bra index a in sector
b + c_w, channels whose sector exists) and d_b columns.
"""
from __future__ import annotations

import numpy as np

# local basis |0>, |up>, |dn>, |up dn>: (particle number, 2 Sz)
LOCAL_Q = [(0, 0), (1, 1), (1, -1), (2, 0)]


def pair_table():
    """Pair charge p -> list of (sigma, sigma') in increasing 4 sigma + sigma'."""
    t = {}
    for a in range(4):
        for b in range(4):
            p = (LOCAL_Q[a][0] - LOCAL_Q[b][0], LOCAL_Q[a][1] - LOCAL_Q[b][1])
            t.setdefault(p, []).append((a, b))
    return dict(sorted(t.items()))


def offsets(sectors):
    """Dense offset of every sector and the total dimension."""
    off, o = [], 0
    for (_, _, d) in sectors:
        off.append(o)
        o += d
    return off, o


def site_blocks(sectors_l, sectors_r):
    """[(offset, l, pair charge, r)] in layout order and the total size."""
    pt = pair_table()
    idx_l = {(n, s): i for i, (n, s, _) in enumerate(sectors_l)}
    out, o = [], 0
    for r, (rn, rs, dr) in enumerate(sectors_r):
        for l, (ln, ls, dl) in enumerate(sectors_l):
            p = (rn - ln, rs - ls)
            if p in pt:
                out.append((o, l, p, r))
                o += dl * len(pt[p]) * dr
    return out, o


def right_groups(sectors_l, sectors_r):
    """[(offset, rows, d_r)] of the right-sector groups, in layout order."""
    pt = pair_table()
    out, off = [], 0
    for (rn, rs, dr) in sectors_r:
        rows = sum(dl * len(pt[(rn - ln, rs - ls)]) for (ln, ls, dl) in sectors_l if (rn - ln, rs - ls) in pt)
        if rows:
            out.append((off, rows, dr))
            off += rows * dr
    return out, off


def site_to_dense(x, sectors_l, sectors_r):
    """Block layout -> dense [a_l, sigma, sigma', a_r]."""
    pt = pair_table()
    ol, Dl = offsets(sectors_l)
    orr, Dr = offsets(sectors_r)
    X = np.zeros((Dl, 4, 4, Dr))
    blocks, total = site_blocks(sectors_l, sectors_r)
    assert total == x.size
    for (o, l, p, r) in blocks:
        dl, dr, pr = sectors_l[l][2], sectors_r[r][2], pt[p]
        b = x[o:o + dl * len(pr) * dr].reshape(dl, len(pr), dr)
        for k, (s, t) in enumerate(pr):
            X[ol[l]:ol[l] + dl, s, t, orr[r]:orr[r] + dr] = b[:, k, :]
    return X


def dense_to_site(X, sectors_l, sectors_r):
    """Dense [a_l, sigma, sigma', a_r] -> block layout (entries outside the
    charge-allowed blocks are dropped; see outside_blocks_norm)."""
    pt = pair_table()
    ol, _ = offsets(sectors_l)
    orr, _ = offsets(sectors_r)
    blocks, total = site_blocks(sectors_l, sectors_r)
    x = np.zeros(total)
    for (o, l, p, r) in blocks:
        dl, dr, pr = sectors_l[l][2], sectors_r[r][2], pt[p]
        b = np.empty((dl, len(pr), dr))
        for k, (s, t) in enumerate(pr):
            b[:, k, :] = X[ol[l]:ol[l] + dl, s, t, orr[r]:orr[r] + dr]
        x[o:o + b.size] = b.ravel()
    return x


def outside_blocks_norm(X, sectors_l, sectors_r):
    """Norm of the dense entries outside the charge-allowed blocks."""
    return float(np.sqrt(max(0.0, (X * X).sum() - (dense_to_site(X, sectors_l, sectors_r) ** 2).sum())))


def env_rows(sectors, chan):
    """[(ket b, offset, [(w, bra a, first row)], rows)] of the environment layout."""
    idx = {(n, s): i for i, (n, s, _) in enumerate(sectors)}
    out, o = [], 0
    for b, (bn, bs, db) in enumerate(sectors):
        rows, row = [], 0
        for w, (cn, cs) in enumerate(chan):
            a = idx.get((bn + cn, bs + cs))
            if a is not None:
                rows.append((w, a, row))
                row += sectors[a][2]
        out.append((b, o, rows, row))
        o += row * db
    return out, o


def env_to_dense(E, sectors, chan):
    """Environment layout -> dense [a, w, b] (bra a, channel w, ket b)."""
    off, D = offsets(sectors)
    T = np.zeros((D, len(chan), D))
    layout, total = env_rows(sectors, chan)
    assert total == E.size
    for (b, o, rows, nrow) in layout:
        db = sectors[b][2]
        M = E[o:o + nrow * db].reshape(nrow, db)
        for (w, a, r0) in rows:
            da = sectors[a][2]
            T[off[a]:off[a] + da, w, off[b]:off[b] + db] = M[r0:r0 + da]
    return T


def mpo_channel_charges(Ws):
    """Channel charges of every MPO bond from the dense tensors W_j[w, sigma,
    tau, w'] (nonzero entries force c_w' = c_w + q(sigma) - q(tau)); bond 0
    carries the single channel of charge 0."""
    ch = [[(0, 0)] * Ws[0].shape[0]]
    for W in Ws:
        nxt = [None] * W.shape[3]
        for wl, s, t, wr in zip(*np.nonzero(W)):
            c = (ch[-1][wl][0] + LOCAL_Q[s][0] - LOCAL_Q[t][0], ch[-1][wl][1] + LOCAL_Q[s][1] - LOCAL_Q[t][1])
            assert nxt[wr] in (None, c), "MPO tensor violates charge conservation"
            nxt[wr] = c
        ch.append([c if c is not None else (0, 0) for c in nxt])
    return ch


def mpo_terms(W):
    """Nonzero entries of W[w, sigma, tau, w'] as (w, w', sigma, tau, value)."""
    return [(int(a), int(d), int(b), int(c), float(W[a, b, c, d])) for a, b, c, d in zip(*np.nonzero(W))]
