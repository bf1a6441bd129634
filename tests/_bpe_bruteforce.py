"""Exhaustive BPE check over every A/C/G/T word of a given length, as whole
NumPy arrays (one row per word), for one merge table.

Two array restatements of reading C7 are computed independently of the C
oracle and of each other:
  * the literal greedy rule -- while a live adjacent pair is in the table,
    merge the pair of lowest rank, leftmost first;
  * the rank sweep -- for r = 0..M-1, merge every occurrence of pair r from
    left to right without overlap.
Merged positions become holes (-1) in place, so a row keeps its width; the
live entries of a row, in order, are its tokens.  The C oracle encodes the
same words as one RAW batch (one record per word) and must give the same
ids and per-record counts.  Every output token is also checked to be
self-encoding and every adjacent pair compatible (the property the CUDA
path's segment stitching relies on).
"""
from __future__ import annotations

import numpy as np

BIG = 1 << 14


def all_words(L: int) -> np.ndarray:
    """Every word of L codes (0..3); row i holds the base-4 digits of i, first
    symbol most significant."""
    i = np.arange(4 ** L, dtype=np.int64)
    return np.stack([(i >> (2 * (L - 1 - p))) & 3 for p in range(L)], axis=1).astype(np.int16)


def _links(tok):
    R, L = tok.shape
    nxt = np.empty((R, L), np.int16)
    prv = np.empty((R, L), np.int16)
    cur = np.full(R, L, np.int16)
    for p in range(L - 1, -1, -1):
        nxt[:, p] = cur
        cur = np.where(tok[:, p] >= 0, p, cur)
    cur = np.full(R, -1, np.int16)
    for p in range(L):
        prv[:, p] = cur
        cur = np.where(tok[:, p] >= 0, p, cur)
    return nxt, prv


def rank_sweep(words: np.ndarray, merges) -> np.ndarray:
    """For r = 0..M-1: every occurrence of pair r, left to right."""
    R, L = words.shape
    W1 = L + 1
    tok = np.concatenate([words, np.full((R, 1), -1, np.int16)], axis=1).ravel()
    nxt = np.empty((R, W1), np.int64)
    nxt[:, :L], _ = _links(words)
    nxt[:, L] = L
    nxt += (np.arange(R, dtype=np.int64) * W1)[:, None]  # flat positions
    nxt = nxt.ravel()
    base = np.arange(R, dtype=np.int64) * W1
    for r, (a, b) in enumerate(merges):
        for p in range(L - 1):
            fp = base + p
            cand = fp[tok[fp] == a]
            if not cand.size:
                continue
            j = nxt[cand]
            hit = tok[j] == b
            hp, jh = cand[hit], j[hit]
            tok[hp] = 4 + r
            tok[jh] = -1
            nxt[hp] = nxt[jh]
    return tok.reshape(R, W1)[:, :L].copy()


def greedy(words: np.ndarray, merges) -> np.ndarray:
    """Lowest-rank adjacent pair first, leftmost on ties, until none is left."""
    R, L = words.shape
    V = 4 + len(merges)
    rank = np.full((V + 1, V + 1), BIG, np.int16)  # index V: no token
    for r, (a, b) in enumerate(merges):
        rank[a, b] = r
    tok = words.copy()
    nxt, prv = _links(tok)
    right = np.where(nxt < L, tok[np.arange(R)[:, None], np.minimum(nxt, L - 1)], V)
    rk = rank[np.where(tok >= 0, tok, V), right]
    out = tok
    idx = np.arange(R)
    while idx.size:
        best = rk.min(axis=1)
        act = best < BIG
        if not act.all():
            out[idx[~act]] = tok[~act]
            idx, tok, nxt, prv, rk, best = (x[act] for x in (idx, tok, nxt, prv, rk, best))
        if not idx.size:
            break
        rows = np.arange(idx.size)
        p = rk.argmin(axis=1)  # leftmost of the minima
        j = nxt[rows, p]
        tok[rows, p] = 4 + best
        tok[rows, j] = -1
        rk[rows, j] = BIG
        nj = nxt[rows, j]
        nxt[rows, p] = nj
        has = nj < L
        prv[rows[has], nj[has]] = p[has]
        rk[rows, p] = np.where(has, rank[tok[rows, p], np.where(has, tok[rows, np.minimum(nj, L - 1)], V)], BIG)
        q = prv[rows, p]
        hq = q >= 0
        rk[rows[hq], q[hq]] = rank[tok[rows[hq], q[hq]], tok[rows[hq], p[hq]]]
    return out


def check_table(merges, max_len: int = 10):
    """All words of length 1..max_len under one table: greedy == rank sweep
    == the C oracle; outputs self-encoding and pairwise compatible.  Returns
    the number of words checked."""
    import oracle
    from oracle import literal

    m = np.array(merges, np.int32).reshape(-1, 2)
    V = 4 + len(merges)
    # token strings, self-encoding flags and the compatibility matrix from
    # the literal definition
    strs = [[t] for t in range(4)]
    for a, b in merges:
        strs.append(strs[a] + strs[b])
    selfenc = np.array([literal.bpe_greedy(s, merges) == [t] for t, s in enumerate(strs)])
    compat = np.zeros((V, V), bool)
    for a in range(V):
        for b in range(V):
            compat[a, b] = literal.bpe_greedy(strs[a] + strs[b], merges) == [a, b]
    n = 0
    for L in range(1, max_len + 1):
        W = all_words(L)
        g = greedy(W, merges)
        s = rank_sweep(W, merges)
        assert np.array_equal(g, s), "greedy and rank sweep differ (L=%d, table %s)" % (L, merges)
        live = g >= 0
        data = np.frombuffer(b"ACGT", np.uint8)[W.reshape(-1)]
        offs = np.arange(0, W.size + 1, L, dtype=np.int64)
        ids, o = oracle.encode(data, oracle.BPE, seq_offsets=offs, merges=m)
        assert np.array_equal(ids, g[live]), "oracle ids differ (L=%d, table %s)" % (L, merges)
        assert np.array_equal(np.diff(o), live.sum(axis=1)), "oracle offsets differ (L=%d)" % L
        assert selfenc[g[live]].all(), "a token that is not self-encoding (L=%d)" % L
        nxt, _ = _links(g)
        pl = live & (nxt < L)
        rr, pp = np.nonzero(pl)
        assert compat[g[rr, pp], g[rr, nxt[rr, pp]]].all(), "incompatible pair (L=%d)" % L
        n += W.shape[0]
    return n
