"""The algorithm the CUDA BPE path uses, written out plainly here and checked
by brute force against the oracle's greedy merge loop (C7: lowest rank
first, leftmost on ties).

Facts it rests on (each pinned below on exhaustive / random cases):
  1. Split: if BPE(w) has a token boundary at p, BPE(w) = BPE(w[:p]) +
     BPE(w[p:]) (merges never cross a final boundary and the merge decisions
     on each side depend only on that side).
  2. Characterization: a tokenization of w equals BPE(w) iff every token t
     is self-encoding (BPE(str t) = [t]) and every adjacent pair (a, b) is
     compatible (BPE(str a + str b) = [a, b]).
  3. Hence the last token of BPE(w[:i]) is the unique self-encoding token t
     that is a suffix of w[:i] and compatible with the last token of
     BPE(w[:i - |t|]) (any t at a word start).  A left-to-right pass that
     picks, at every i, the first such t (longest first) computes last(i)
     for every prefix; BPE(w) is read back from the end through
     i -> i - |last(i)|.
  4. Sync: the choice at i depends only on last(j) for j in [i - Lmax, i).
     A pass started at an arbitrary position (pretending a word starts
     there) therefore agrees with the true pass from the first window of
     Lmax consecutive agreeing values on.
"""
import itertools

import numpy as np

import oracle
from oracle import literal
from tests.test_oracle_pins import _tables


def _strings(merges):
    s = [(0,), (1,), (2,), (3,)]
    for a, b in merges:
        s.append(s[a] + s[b])
    return s


class Dp:
    def __init__(self, merges):
        self.merges = merges
        self.strs = _strings(merges)
        self.tok_of = {}
        for t, s in enumerate(self.strs):
            if literal.bpe_greedy(list(s), merges) == [t]:  # self-encoding only
                self.tok_of.setdefault(s, t)
        self.lmax = max(len(s) for s in self.tok_of)
        self.cache = {}

    def compat(self, a, b):
        key = (a, b)
        if key not in self.cache:
            self.cache[key] = literal.bpe_greedy(list(self.strs[a] + self.strs[b]),
                                                 self.merges) == [a, b]
        return self.cache[key]

    def forward(self, w, start=0, last=None):
        """last[i] = token ending at prefix length i, for i in (start, len(w)];
        position `start` acts as a word start."""
        last = [None] * (len(w) + 1) if last is None else last
        for i in range(start + 1, len(w) + 1):
            cands = [(L, self.tok_of[tuple(w[i - L:i])])
                     for L in range(min(self.lmax, i - start), 0, -1)
                     if tuple(w[i - L:i]) in self.tok_of]
            pick = cands[-1][1]  # deterministic choice if nothing fits
            for L, t in cands:
                if i - L == start or self.compat(last[i - L], t):
                    pick = t
                    break
            last[i] = pick
        return last

    def backtrack(self, last, n):
        out, i = [], n
        while i > 0:
            out.append(last[i])
            i -= len(self.strs[last[i]])
        return out[::-1]


def test_dp_equals_greedy_on_all_short_strings():
    for merges in _tables(6, seed=5):
        dp = Dp(merges)
        for L in range(1, 8):
            for w in itertools.product(range(4), repeat=L):
                want = oracle.bpe_word(np.array(w, np.int32), merges).tolist()
                assert dp.backtrack(dp.forward(list(w)), L) == want, (merges, w)


def test_dp_equals_greedy_on_random_words():
    rng = np.random.default_rng(31)
    for merges in _tables(30, seed=32):
        dp = Dp(merges)
        for _ in range(25):
            w = rng.integers(0, 4, size=int(rng.integers(10, 60))).tolist()
            want = oracle.bpe_word(np.array(w, np.int32), merges).tolist()
            assert dp.backtrack(dp.forward(w), len(w)) == want


def test_characterization_uniqueness_by_enumeration():
    """Every tokenization of w into self-encoding tokens with all adjacent
    pairs compatible is BPE(w) (so there is at most one)."""
    for merges in _tables(8, seed=41):
        dp = Dp(merges)
        for L in range(1, 7):
            for w in itertools.product(range(4), repeat=L):
                want = oracle.bpe_word(np.array(w, np.int32), merges).tolist()

                def splits(i):
                    if i == L:
                        yield []
                        return
                    for j in range(i + 1, min(L, i + dp.lmax) + 1):
                        t = dp.tok_of.get(tuple(w[i:j]))
                        if t is not None:
                            for rest in splits(j):
                                yield [t] + rest

                good = [s for s in splits(0)
                        if all(dp.compat(a, b) for a, b in zip(s, s[1:]))]
                assert good == [want], (merges, w, good)


def test_fresh_start_syncs_and_stays_synced():
    """A pass started mid-word agrees with the true pass after the first
    window of lmax agreeing values, at every later position."""
    rng = np.random.default_rng(51)
    m = np.loadtxt("tests/golden/bpe_merges_markov45_seed45_4096.txt", dtype=np.int64)[:600]
    merges = [tuple(x) for x in m.tolist()]
    dp = Dp(merges)
    w = rng.integers(0, 4, size=3000).tolist()
    truth = dp.forward(w)
    assert dp.backtrack(truth, len(w)) == oracle.bpe_word(np.array(w, np.int32), merges).tolist()
    for start in range(5, 2500, 211):
        part = dp.forward(w, start=start)
        run, synced_at = 0, None
        for i in range(start + 1, len(w) + 1):
            run = run + 1 if part[i] == truth[i] else 0
            if run >= dp.lmax:
                synced_at = i
                break
        assert synced_at is not None and synced_at - start < 200
        assert part[synced_at:] == truth[synced_at:]
