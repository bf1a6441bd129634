"""The host half of the split-stream protocol, without a GPU:
dnatok_part_combine against the scan element written out from its
definition on random spans of symbols and record boundaries (the state after
two spans must be the state of the one span they make), and the line-state
map composition the ranks do in Python against the FASTA line state machine
run byte by byte."""
import numpy as np
import pytest

import __graft_entry__


@pytest.fixture(scope="module")
def B():
    __graft_entry__.build()
    from paper_2601_05531_gb300 import binding
    return binding


def span_state(events, k):
    """The scan element of a span, from its definition.  events: symbol
    codes 0..4 (4 = N) and None for a record boundary.  Returns [nb, h, d, t,
    codes] (codes: the open record's last min(open, k - 1) symbols, 3 bits
    each, newest lowest, their number in bits 58..61)."""
    nb = sum(e is None for e in events)
    if nb == 0:
        h, t, d = len(events), 0, 0
        open_syms = list(events)
    else:
        first = events.index(None)
        last = len(events) - 1 - events[::-1].index(None)
        h = first
        open_syms = events[last + 1:]
        t = len(open_syms)
        d = 0
        run = 0
        for e in events[first + 1:last + 1]:  # records closed inside the span
            if e is None:
                d += -(-run // k)
                run = 0
            else:
                run += 1
        d += t // k
    tail = open_syms[len(open_syms) - min(len(open_syms), k - 1):] if k > 1 else []
    bits = 0
    for c in tail:
        bits = (bits << 3) | c
    codes = (len(tail) << 58) | bits if k > 1 else 0
    return [nb, h, d, t, codes]


def random_events(rng, n, p_bnd):
    return [None if rng.random() < p_bnd else int(rng.integers(0, 5)) for _ in range(n)]


@pytest.mark.parametrize("k", [1, 2, 3, 6, 13, 15])
def test_combine_matches_the_definition(B, k):
    rng = np.random.default_rng(100 + k)
    for trial in range(400):
        ev = random_events(rng, int(rng.integers(0, 60)), float(rng.choice([0.0, 0.02, 0.2, 0.6])))
        cut = int(rng.integers(0, len(ev) + 1))
        a = span_state(ev[:cut], k)
        b = span_state(ev[cut:], k)
        ls_a, ls_b = int(rng.integers(0, 3)), int(rng.integers(0, 3))
        got = B.dnatok_part_combine(k, B.PartState.from_list(a + [ls_a]),
                                    B.PartState.from_list(b + [ls_b])).as_list()
        want = span_state(ev, k) + [ls_b]
        assert got == want, (k, trial, ev, cut, got, want)


def test_combine_three_ways_and_identity(B):
    rng = np.random.default_rng(7)
    k = 6
    for _ in range(200):
        ev = random_events(rng, 80, 0.05)
        i, j = sorted(rng.integers(0, len(ev) + 1, size=2))
        s = [B.PartState.from_list(span_state(x, k) + [2]) for x in (ev[:i], ev[i:j], ev[j:])]
        left = B.dnatok_part_combine(k, B.dnatok_part_combine(k, s[0], s[1]), s[2]).as_list()
        right = B.dnatok_part_combine(k, s[0], B.dnatok_part_combine(k, s[1], s[2])).as_list()
        assert left == right == span_state(ev, k) + [2]
        zero = B.PartState.from_list([0, 0, 0, 0, 0, 2])
        assert B.dnatok_part_combine(k, zero, s[1]).as_list() == s[1].as_list()
        assert B.dnatok_part_combine(k, s[1], zero).as_list() == s[1].as_list()


def test_combine_refuses_bad_k(B):
    z = B.PartState()
    for k in (0, 16):
        with pytest.raises(B.DnatokError):
            B.dnatok_part_combine(k, z, z)


def line_states(text, s=0):
    """The FASTA line state after each prefix (0 line start, 1 header, 2
    sequence), byte by byte."""
    for b in text:
        if b == ord("\n"):
            s = 0
        elif s == 0:
            s = 1 if b == ord(">") else 2
    return s


def line_map(text):
    """What dnatok_part_line_map computes, from its definition: the end
    state for each start state."""
    return sum(line_states(text, s) << (2 * s) for s in range(3))


def test_line_maps_compose_to_the_byte_by_byte_state():
    # the composition StreamPart.summary does, against one walk over the text
    rng = np.random.default_rng(3)
    alphabet = np.frombuffer(b">ACGTN\n\r x", np.uint8)
    for _ in range(300):
        text = bytes(rng.choice(alphabet, size=int(rng.integers(0, 40))))
        cuts = sorted(rng.integers(0, len(text) + 1, size=3))
        parts = [text[a:b] for a, b in zip([0] + cuts, cuts + [len(text)])]
        s = 0
        for r, part in enumerate(parts):
            assert s == line_states(text[:sum(len(p) for p in parts[:r])])
            s = (line_map(part) >> (2 * s)) & 3
        assert s == line_states(text)
