"""Pins for the CPU oracle: each test checks it against something other than
itself -- hand-worked values from the paper's tables, closed forms, invariants,
and literal brute-force definitions on tiny inputs."""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import literal
from tests import _golden as G

PAPER_FALLBACK = np.zeros(256, dtype=np.int32)
for _c, _v in zip(b"ACGTNacgtn", [1, 2, 3, 4, 0, 1, 2, 3, 4, 0]):
    PAPER_FALLBACK[_c] = _v


def _lut(name):
    return PAPER_FALLBACK if name == "paper_fallback" else None


# ---------------------------------------------------------------- single base

def test_char_worked_examples():
    n = 0
    for lut_name, text, want in G.rows("char_worked_example.txt"):
        ids, offs = oracle.encode(G.unescape(text), oracle.CHAR, lut=_lut(lut_name))
        assert ids.tolist() == G.ints(want), (lut_name, text)
        assert offs.tolist() == [0, len(G.ints(want))]
        n += 1
    assert n >= 7


def test_default_lut_matches_reading_c5():
    lut = oracle.default_lut()
    for b in range(256):
        ch = bytes([b])
        if ch in b"ACGT":
            want = b"ACGT".index(ch)
        elif ch in b"acgt":
            want = b"acgt".index(ch)
        elif ch in b"\n\r \t":
            want = -1
        else:
            want = 4
        assert lut[b] == want, b


# ---------------------------------------------------------------------- k-mer

def test_kmer_closed_form_examples():
    n = 0
    for k, text, want in G.rows("kmer_closed_form.txt"):
        ids, _ = oracle.encode(G.unescape(text), oracle.KMER, k=int(k))
        assert ids.tolist() == G.ints(want), (k, text)
        n += 1
    assert n >= 18


@pytest.mark.parametrize("k", [1, 2, 3, 5, 6, 7, 15])
def test_kmer_matches_literal_definition(k):
    data = synth.iid_sequence(3000, seed=100 + k, n_fraction=0.02, lower_fraction=0.2)
    ids, _ = oracle.encode(data, oracle.KMER, k=k)
    sym = literal.kept_symbols(bytes(data))
    assert ids.tolist() == literal.kmer_ids(sym, k)


@pytest.mark.parametrize("L,k", [(0, 6), (1, 6), (5, 6), (6, 6), (13, 6), (12, 6), (7, 1),
                                 (29, 15), (30, 15)])
def test_kmer_output_length_is_ceil(L, k):
    data = synth.iid_sequence(L, seed=L * 31 + k, n_fraction=0.0) if L else np.zeros(0, np.uint8)
    ids, offs = oracle.encode(data, oracle.KMER, k=k)
    assert len(ids) == (L + k - 1) // k == L // k + (L % k > 0)
    if L % k:
        assert ids[-1] == 4 ** k


def test_k1_equals_default_char():
    data = synth.random_bytes(5000, seed=7)
    a, oa = oracle.encode(data, oracle.KMER, k=1)
    b, ob = oracle.encode(data, oracle.CHAR)
    assert a.tolist() == b.tolist() and oa.tolist() == ob.tolist()


@pytest.mark.parametrize("mode,k", [(oracle.CHAR, 1), (oracle.KMER, 6), (oracle.KMER, 4),
                                    (oracle.BPE, 1), (oracle.KMER_OVERLAP, 6)])
def test_separator_insertion_is_invariant(mode, k):
    rng = np.random.default_rng(11)
    merges = [(0, 0), (1, 2), (4, 3), (2, 2), (5, 0)]
    base = synth.iid_sequence(2000, seed=12, n_fraction=0.01, lower_fraction=0.1)
    ref, _ = oracle.encode(base, mode, k=k, merges=merges)
    for trial in range(5):
        pos = np.sort(rng.choice(len(base) + 1, size=60))
        seps = rng.choice(np.frombuffer(b"\n\r \t", np.uint8), size=60)
        wrapped = np.insert(base, pos, seps)
        got, _ = oracle.encode(wrapped, mode, k=k, merges=merges)
        assert got.tolist() == ref.tolist()


# ------------------------------------------------------ overlapping k-mers

def test_kmer_overlap_hand_examples():
    n = 0
    for k, text, want in G.rows("kmer_overlap_examples.txt"):
        ids, offs = oracle.encode(G.unescape(text), oracle.KMER_OVERLAP, k=int(k))
        assert ids.tolist() == G.ints(want), (k, text)
        assert offs.tolist() == [0, len(G.ints(want))]
        n += 1
    assert n >= 11


@pytest.mark.parametrize("k", [1, 2, 3, 5, 6, 9, 15])
def test_kmer_overlap_matches_literal_definition(k):
    data = synth.iid_sequence(2500, seed=200 + k, n_fraction=0.03, lower_fraction=0.2)
    rng = np.random.default_rng(k)
    pos = np.sort(rng.choice(len(data) + 1, size=40))
    data = np.insert(data, pos, rng.choice(np.frombuffer(b"\n\r \t", np.uint8), size=40))
    ids, _ = oracle.encode(data, oracle.KMER_OVERLAP, k=k)
    assert ids.tolist() == literal.kmer_overlap(bytes(data), k)


def test_kmer_overlap_counts_per_record():
    # L - k + 1 tokens per record (none when L < k), records independent
    rng = np.random.default_rng(3)
    lens = [0, 1, 5, 6, 7, 40, 3, 6]
    data, offs = synth.markov_batch(lens, 0.4, seed=3)
    for k in (1, 6, 7):
        ids, o = oracle.encode(data, oracle.KMER_OVERLAP, k=k, seq_offsets=offs)
        assert np.diff(o).tolist() == [max(0, L - k + 1) for L in lens]
        for r, L in enumerate(lens):
            rec = bytes(data[offs[r]:offs[r + 1]])
            assert ids[o[r]:o[r + 1]].tolist() == literal.kmer_overlap(rec, k)


@pytest.mark.parametrize("k", [2, 4, 6, 11])
def test_kmer_overlap_every_kth_window_is_the_blocked_kmer(k):
    data = synth.iid_sequence(30 * k + 7, seed=k, n_fraction=0.02, lower_fraction=0.1)
    ovl, _ = oracle.encode(data, oracle.KMER_OVERLAP, k=k)
    blk, _ = oracle.encode(data, oracle.KMER, k=k)
    full = len(data) // k  # blocks without the UNK tail
    assert ovl[::k][:full].tolist() == blk[:full].tolist()


def test_kmer_overlap_k1_equals_default_char():
    data = synth.random_bytes(3000, seed=8)
    a, oa = oracle.encode(data, oracle.KMER_OVERLAP, k=1)
    b, ob = oracle.encode(data, oracle.CHAR)
    assert a.tolist() == b.tolist() and oa.tolist() == ob.tolist()


def test_kmer_overlap_fasta_matches_records():
    text = synth.fuzz_fasta(5, n_records=6, max_len=300)
    ids, offs = oracle.encode(text, oracle.KMER_OVERLAP, k=5, fmt=oracle.FASTA)
    recs = literal.fasta_records(bytes(text))
    assert len(offs) == len(recs) + 1
    for r, body in enumerate(recs):
        assert ids[offs[r]:offs[r + 1]].tolist() == literal.kmer_overlap(body, 5)


# --------------------------------------------------------------------- decode

def test_decode_roundtrip_kmer_overlap():
    for k in (1, 3, 6, 15):
        data = synth.iid_sequence(500 + k, seed=40 + k, n_fraction=0.0, lower_fraction=0.3)
        ids, _ = oracle.encode(data, oracle.KMER_OVERLAP, k=k)
        assert len(ids) == len(data) - k + 1
        assert oracle.decode(ids, oracle.KMER_OVERLAP, k=k) == bytes(data).upper()


def test_decode_roundtrip_kmer():
    for k in (1, 2, 6, 11, 15):
        data = synth.iid_sequence(k * 200, seed=k, n_fraction=0.0, lower_fraction=0.3)
        ids, _ = oracle.encode(data, oracle.KMER, k=k)
        assert oracle.decode(ids, oracle.KMER, k=k) == bytes(data).upper()


def test_decode_roundtrip_char_with_n():
    data = synth.random_bytes(4000, seed=3)
    ids, _ = oracle.encode(data, oracle.CHAR)
    txt = bytes(data)
    want = bytes(c if c in b"ACGT" else ord("N")
                 for c in txt.upper() if c not in b"\n\r \t")
    # upper() maps bytes >= 128 unchanged and they are N-class, as are IUPAC
    assert oracle.decode(ids, oracle.CHAR) == want


def test_decode_roundtrip_bpe():
    corpus = synth.bpe_training_corpus(seed=5, n=20000)
    merges = oracle.bpe_train(oracle.codes_of(bytes(corpus)), 200)
    data = synth.iid_sequence(5000, seed=9, n_fraction=0.02, lower_fraction=0.1)
    ids, _ = oracle.encode(data, oracle.BPE, merges=merges)
    txt = bytes(data).upper()
    want = bytes(c if c in b"ACGT" else ord("N") for c in txt if c not in b"\n\r \t")
    assert oracle.decode(ids, oracle.BPE, merges=merges) == want


# ---------------------------------------------------------------------- FASTA

def test_fasta_hand_example():
    kv = G.keyvals("fasta_records.txt")
    for sfx in ("", "2"):
        text = G.unescape(kv["text" + sfx])
        ids, offs = oracle.encode(text, oracle.KMER, k=2, fmt=oracle.FASTA)
        assert ids.tolist() == G.ints(kv["kmer2_ids" + sfx])
        assert offs.tolist() == G.ints(kv["kmer2_offsets" + sfx])
        ids, offs = oracle.encode(text, oracle.CHAR, fmt=oracle.FASTA)
        assert ids.tolist() == G.ints(kv["char_ids" + sfx])
        assert offs.tolist() == G.ints(kv["char_offsets" + sfx])


def test_fasta_empty_and_degenerate():
    ids, offs = oracle.encode(b"", oracle.KMER, k=6, fmt=oracle.FASTA)
    assert ids.size == 0 and offs.tolist() == [0]
    ids, offs = oracle.encode(b">only a header", oracle.CHAR, fmt=oracle.FASTA)
    assert ids.size == 0 and offs.tolist() == [0, 0]
    ids, offs = oracle.encode(b">\n>\n>\n", oracle.CHAR, fmt=oracle.FASTA)
    assert offs.tolist() == [0, 0, 0, 0]
    ids, offs = oracle.encode(b"\n>a\nAC", oracle.CHAR, fmt=oracle.FASTA)
    assert offs.tolist() == [0, 0, 2] and ids.tolist() == [0, 1]


@pytest.mark.parametrize("seed", range(40))
def test_fasta_matches_line_based_definition(seed):
    text = bytes(synth.fuzz_fasta(seed))
    merges = [(0, 1), (2, 3), (4, 5), (0, 0), (6, 6)]
    recs = literal.fasta_records(text)
    lut = oracle.default_lut()
    for mode, k in ((oracle.CHAR, 1), (oracle.KMER, 3), (oracle.KMER, 6), (oracle.BPE, 1)):
        ids, offs = oracle.encode(text, mode, k=k, fmt=oracle.FASTA, merges=merges)
        want, woffs = [], [0]
        for body in recs:
            if mode == oracle.CHAR:
                want += literal.char_ids(body, lut)
            elif mode == oracle.KMER:
                want += literal.kmer_ids(literal.kept_symbols(body), k)
            else:
                want += literal.bpe_ids(literal.kept_symbols(body), merges)
            woffs.append(len(want))
        assert ids.tolist() == want, (seed, mode, k)
        assert offs.tolist() == woffs, (seed, mode, k)


def test_raw_records_concatenate():
    data, offs = synth.markov_batch([0, 5, 1, 0, 300, 17, 0], 0.4, seed=3)
    for mode, k in ((oracle.CHAR, 1), (oracle.KMER, 6), (oracle.BPE, 1)):
        merges = [(0, 1), (2, 2), (4, 3)]
        ids, ioffs = oracle.encode(data, mode, k=k, seq_offsets=offs, merges=merges)
        for r in range(len(offs) - 1):
            one, _ = oracle.encode(data[offs[r]:offs[r + 1]], mode, k=k, merges=merges)
            assert ids[ioffs[r]:ioffs[r + 1]].tolist() == one.tolist()


def test_bad_arguments_rejected():
    with pytest.raises(RuntimeError):
        oracle.encode(b"ACGT", oracle.KMER, k=16)
    with pytest.raises(RuntimeError):
        oracle.encode(b"ACGT", oracle.KMER, k=0)
    with pytest.raises(RuntimeError):
        oracle.encode(b"ACGT", oracle.CHAR, seq_offsets=np.array([0, 3, 2, 4]))
    with pytest.raises(RuntimeError):
        oracle.encode(b"ACGT", oracle.CHAR, seq_offsets=np.array([0, 3]))


# ------------------------------------------------------------------------ BPE

def test_bpe_hand_examples():
    n = 0
    for m, text, want in G.rows("bpe_hand.txt"):
        merges = G.merges(m)
        ids, _ = oracle.encode(G.unescape(text), oracle.BPE, merges=merges)
        assert ids.tolist() == G.ints(want), (m, text)
        n += 1
    assert n >= 11


def test_bpe_without_merges_is_char():
    data = synth.iid_sequence(2000, seed=21)
    a, _ = oracle.encode(data, oracle.BPE, merges=[])
    b, _ = oracle.encode(data, oracle.CHAR)
    assert a.tolist() == b.tolist()


def random_table(rng, m, max_id_bias=True):
    seen, out = set(), []
    while len(out) < m:
        hi = 4 + len(out)
        if max_id_bias:
            a = int(min(rng.geometric(0.35) - 1, hi - 1))
            b = int(min(rng.geometric(0.35) - 1, hi - 1))
            if rng.random() < 0.5:
                a = int(rng.integers(0, hi))
        else:
            a, b = int(rng.integers(0, hi)), int(rng.integers(0, hi))
        if (a, b) not in seen:
            seen.add((a, b))
            out.append((a, b))
    return out


def _tables(n, seed):
    rng = np.random.default_rng(seed)
    tabs = [random_table(rng, int(rng.integers(1, 13)), bool(i % 2)) for i in range(n)]
    # tables the trainer learns on short random strings
    for i in range(4):
        s = rng.integers(0, 4, size=200).astype(np.uint8)
        tabs.append([tuple(x) for x in oracle.bpe_train(s, 12).tolist()])
    return tabs


def test_bpe_bruteforce_all_short_strings():
    """Every A/C/G/T word of length 1..10 under 50 random valid tables of at
    most 12 merges (46 drawn at random, 4 learned by the trainer): the
    literal greedy rule, the rank sweep and the C oracle agree on every word,
    and every output is self-encoding and pairwise compatible (reading C7).
    Tables are checked in worker processes (spawned, so no inherited state)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    from tests import _bpe_bruteforce

    tables = _tables(46, seed=5)
    assert len(tables) == 50 and all(1 <= len(t) <= 12 for t in tables)
    workers = max(1, min(len(tables), len(os.sched_getaffinity(0))))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        counts = list(ex.map(_bpe_bruteforce.check_table, tables))
    assert counts == [sum(4 ** L for L in range(1, 11))] * 50


def test_bpe_bruteforce_literal_empty_and_short():
    """The Python literal definitions themselves on every word of length
    0..5 (the array forms above start at length 1)."""
    tables = _tables(6, seed=5)
    words = [w for L in range(0, 6) for w in itertools.product(range(4), repeat=L)]
    for merges in tables:
        for w in words:
            c = oracle.bpe_word(np.array(w, dtype=np.int32), merges).tolist()
            assert c == literal.bpe_greedy(w, merges), (merges, w)
            assert c == literal.bpe_rank_sweep(w, merges), (merges, w)


def test_bpe_bruteforce_random_longer():
    rng = np.random.default_rng(8)
    tables = _tables(44, seed=9)
    for merges in tables:
        for _ in range(40):
            w = rng.integers(0, 4, size=int(rng.integers(8, 11))).tolist()
            c = oracle.bpe_word(np.array(w, dtype=np.int32), merges).tolist()
            assert c == literal.bpe_greedy(w, merges)
            assert c == literal.bpe_rank_sweep(w, merges)


def _text_of(t, merges):
    return oracle.decode(np.array([t], np.int32), oracle.BPE, merges=merges)


def _compatible(a, b, merges):
    s = oracle.codes_of(_text_of(a, merges) + _text_of(b, merges))
    return oracle.bpe_word(s, merges).tolist() == [a, b]


def test_bpe_split_certificate():
    """If the last token of BPE(u) and the first of BPE(v) re-encode to
    themselves when joined, BPE(uv) = BPE(u) + BPE(v).  The CUDA path stitches
    independently encoded pieces with exactly this check."""
    rng = np.random.default_rng(13)
    checked = 0
    for merges in _tables(30, seed=14):
        for _ in range(60):
            u = rng.integers(0, 4, size=int(rng.integers(1, 9))).astype(np.int32)
            v = rng.integers(0, 4, size=int(rng.integers(1, 9))).astype(np.int32)
            bu, bv = oracle.bpe_word(u, merges), oracle.bpe_word(v, merges)
            buv = oracle.bpe_word(np.concatenate([u, v]), merges)
            if _compatible(int(bu[-1]), int(bv[0]), merges):
                checked += 1
                assert buv.tolist() == bu.tolist() + bv.tolist()
    assert checked > 200


def test_bpe_output_is_self_encoding_and_pairwise_compatible():
    rng = np.random.default_rng(15)
    for merges in _tables(20, seed=16):
        for _ in range(30):
            w = rng.integers(0, 4, size=int(rng.integers(2, 12))).astype(np.int32)
            out = oracle.bpe_word(w, merges).tolist()
            for t in out:
                assert oracle.bpe_word(oracle.codes_of(_text_of(t, merges)), merges).tolist() == [t]
            for a, b in zip(out, out[1:]):
                assert _compatible(a, b, merges)


# -------------------------------------------------------------------- trainer

def test_trainer_hand_examples():
    n = 0
    for corpus, m, want in G.rows("bpe_train_hand.txt"):
        got = oracle.bpe_train(oracle.codes_of(corpus), int(m))
        assert [tuple(x) for x in got.tolist()] == G.merges(want), corpus
        n += 1
    assert n >= 6


def test_trainer_is_deterministic_and_valid():
    corpus = oracle.codes_of(bytes(synth.bpe_training_corpus(seed=77, n=50000)))
    a = oracle.bpe_train(corpus, 300)
    b = oracle.bpe_train(corpus.copy(), 300)
    assert a.tolist() == b.tolist() and len(a) == 300
    seen = set()
    for r, (l, rr) in enumerate(a.tolist()):
        assert 0 <= l < 4 + r and 0 <= rr < 4 + r
        assert (l, rr) not in seen
        seen.add((l, rr))


def test_trainer_first_merge_is_most_frequent_pair():
    rng = np.random.default_rng(3)
    for _ in range(5):
        s = rng.integers(0, 4, size=500).astype(np.uint8)
        counts = {}
        for a, b in zip(s[:-1], s[1:]):
            counts[(int(a), int(b))] = counts.get((int(a), int(b)), 0) + 1
        best = max(counts.items(), key=lambda kv: (kv[1], (-kv[0][0], -kv[0][1])))[0]
        assert tuple(oracle.bpe_train(s, 1)[0].tolist()) == best


# ------------------------------------------------- table-driven k-mers (C16)

def _closed4(digits):
    v = 0
    for d in digits:
        v = 4 * v + d
    return v


def _digits5(index, k):
    out = []
    for _ in range(k):
        out.append(index % 5)
        index //= 5
    return out[::-1]


def ktab_named(name):
    """The tables the hand-worked fixture names, built from their stated rules."""
    if name == "T1":
        return 1, np.array([7, 8, 9, 10, -1], np.int32), np.array([0, 1, 2, 3, 4], np.int32)
    if name == "T2":
        lut = np.array([10 + i if 4 not in _digits5(i, 2) else -1 for i in range(25)], np.int32)
        return 2, lut, np.array([0, 1, 2, 3, 4], np.int32)
    if name == "T3":
        lut = np.array([100 + _closed4(_digits5(i, 3)) if 4 not in _digits5(i, 3) else -1
                        for i in range(125)], np.int32)
        return 3, lut, np.array([1, 2, 3, 4, 0], np.int32)
    raise KeyError(name)


def random_ktab(rng, k, hole_p=0.3):
    lut = rng.integers(0, 50000, size=5 ** k).astype(np.int32)
    lut[rng.random(5 ** k) < hole_p] = -1
    return lut, rng.integers(0, 50000, size=5).astype(np.int32)


def test_ktab_hand_examples():
    n = 0
    for name, text, want in G.rows("kmer_table_examples.txt"):
        k, lut, base = ktab_named(name)
        ids, offs = oracle.encode_ktab(G.unescape(text), k, lut, base)
        assert ids.tolist() == G.ints(want), (name, text)
        assert offs.tolist() == [0, len(G.ints(want))]
        n += 1
    assert n >= 14


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_ktab_matches_literal_definition(k):
    rng = np.random.default_rng(300 + k)
    lut, base = random_ktab(rng, k)
    lens = [0, 1, k - 1, k, k + 1, 3 * k, 97, 400]
    data, offs = synth.markov_batch(lens, 0.4, seed=300 + k)
    ids, o = oracle.encode_ktab(data, k, lut, base, seq_offsets=offs)
    for r in range(len(lens)):
        syms = literal.kept_symbols(bytes(data[offs[r]:offs[r + 1]]))
        assert ids[o[r]:o[r + 1]].tolist() == literal.kmer_table(syms, k, lut, base)


def test_ktab_counts():
    # floor(L/k) windows, k - 1 more tokens per window without an entry, plus
    # the L mod k tail symbols
    rng = np.random.default_rng(7)
    for k in (2, 5, 6):
        lut, base = random_ktab(rng, k, hole_p=0.5)
        data = synth.iid_sequence(1000 + k, seed=k, n_fraction=0.05, lower_fraction=0.2)
        ids, _ = oracle.encode_ktab(data, k, lut, base)
        syms = literal.kept_symbols(bytes(data))
        L = len(syms)
        holes = 0
        for t in range(L // k):
            idx = 0
            for s in syms[t * k:(t + 1) * k]:
                idx = 5 * idx + (4 if s is None else s)
            holes += lut[idx] < 0
        assert len(ids) == L // k + (k - 1) * holes + L % k


@pytest.mark.parametrize("k", [1, 3, 6, 10])
def test_ktab_with_the_closed_form_table_is_the_kmer_mode(k):
    # entries = base-4 closed form for windows without N, 4^k (UNK) with N:
    # on records whose length is a multiple of k (no tail) this is DNATOK_KMER
    lut = np.empty(5 ** k, np.int32)
    for i in range(5 ** k):
        d = _digits5(i, k)
        lut[i] = (1 << (2 * k)) if 4 in d else _closed4(d)
    lens = [k * m for m in (0, 1, 2, 17, 150)]
    data, offs = synth.markov_batch(lens, 0.4, seed=k)
    a, oa = oracle.encode_ktab(data, k, lut, np.arange(5, dtype=np.int32), seq_offsets=offs)
    b, ob = oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs)
    assert a.tolist() == b.tolist() and oa.tolist() == ob.tolist()


def test_ktab_k1_identity_table_is_default_char():
    data = synth.random_bytes(3000, seed=11)
    a, oa = oracle.encode_ktab(data, 1, np.arange(5, dtype=np.int32), np.arange(5, dtype=np.int32))
    b, ob = oracle.encode(data, oracle.CHAR)
    assert a.tolist() == b.tolist() and oa.tolist() == ob.tolist()


def test_ktab_fasta_matches_records():
    rng = np.random.default_rng(5)
    lut, base = random_ktab(rng, 3)
    text = synth.fuzz_fasta(6, n_records=6, max_len=300)
    ids, offs = oracle.encode_ktab(text, 3, lut, base, fmt=oracle.FASTA)
    recs = literal.fasta_records(bytes(text))
    assert len(offs) == len(recs) + 1
    for r, body in enumerate(recs):
        assert ids[offs[r]:offs[r + 1]].tolist() == literal.kmer_table(
            literal.kept_symbols(body), 3, lut, base)


def test_ktab_decode_roundtrip():
    # an injective table whose ids differ from the base ids decodes back to
    # the kept symbols (bases upper-cased, N-class as N), whatever its holes
    rng = np.random.default_rng(9)
    for k in (1, 2, 6):
        lut = (rng.permutation(5 ** k) + 10).astype(np.int32)
        lut[rng.random(5 ** k) < 0.4] = -1
        base = np.array([0, 1, 2, 3, 4], np.int32)
        data = synth.iid_sequence(700 + k, seed=k, n_fraction=0.05, lower_fraction=0.3)
        ids, _ = oracle.encode_ktab(data, k, lut, base)
        want = bytes(b"ACGTN"[4 if s is None else s] for s in literal.kept_symbols(bytes(data)))
        assert oracle.decode_ktab(ids, k, lut, base) == want


# ------------------------------------------------------------ decode (C17)

def test_decode_lut_paper_fallback_table():
    # Algorithm 1's fixed DNA table: A1 C2 G3 T4, N and every other byte 0
    ids, _ = oracle.encode(b"ACGTNacgtn", oracle.CHAR, lut=PAPER_FALLBACK)
    assert ids.tolist() == [1, 2, 3, 4, 0, 1, 2, 3, 4, 0]
    assert oracle.decode_lut(ids, PAPER_FALLBACK) == b"ACGTNACGTN"


def test_decode_lut_default_table_is_the_char_decoder():
    data = synth.random_bytes(2000, seed=4)
    ids, _ = oracle.encode(data, oracle.CHAR)
    assert oracle.decode_lut(ids, oracle.default_lut()) == oracle.decode(ids, oracle.CHAR)


def test_decode_lut_preference_order():
    lut = np.full(256, -1, np.int32)
    lut[ord("x")] = 5
    lut[ord("Q")] = 5    # upper case before lower case
    lut[ord("b")] = 6
    lut[0x07] = 7        # only a control byte
    assert oracle.decode_lut([5, 6, 7], lut) == b"Qb\x07"
    with pytest.raises(RuntimeError):
        oracle.decode_lut([8], lut)


# ------------------------------------------------ reverse complement (C18)

def test_revcomp_hand_examples():
    n = 0
    for text, want in G.rows("revcomp_examples.txt"):
        assert oracle.revcomp(G.unescape(text)).tobytes() == G.unescape(want), text
        n += 1
    assert n >= 7


def test_revcomp_is_an_involution_and_matches_literal():
    data = synth.random_bytes(5000, seed=12)
    offs = np.array([0, 1, 10, 10, 999, 4000, 5000], np.int64)
    rc = oracle.revcomp(data, offs)
    for r in range(len(offs) - 1):
        body = bytes(data[offs[r]:offs[r + 1]])
        assert rc[offs[r]:offs[r + 1]].tobytes() == literal.reverse_complement(body)
    assert oracle.revcomp(rc, offs).tobytes() == bytes(data)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_revcomp_kmer_ids_are_reversed_and_complemented(k):
    # for ACGT records with L mod k = 0, the k-mer ids of the reverse
    # complement are the reversed list of each id's reverse complement in
    # base 4: digit i -> 3 - digit(k-1-i)
    lens = [k * m for m in (1, 5, 60)]
    data, offs = synth.markov_batch(lens, 0.4, seed=k, n_runs=False)
    ids, o = oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs)
    rids, ro = oracle.encode(oracle.revcomp(data, offs), oracle.KMER, k=k, seq_offsets=offs)
    assert o.tolist() == ro.tolist()
    for r in range(len(lens)):
        fw = ids[o[r]:o[r + 1]].tolist()
        want = []
        for v in reversed(fw):
            d = [(v >> (2 * (k - 1 - i))) & 3 for i in range(k)]
            want.append(_closed4([3 - x for x in reversed(d)]))
        assert rids[ro[r]:ro[r + 1]].tolist() == want


# -------------------------------------------------- fixed-shape feed (C19)

def test_feed_hand_examples():
    n = 0
    for tl, pad, toks, row in G.rows("feed_examples.txt"):
        t = G.ints(toks)
        out = oracle.feed(np.array(t, np.int32), [0, len(t)], int(tl), int(pad))
        assert out.shape == (1, int(tl))
        assert out[0].tolist() == G.ints(row), (tl, pad, toks)
        n += 1
    assert n >= 6


def test_feed_equal_length_rows_are_numpy_left_pad():
    # Algorithm 2's B x T case: every row has T tokens; token_len > T pads
    # each on the left
    rng = np.random.default_rng(1)
    B, T, TL = 7, 13, 20
    ids = rng.integers(0, 4097, size=B * T).astype(np.int32)
    out = oracle.feed(ids, np.arange(B + 1) * T, TL, 4098)
    want = np.pad(ids.reshape(B, T), ((0, 0), (TL - T, 0)), constant_values=4098)
    assert np.array_equal(out, want) and out.dtype == np.int64


def test_feed_row_window():
    ids = np.arange(10, dtype=np.int32)
    offs = [0, 2, 2, 7, 10]
    out = oracle.feed(ids, offs, 4, -1, row_begin=1, n_rows=2, dtype=np.int32)
    assert out.tolist() == [[-1, -1, -1, -1], [2, 3, 4, 5]]
