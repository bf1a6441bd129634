"""Pins for the CPU oracle: each test checks it against something other than
itself -- hand-worked values from the paper's tables, closed forms, invariants,
and literal brute-force definitions on tiny inputs."""
import itertools

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
    tables = _tables(6, seed=5)
    words = [w for L in range(0, 8) for w in itertools.product(range(4), repeat=L)]
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
