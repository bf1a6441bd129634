"""Parity of the GPU decode (ids -> text through inverse tables) with the
oracle's decoders, record by record: every mode (single-nucleotide with the
default and the paper's fallback table, k-mers, overlapping k-mers, BPE,
table-driven k-mers), ids with no inverse counted and skipped, empty
records, and the 4096-sequence 6-mer batch at full size.  The ids come from
the oracle's encoder, so the decode is checked on its own."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import PAPER_FALLBACK, random_ktab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    return P


def gpu_decode(tok, ids, offs):
    import torch
    ti = torch.from_numpy(np.ascontiguousarray(ids, dtype=np.int32)).cuda()
    to = torch.from_numpy(np.ascontiguousarray(offs, dtype=np.int64)).cuda()
    out, bo, tot = tok.decode(ti, to)
    tok.sync()
    n, bad = (int(x) for x in tot.cpu().tolist())
    return out[:n].cpu().numpy().tobytes(), bo.cpu().numpy(), bad


def check(tok, ids, offs, dec_one):
    got, bo, bad = gpu_decode(tok, ids, offs)
    assert bad == 0
    pos = 0
    for r in range(len(offs) - 1):
        want = dec_one(ids[offs[r]:offs[r + 1]])
        assert bo[r] == pos, "record %d offset" % r
        assert got[pos:pos + len(want)] == want, "record %d text" % r
        pos += len(want)
    assert bo[-1] == pos == len(got)


def batch(seed, n_seq=150, hi=3000, n_runs=True):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, hi, size=n_seq)
    lens[rng.random(n_seq) < 0.1] = 0
    return synth.markov_batch(lens, 0.4, seed=seed, n_runs=n_runs)


def test_decode_char_default_and_paper_table(P):
    data, offs = batch(1)
    for lut in (None, PAPER_FALLBACK):
        ids, o = oracle.encode(data, oracle.CHAR, seq_offsets=offs, lut=lut)
        table = oracle.default_lut() if lut is None else lut
        with P.Tokenizer(P.CHAR, lut=lut) as tok:
            check(tok, ids, o, lambda x: oracle.decode_lut(x, table))


@pytest.mark.parametrize("k", [1, 2, 6, 11, 15])
def test_decode_kmer(P, k):
    data, offs = batch(10 + k)
    ids, o = oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs)
    with P.Tokenizer(P.KMER, k=k) as tok:
        check(tok, ids, o, lambda x: oracle.decode(x, oracle.KMER, k=k))


@pytest.mark.parametrize("k", [1, 3, 6, 15])
def test_decode_kmer_overlap(P, k):
    data, offs = batch(20 + k)
    ids, o = oracle.encode(data, oracle.KMER_OVERLAP, k=k, seq_offsets=offs)
    with P.Tokenizer(P.KMER_OVERLAP, k=k) as tok:
        check(tok, ids, o, lambda x: oracle.decode(x, oracle.KMER_OVERLAP, k=k))


def test_decode_bpe(P):
    corpus = synth.bpe_training_corpus(seed=5, n=30000)
    merges = oracle.bpe_train(oracle.codes_of(bytes(corpus)), 300)
    data, offs = batch(30)
    ids, o = oracle.encode(data, oracle.BPE, seq_offsets=offs, merges=merges)
    with P.Tokenizer(P.BPE, merges=merges) as tok:
        check(tok, ids, o, lambda x: oracle.decode(x, oracle.BPE, merges=merges))


@pytest.mark.parametrize("k", [1, 3, 6, 10])
def test_decode_kmer_table(P, k):
    rng = np.random.default_rng(k)
    lut, base = random_ktab(rng, k, hole_p=0.3)
    data, offs = batch(40 + k)
    ids, o = oracle.encode_ktab(data, k, lut, base, seq_offsets=offs)
    with P.Tokenizer(P.KMER_TABLE, k=k, kmer_lut=lut, base_ids=base) as tok:
        check(tok, ids, o, lambda x: oracle.decode_ktab(x, k, lut, base))


def test_decode_ids_without_text(P):
    # PAD and out-of-range ids write nothing and are counted
    k = 4
    data, offs = batch(50, n_seq=20, hi=400)
    ids, o = oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs)
    rng = np.random.default_rng(0)
    bad_ids = np.array([(1 << 2 * k) + 1, -3, 1 << 30], np.int32)
    ins = np.sort(rng.choice(len(ids) + 1, size=9))
    ids2 = np.insert(ids, ins, np.resize(bad_ids, 9))
    o2 = o + np.searchsorted(ins, o, side="left")  # (offsets after the insertions)
    o2[-1] = len(ids2)
    with P.Tokenizer(P.KMER, k=k) as tok:
        got, _, bad = gpu_decode(tok, ids2, o2)
    assert bad == 9
    assert got == oracle.decode(ids, oracle.KMER, k=k)


def test_decode_empty(P):
    with P.Tokenizer(P.KMER, k=3) as tok:
        got, bo, bad = gpu_decode(tok, np.zeros(0, np.int32), np.zeros(4, np.int64))
        assert got == b"" and bo.tolist() == [0, 0, 0, 0] and bad == 0


def test_decode_capacity_checked(P):
    import torch
    with P.Tokenizer(P.KMER, k=6) as tok:
        ids = torch.zeros(10, dtype=torch.int32, device="cuda")
        offs = torch.tensor([0, 10], dtype=torch.int64, device="cuda")
        out = torch.empty(59, dtype=torch.uint8, device="cuda")
        with pytest.raises(P.DnatokError):
            tok.decode(ids, offs, out=out)


def test_decode_full_kmer_batch_4096(P):
    data, offs = synth.kmer_batch_4096()
    ids, o = oracle.encode(data, oracle.KMER, k=6, seq_offsets=offs)
    with P.Tokenizer(P.KMER, k=6) as tok:
        got, bo, bad = gpu_decode(tok, ids, o)
    assert bad == 0
    want = b"".join(oracle.decode(ids[o[r]:o[r + 1]], oracle.KMER, k=6) for r in range(len(o) - 1))
    assert got == want
    lens = [len(oracle.decode(ids[o[r]:o[r + 1]], oracle.KMER, k=6)) for r in (0, 1, 4095)]
    assert bo[1] - bo[0] == lens[0] and bo[2] - bo[1] == lens[1] and bo[4096] - bo[4095] == lens[2]
