"""Parity of the overlapping (stride-1) k-mer path with the CPU oracle: ids
and offsets bit-identical on ragged RAW batches (with and without the
direct symbol pass), separators inside windows, FASTA text, misaligned
inputs, records shorter than k, runs of tiny and empty records (more record
starts per tile than the kernel's window holds), and the 4096-sequence
batch at full size."""
import numpy as np
import pytest

import oracle
import synth

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


def run(P, data, k, offs=None, fmt=0, pad=0, direct=True):
    import torch
    with P.Tokenizer(P.KMER_OVERLAP, k=k, fmt=fmt) as tok:
        P.binding.dnatok_set_direct(tok.h, direct)
        raw = np.zeros(len(data) + pad, dtype=np.uint8)
        raw[pad:] = data
        d = torch.from_numpy(raw).cuda()[pad:]
        so = None
        if fmt == P.RAW:
            if offs is None:
                offs = np.array([0, len(data)], dtype=np.int64)
            so = torch.from_numpy(np.asarray(offs, dtype=np.int64)).cuda()
        ids, o, tot = tok.encode(d, so)
        tok.sync()
        n_ids, n_rec = (int(x) for x in tot.cpu().tolist())
        return ids[:n_ids].cpu().numpy(), o[: n_rec + 1].cpu().numpy()


def want(data, k, offs=None, fmt=0):
    return oracle.encode(data, oracle.KMER_OVERLAP, k=k, seq_offsets=offs, fmt=fmt)


def same(got, exp, what=""):
    gi, go = got
    wi, wo = exp
    assert go.tolist() == wo.tolist(), "offsets differ " + what
    assert len(gi) == len(wi), "id counts differ %s: %d vs %d" % (what, len(gi), len(wi))
    if not np.array_equal(gi, wi):
        bad = np.nonzero(gi != wi)[0]
        raise AssertionError("ids differ %s at %d of %d" % (what, int(bad[0]), len(wi)))


def ragged(seed, n_seq, lo, hi):
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, size=n_seq)
    lens[rng.random(n_seq) < 0.1] = 0
    return synth.markov_batch(lens, 0.4, seed=seed)


@pytest.mark.parametrize("direct", [True, False])
@pytest.mark.parametrize("k", [1, 2, 3, 6, 8, 11, 15])
def test_overlap_raw_ragged(P, k, direct):
    data, offs = ragged(300 + k, 250, 0, 4000)
    same(run(P, data, k, offs, direct=direct), want(data, k, offs), "k=%d" % k)


def test_overlap_hand_examples(P):
    from tests import _golden as G
    for k, text, exp in G.rows("kmer_overlap_examples.txt"):
        d = np.frombuffer(G.unescape(text), np.uint8)
        ids, offs = run(P, d, int(k))
        assert ids.tolist() == G.ints(exp), (k, text)


@pytest.mark.parametrize("k", [3, 6])
def test_overlap_separators_and_n(P, k):
    data, offs = ragged(40 + k, 120, 0, 3000)
    rng = np.random.default_rng(k)
    parts, new_offs = [], [0]
    for r in range(len(offs) - 1):
        rec = data[offs[r]:offs[r + 1]]
        pos = np.sort(rng.choice(len(rec) + 1, size=len(rec) // 20))
        rec = np.insert(rec, pos, rng.choice(np.frombuffer(b"\n\r \tNnRY", np.uint8), size=len(pos)))
        parts.append(rec)
        new_offs.append(new_offs[-1] + len(rec))
    d2 = np.concatenate(parts)
    o2 = np.array(new_offs, dtype=np.int64)
    same(run(P, d2, k, o2), want(d2, k, o2), "k=%d" % k)


@pytest.mark.parametrize("seed", range(8))
def test_overlap_fasta(P, seed):
    text = synth.fuzz_fasta(seed, n_records=3 + seed, max_len=200 + 300 * seed)
    for k in (1, 5, 6):
        same(run(P, text, k, fmt=P.FASTA), want(text, k, fmt=oracle.FASTA), "seed %d k=%d" % (seed, k))


@pytest.mark.parametrize("pad", [1, 7, 15])
def test_overlap_misaligned(P, pad):
    data, offs = ragged(60 + pad, 80, 0, 6000)
    same(run(P, data, 6, offs, pad=pad), want(data, 6, offs), "pad %d" % pad)


def test_overlap_short_and_tiny_records(P):
    # records shorter than k, runs of empty records, and far more record
    # starts per 4096-symbol tile than the kernel keeps in its window
    rng = np.random.default_rng(17)
    lens = rng.integers(0, 9, size=6000)
    lens[2000:3000] = 0
    data, offs = synth.markov_batch(lens, 0.4, seed=17)
    for k in (2, 6, 9):
        same(run(P, data, k, offs), want(data, k, offs), "k=%d" % k)


def test_overlap_empty(P):
    e = np.zeros(0, np.uint8)
    same(run(P, e, 6, np.array([0], np.int64)), (np.zeros(0), np.array([0])))
    same(run(P, e, 6, np.array([0, 0, 0], np.int64)), (np.zeros(0), np.array([0, 0, 0])))


def test_overlap_streams_refused(P):
    import torch
    with P.Tokenizer(P.KMER_OVERLAP, k=6) as tok:
        ids = torch.empty(16, dtype=torch.int32, device="cuda")
        o = torch.empty(4, dtype=torch.int64, device="cuda")
        with pytest.raises(P.DnatokError):
            tok.stream_open(ids, o)


def test_overlap_full_kmer_batch_4096(P):
    data, offs = synth.kmer_batch_4096()
    same(run(P, data, 6, offs), want(data, 6, offs), "4096 sequences")
