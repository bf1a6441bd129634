"""Parity of the table-driven k-mer path (5^k table with single-symbol
fallback) with the CPU oracle: ids and offsets bit-identical on the
hand-worked fixture, random tables for every k in 1..10 on ragged RAW
batches, separators and IUPAC bytes inside windows, FASTA text, misaligned
inputs, runs of tiny and empty records (more record starts per tile than the
kernel's window holds), graph replays, a FASTA offsets array too small for
its records, and the 4096-sequence batch at full size with a vocabulary laid
out like a blocked 6-mer model's."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import ktab_named, random_ktab

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


def run(P, data, k, lut, base, offs=None, fmt=0, pad=0, direct=True):
    import torch
    with P.Tokenizer(P.KMER_TABLE, k=k, fmt=fmt, kmer_lut=lut, base_ids=base) as tok:
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


def want(data, k, lut, base, offs=None, fmt=0):
    return oracle.encode_ktab(data, k, lut, base, seq_offsets=offs, fmt=fmt)


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


def test_ktab_hand_examples(P):
    from tests import _golden as G
    for name, text, exp in G.rows("kmer_table_examples.txt"):
        k, lut, base = ktab_named(name)
        d = np.frombuffer(G.unescape(text), np.uint8)
        ids, offs = run(P, d, k, lut, base)
        assert ids.tolist() == G.ints(exp), (name, text)
        assert offs.tolist() == [0, len(G.ints(exp))]


@pytest.mark.parametrize("direct", [True, False])
@pytest.mark.parametrize("k", list(range(1, 11)))
def test_ktab_raw_ragged(P, k, direct):
    rng = np.random.default_rng(500 + k)
    lut, base = random_ktab(rng, k, hole_p=0.3)
    data, offs = ragged(500 + k, 200, 0, 4000)
    same(run(P, data, k, lut, base, offs, direct=direct), want(data, k, lut, base, offs), "k=%d" % k)


@pytest.mark.parametrize("hole_p", [0.0, 1.0])
def test_ktab_all_or_no_entries(P, hole_p):
    rng = np.random.default_rng(3)
    lut, base = random_ktab(rng, 5, hole_p=hole_p)
    data, offs = ragged(7, 150, 0, 3000)
    same(run(P, data, 5, lut, base, offs), want(data, 5, lut, base, offs), "holes %g" % hole_p)


@pytest.mark.parametrize("k", [3, 6])
def test_ktab_separators_and_iupac(P, k):
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
    lut, base = random_ktab(rng, k)
    same(run(P, d2, k, lut, base, o2), want(d2, k, lut, base, o2), "k=%d" % k)


@pytest.mark.parametrize("seed", range(6))
def test_ktab_fasta(P, seed):
    text = synth.fuzz_fasta(seed, n_records=3 + seed, max_len=200 + 300 * seed)
    rng = np.random.default_rng(seed)
    for k in (1, 4, 6):
        lut, base = random_ktab(rng, k)
        same(run(P, text, k, lut, base, fmt=P.FASTA),
             want(text, k, lut, base, fmt=oracle.FASTA), "seed %d k=%d" % (seed, k))


@pytest.mark.parametrize("pad", [1, 7, 15])
def test_ktab_misaligned(P, pad):
    lut, base = synth.kmer_vocab(6, seed=pad)
    data, offs = ragged(60 + pad, 80, 0, 6000)
    same(run(P, data, 6, lut, base, offs, pad=pad), want(data, 6, lut, base, offs), "pad %d" % pad)


def test_ktab_short_and_tiny_records(P):
    rng = np.random.default_rng(17)
    lens = rng.integers(0, 9, size=6000)
    lens[2000:3000] = 0
    data, offs = synth.markov_batch(lens, 0.4, seed=17)
    for k in (2, 6, 9):
        lut, base = random_ktab(rng, k)
        same(run(P, data, k, lut, base, offs), want(data, k, lut, base, offs), "k=%d" % k)


def test_ktab_empty(P):
    lut, base = random_ktab(np.random.default_rng(1), 3)
    e = np.zeros(0, np.uint8)
    same(run(P, e, 3, lut, base, np.array([0], np.int64)), (np.zeros(0), np.array([0])))
    same(run(P, e, 3, lut, base, np.array([0, 0, 0], np.int64)), (np.zeros(0), np.array([0, 0, 0])))


def test_ktab_bad_tables_refused(P):
    lut, base = random_ktab(np.random.default_rng(1), 2)
    bad = lut.copy()
    bad[3] = -2
    with pytest.raises(P.DnatokError):
        P.Tokenizer(P.KMER_TABLE, k=2, kmer_lut=bad, base_ids=base)
    with pytest.raises(P.DnatokError):
        P.Tokenizer(P.KMER_TABLE, k=2, kmer_lut=lut, base_ids=np.array([0, 1, 2, 3, -1]))
    with pytest.raises(P.DnatokError):
        P.Tokenizer(P.KMER_TABLE, k=11, kmer_lut=np.zeros(5 ** 11, np.int32), base_ids=base)
    with pytest.raises(P.DnatokError):
        P.Tokenizer(P.KMER_TABLE, k=2)


def test_ktab_streams_refused(P):
    import torch
    lut, base = random_ktab(np.random.default_rng(1), 2)
    with P.Tokenizer(P.KMER_TABLE, k=2, kmer_lut=lut, base_ids=base) as tok:
        ids = torch.empty(16, dtype=torch.int32, device="cuda")
        o = torch.empty(4, dtype=torch.int64, device="cuda")
        with pytest.raises(P.DnatokError):
            tok.stream_open(ids, o)


@pytest.mark.parametrize("mode", ["overlap", "table"])
def test_fasta_offsets_too_small(P, mode):
    # more FASTA records than id_offsets holds: the encode reports a capacity
    # error and writes nothing outside the arrays
    import torch
    text = synth.fuzz_fasta(3, n_records=12, max_len=300)
    lut, base = random_ktab(np.random.default_rng(2), 3)
    if mode == "overlap":
        tok = P.Tokenizer(P.KMER_OVERLAP, k=3, fmt=P.FASTA)
    else:
        tok = P.Tokenizer(P.KMER_TABLE, k=3, fmt=P.FASTA, kmer_lut=lut, base_ids=base)
    with tok:
        d = torch.from_numpy(np.ascontiguousarray(text)).cuda()
        ids = torch.full((len(text) + 64,), -7, dtype=torch.int32, device="cuda")
        offs = torch.full((16,), -7, dtype=torch.int64, device="cuda")
        tot = torch.zeros(2, dtype=torch.int64, device="cuda")
        P.binding.dnatok_encode(tok.h, d.data_ptr(), len(text), 0, 0, ids.data_ptr(), len(text),
                                offs.data_ptr(), 4, tot.data_ptr(), P._stream_ptr(None))
        with pytest.raises(P.DnatokError):
            tok.sync()
        assert (offs[4:] == -7).all() and (ids[len(text):] == -7).all()
        # the handle works again after the error was reported
        _, want_offs = oracle.encode_ktab(text, 3, lut, base, fmt=oracle.FASTA)
        i2, o2, t2 = tok.encode(d)
        tok.sync()
        assert int(t2[1]) == len(want_offs) - 1


def test_ktab_graph_replay(P):
    import torch
    lut, base = synth.kmer_vocab(6, seed=3)
    data, offs = ragged(21, 300, 0, 5000)
    exp = want(data, 6, lut, base, offs)
    with P.Tokenizer(P.KMER_TABLE, k=6, kmer_lut=lut, base_ids=base) as tok:
        tok.reserve(len(data), len(offs) - 1)
        d = torch.from_numpy(data).cuda()
        so = torch.from_numpy(offs).cuda()
        ids, o, tot = tok.alloc_outputs(len(data), len(offs) - 1)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            P.binding.dnatok_graph_begin(tok.h, s.cuda_stream)
            tok.encode(d, so, ids, o, tot, stream=s)
            g = P.binding.dnatok_graph_end(tok.h, s.cuda_stream)
        for _ in range(2):
            ids.fill_(-1)
            P.binding.dnatok_graph_launch(g, s.cuda_stream)
            s.synchronize()
            n = int(tot[0])
            same((ids[:n].cpu().numpy(), o.cpu().numpy()), exp, "replay")
        P.binding.dnatok_graph_destroy(g)


def test_ktab_full_kmer_batch_4096(P):
    lut, base = synth.kmer_vocab(6, seed=49)
    data, offs = synth.kmer_batch_4096()
    same(run(P, data, 6, lut, base, offs), want(data, 6, lut, base, offs), "4096 sequences")


@pytest.mark.parametrize("k", [2, 6])
def test_ktab_wide_ids_global_table(P, k):
    # ids that do not fit 16 bits keep the table in global memory
    rng = np.random.default_rng(70 + k)
    lut = rng.integers(0, 1 << 30, size=5 ** k).astype(np.int32)
    lut[rng.random(5 ** k) < 0.2] = -1
    base = rng.integers(0, 1 << 30, size=5).astype(np.int32)
    data, offs = ragged(80 + k, 150, 0, 5000)
    same(run(P, data, k, lut, base, offs), want(data, k, lut, base, offs), "k=%d" % k)


def test_ktab_u16_boundary_ids(P):
    # 0xFFFE is the largest id the shared-memory table holds; one id of
    # 0xFFFF moves the table to global memory; both give the same ids
    rng = np.random.default_rng(5)
    data, offs = ragged(90, 100, 0, 4000)
    for top in (0xFFFE, 0xFFFF):
        lut = rng.integers(0, 1000, size=5 ** 3).astype(np.int32)
        lut[7] = top
        lut[rng.random(5 ** 3) < 0.3] = -1
        lut[8] = top
        base = np.array([0, 1, 2, 3, 4], np.int32)
        same(run(P, data, 3, lut, base, offs), want(data, 3, lut, base, offs), "top %d" % top)
