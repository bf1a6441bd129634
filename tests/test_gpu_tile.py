"""Parity of the CUDA single-nucleotide / k-mer path with the CPU oracle:
ids and offsets must be bit-identical.  Sizes span several tiles with ragged
tails; edge cases cover empty and one-byte records, separators inside
k-mers, N at every phase, misaligned inputs, many boundaries in one tile,
FASTA headers across tiles, every launch shape, and the full-size
workloads."""
import numpy as np
import pytest

import oracle
import synth
from tests import _golden as G

pytestmark = pytest.mark.gpu

SHAPES = [(8192, 256, 4, 8), (16384, 256, 4, 4), (16384, 256, 3, 8), (32768, 512, 2, 4)]


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    return P


def run_gpu(P, data, mode, k=1, offs=None, fmt=0, lut=None, shape=None, pad=0, direct=None):
    """direct: try the direct path on RAW input (default: only when no launch
    shape is forced, since a shape is a setting of the general kernel)."""
    import torch
    with P.Tokenizer(mode, k=k, lut=lut, fmt=fmt) as tok:
        if shape:
            tok.set_launch(*shape)
        if direct is None:
            direct = shape is None
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


def assert_same(got, want, what=""):
    gi, go = got
    wi, wo = want
    assert go.tolist() == wo.tolist(), "offsets differ %s" % what
    if not np.array_equal(gi, wi):
        bad = np.nonzero(gi[: min(len(gi), len(wi))] != wi[: min(len(gi), len(wi))])[0]
        first = int(bad[0]) if len(bad) else min(len(gi), len(wi))
        raise AssertionError("ids differ %s: len %d vs %d, first mismatch at %d" %
                             (what, len(gi), len(wi), first))


def with_separators(data, seed, frac=0.01):
    rng = np.random.default_rng(seed)
    n = int(len(data) * frac)
    pos = np.sort(rng.choice(len(data) + 1, size=n))
    seps = rng.choice(np.frombuffer(b"\n\r \t", np.uint8), size=n)
    return np.insert(data, pos, seps)


def ragged(seed, n_seq, lo, hi, gc=0.4):
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, size=n_seq)
    lens[rng.random(n_seq) < 0.1] = 0
    return synth.markov_batch(lens, gc, seed=seed)


# --------------------------------------------------------------- worked examples

def test_worked_examples_on_gpu(P):
    fallback = np.zeros(256, dtype=np.int32)
    for c, v in zip(b"ACGTNacgtn", [1, 2, 3, 4, 0, 1, 2, 3, 4, 0]):
        fallback[c] = v
    for lut_name, text, want in G.rows("char_worked_example.txt"):
        d = np.frombuffer(G.unescape(text), np.uint8)
        ids, _ = run_gpu(P, d, P.CHAR, lut=fallback if lut_name == "paper_fallback" else None)
        assert ids.tolist() == G.ints(want)
    for k, text, want in G.rows("kmer_closed_form.txt"):
        d = np.frombuffer(G.unescape(text), np.uint8)
        ids, _ = run_gpu(P, d, P.KMER, k=int(k))
        assert ids.tolist() == G.ints(want), (k, text)
    kv = G.keyvals("fasta_records.txt")
    for sfx in ("", "2"):
        d = np.frombuffer(G.unescape(kv["text" + sfx]), np.uint8)
        ids, offs = run_gpu(P, d, P.KMER, k=2, fmt=P.FASTA)
        assert ids.tolist() == G.ints(kv["kmer2_ids" + sfx])
        assert offs.tolist() == G.ints(kv["kmer2_offsets" + sfx])
        ids, offs = run_gpu(P, d, P.CHAR, fmt=P.FASTA)
        assert ids.tolist() == G.ints(kv["char_ids" + sfx])
        assert offs.tolist() == G.ints(kv["char_offsets" + sfx])


# -------------------------------------------------------------------- RAW input

@pytest.mark.parametrize("direct", [True, False])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8, 11, 14, 15])
def test_kmer_raw_ragged(P, k, direct):
    data, offs = ragged(100 + k, 300, 0, 3000)
    assert_same(run_gpu(P, data, P.KMER, k=k, offs=offs, direct=direct),
                oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs), "k=%d" % k)


@pytest.mark.parametrize("shape", SHAPES)
def test_kmer_raw_every_shape(P, shape):
    data, offs = ragged(7, 200, 0, 40000)
    for k in (1, 6):
        assert_same(run_gpu(P, data, P.KMER, k=k, offs=offs, shape=shape),
                    oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs), str(shape))
    assert_same(run_gpu(P, data, P.CHAR, offs=offs, shape=shape),
                oracle.encode(data, oracle.CHAR, seq_offsets=offs), str(shape))


@pytest.mark.parametrize("direct", [True, False])
@pytest.mark.parametrize("pad", [1, 3, 7, 8, 15])
def test_misaligned_input(P, pad, direct):
    data, offs = ragged(50 + pad, 60, 0, 5000)
    for mode, k in ((P.CHAR, 1), (P.KMER, 6), (P.KMER, 5)):
        assert_same(run_gpu(P, data, mode, k=k, offs=offs, pad=pad, direct=direct),
                    oracle.encode(data, mode, k=k, seq_offsets=offs), "pad %d" % pad)


@pytest.mark.parametrize("k", [1, 3, 6, 13])
def test_separators_inside_kmers(P, k):
    data, offs = ragged(200 + k, 150, 0, 4000)
    # separators inserted per record keep the record layout valid
    parts, new_offs = [], [0]
    for r in range(len(offs) - 1):
        rec = with_separators(data[offs[r]:offs[r + 1]], seed=r, frac=0.05)
        parts.append(rec)
        new_offs.append(new_offs[-1] + len(rec))
    d2 = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    o2 = np.array(new_offs, dtype=np.int64)
    for mode in (P.KMER, P.CHAR):
        kk = k if mode == P.KMER else 1
        assert_same(run_gpu(P, d2, mode, k=kk, offs=o2),
                    oracle.encode(d2, mode, k=kk, seq_offsets=o2), "k=%d" % kk)


def test_n_at_every_phase(P):
    k = 6
    base = synth.iid_sequence(6 * 50, seed=3, n_fraction=0.0)
    recs = []
    for ph in range(k):
        r = base.copy()
        r[ph::k * 7] = ord("N")
        recs.append(r)
    data = np.concatenate(recs)
    offs = np.cumsum([0] + [len(r) for r in recs]).astype(np.int64)
    assert_same(run_gpu(P, data, P.KMER, k=k, offs=offs),
                oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs))


def test_random_bytes_all_classes(P):
    data = synth.random_bytes(200_000, seed=11)
    offs = np.array([0, 1, 2, 50_000, 50_001, 199_999, 200_000], dtype=np.int64)
    for mode, k in ((P.CHAR, 1), (P.KMER, 1), (P.KMER, 4), (P.KMER, 15)):
        assert_same(run_gpu(P, data, mode, k=k, offs=offs),
                    oracle.encode(data, mode, k=k, seq_offsets=offs))


def test_user_lut(P):
    rng = np.random.default_rng(5)
    lut = rng.integers(-1, 1000, size=256).astype(np.int32)
    data = synth.random_bytes(70_000, seed=12)
    offs = np.array([0, 30_000, 70_000], dtype=np.int64)
    assert_same(run_gpu(P, data, P.CHAR, lut=lut, offs=offs),
                oracle.encode(data, oracle.CHAR, lut=lut, seq_offsets=offs))


def test_many_boundaries_in_one_tile(P):
    # 5000 records in 20 kB, many of them empty, plus a run of empties at one position
    rng = np.random.default_rng(9)
    lens = rng.integers(0, 9, size=5000)
    lens[1000:2500] = 0
    data, offs = synth.markov_batch(lens, 0.4, seed=9)
    for mode, k in ((P.KMER, 3), (P.KMER, 6), (P.CHAR, 1)):
        for shape in (SHAPES[0], SHAPES[3], None):
            assert_same(run_gpu(P, data, mode, k=k, offs=offs, shape=shape),
                        oracle.encode(data, mode, k=k, seq_offsets=offs))


@pytest.mark.parametrize("k", [2, 6, 15])
def test_direct_record_density(P, k):
    # the direct path with 1-600 byte records: steps holding from zero to
    # dozens of record starts, runs of empty records, records ending inside a
    # k-mer's 16-byte window
    rng = np.random.default_rng(40 + k)
    for hi in (8, 40, 600):
        lens = rng.integers(0, hi + 1, size=3000)
        lens[rng.random(3000) < 0.05] = 0
        data, offs = synth.markov_batch(lens, 0.4, seed=int(hi))
        for pad in (0, 5):
            assert_same(run_gpu(P, data, P.KMER, k=k, offs=offs, pad=pad, direct=True),
                        oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs),
                        "k=%d hi=%d pad=%d" % (k, hi, pad))


def test_empty_inputs(P):
    e = np.zeros(0, np.uint8)
    for mode, k in ((P.CHAR, 1), (P.KMER, 6)):
        assert_same(run_gpu(P, e, mode, k=k, offs=np.array([0], np.int64)), (np.zeros(0), np.array([0])))
        assert_same(run_gpu(P, e, mode, k=k, offs=np.array([0, 0, 0], np.int64)),
                    (np.zeros(0), np.array([0, 0, 0])))
        assert_same(run_gpu(P, e, mode, k=k, fmt=P.FASTA), (np.zeros(0), np.array([0])))


def test_one_long_record_many_tiles(P):
    data = synth.iid_sequence(3_000_000, seed=21, n_fraction=0.01, lower_fraction=0.05)
    data = with_separators(data, seed=22, frac=0.001)
    offs = np.array([0, len(data)], dtype=np.int64)
    for k in (1, 6, 7):
        assert_same(run_gpu(P, data, P.KMER, k=k, offs=offs),
                    oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs), "k=%d" % k)


# ------------------------------------------------------------------------ FASTA

@pytest.mark.parametrize("seed", range(25))
def test_fasta_fuzz(P, seed):
    text = synth.fuzz_fasta(seed, n_records=int(3 + seed % 7), max_len=int(50 + 400 * (seed % 5)))
    for mode, k in ((P.CHAR, 1), (P.KMER, 3), (P.KMER, 6)):
        assert_same(run_gpu(P, text, mode, k=k, fmt=P.FASTA),
                    oracle.encode(text, mode, k=k, fmt=oracle.FASTA), "seed %d" % seed)


def test_fasta_large_with_long_lines(P):
    text, _ = synth.fasta_stream(4_000_000, seed=31, rec_lo=100, rec_hi=300_000)
    for k in (1, 6):
        for shape in (SHAPES[0], SHAPES[2]):
            assert_same(run_gpu(P, text, P.KMER, k=k, fmt=P.FASTA, shape=shape),
                        oracle.encode(text, oracle.KMER, k=k, fmt=oracle.FASTA))


def test_fasta_headers_only_and_long_header(P):
    text = np.frombuffer(b">" + b"x" * 100_000 + b"\nACGTACGTAC\n>\n>\nGG" + b"\n" * 40_000 + b"T",
                         np.uint8)
    for mode, k in ((P.CHAR, 1), (P.KMER, 3)):
        assert_same(run_gpu(P, text, mode, k=k, fmt=P.FASTA),
                    oracle.encode(text, mode, k=k, fmt=oracle.FASTA))


# ----------------------------------------------------------------------- errors

def test_bad_seq_offsets_reported(P):
    import torch
    with P.Tokenizer(P.KMER, k=6) as tok:
        d = torch.zeros(1000, dtype=torch.uint8, device="cuda")
        so = torch.tensor([0, 600, 500, 1000], dtype=torch.int64, device="cuda")
        tok.encode(d, so)
        with pytest.raises(P.DnatokError) as e:
            tok.sync()
        assert e.value.status == -10
        # the error is cleared: the handle works again
        ids, offs = tok.encode_host(np.frombuffer(b"ACGTAC", np.uint8))
        assert ids.tolist() == [433]


def test_capacity_checked_on_host(P):
    import torch
    with P.Tokenizer(P.CHAR) as tok:
        d = torch.zeros(100, dtype=torch.uint8, device="cuda")
        so = torch.tensor([0, 100], dtype=torch.int64, device="cuda")
        ids = torch.empty(99, dtype=torch.int32, device="cuda")
        offs = torch.empty(2, dtype=torch.int64, device="cuda")
        tot = torch.empty(2, dtype=torch.int64, device="cuda")
        with pytest.raises(P.DnatokError) as e:
            tok.encode(d, so, ids, offs, tot)
        assert e.value.status == -3


def test_bad_tables_rejected(P):
    with pytest.raises(P.DnatokError):
        P.Tokenizer(P.KMER, k=16)
    lut = np.zeros(256, dtype=np.int32)
    lut[5] = -2
    with pytest.raises(P.DnatokError):
        P.Tokenizer(P.CHAR, lut=lut)


# ------------------------------------------------------------ full-size workloads

@pytest.mark.parametrize("direct", [True, False])
def test_full_single_sequence_1mb(P, direct):
    data, offs = synth.single_sequence_1mb()
    assert_same(run_gpu(P, data, P.CHAR, offs=offs, direct=direct),
                oracle.encode(data, oracle.CHAR, seq_offsets=offs))


@pytest.mark.parametrize("direct", [True, False])
def test_full_kmer_batch_4096(P, direct):
    data, offs = synth.kmer_batch_4096()
    assert_same(run_gpu(P, data, P.KMER, k=6, offs=offs, direct=direct),
                oracle.encode(data, oracle.KMER, k=6, seq_offsets=offs))
