"""Parity of the compacted FASTA k-mer path with the CPU oracle: FASTA text of
64 KiB or more (16-byte aligned, k >= 2) is compacted on the device to its
sequence bytes and record starts and then tokenized by the direct k-mer
kernels.  Ids and offsets must be bit-identical to the oracle's and to the
general kernel's (the direct path switched off).  Cases: wrapped records with
N runs and soft-masking, concatenated fuzz text (CRLF, blank lines, '>'
inside sequence lines, IUPAC letters, sequence before the first header,
blanks and tabs), long headers across vectors and tiles, a header or a
record cut at the end, records without bases, more records than the direct
plan takes and too few id offsets (both hand the encode to the general
kernel), control bytes the direct kernel declines, misaligned input, and
graph replay."""
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


def run(P, text, k, direct=True, pad=0, offsets_capacity=None):
    import torch
    with P.Tokenizer(P.KMER, k=k, fmt=P.FASTA) as tok:
        P.binding.dnatok_set_direct(tok.h, direct)
        raw = np.zeros(len(text) + pad + 16, dtype=np.uint8)
        raw[pad:pad + len(text)] = text
        d = torch.from_numpy(raw).cuda()[pad:pad + len(text)]
        ids, o, tot = tok.alloc_outputs(len(text), 0, offsets_capacity=offsets_capacity)
        ids.fill_(-7)
        o.fill_(-7)
        tok.encode(d, None, ids, o, tot)
        tok.sync()
        run.path = P.binding.dnatok_direct_ran(tok.h)
        n_ids, n_rec = (int(x) for x in tot.cpu().tolist())
        return ids[:n_ids].cpu().numpy(), o[: n_rec + 1].cpu().numpy()


def check(P, text, ks=(2, 3, 6, 15), what="", direct_path=1):
    """direct_path: what dnatok_direct_ran must say for the direct-on run
    (1 = the compacted path produced everything, 0 = it declined, None =
    either)."""
    for k in ks:
        want = oracle.encode(text, oracle.KMER, k=k, fmt=oracle.FASTA)
        for direct in (True, False):
            gi, go = run(P, text, k, direct=direct)
            if direct_path is not None or not direct:
                assert run.path == (direct_path if direct else -1), (k, direct, run.path, what)
            assert go.tolist() == want[1].tolist(), "offsets differ k=%d direct=%s %s" % (k, direct, what)
            if not np.array_equal(gi, want[0]):
                m = min(len(gi), len(want[0]))
                bad = np.nonzero(gi[:m] != want[0][:m])[0]
                raise AssertionError("ids differ k=%d direct=%s %s: len %d vs %d, first at %s" %
                                     (k, direct, what, len(gi), len(want[0]),
                                      int(bad[0]) if len(bad) else m))


def fuzz_concat(seed, n_bytes):
    parts, total, s = [], 0, seed * 1000
    while total < n_bytes:
        t = synth.fuzz_fasta(s, n_records=8, max_len=2000, crlf_p=0.3, blank_p=0.1)
        s += 1
        parts.append(t)
        total += len(t)
    return np.concatenate(parts)


def test_wrapped_records(P):
    text, _ = synth.fasta_stream(3_000_000, seed=61, rec_lo=100, rec_hi=400_000)
    check(P, text, what="wrapped records")


@pytest.mark.parametrize("seed", range(6))
def test_fuzz_concatenated(P, seed):
    text = fuzz_concat(seed, 70_000 + 90_000 * seed)
    check(P, text, ks=(2, 5, 6, 13), what="seed %d" % seed)


def test_blanks_tabs_and_leading_sequence(P):
    rng = np.random.default_rng(5)
    seq = rng.choice(np.frombuffer(b"ACGTNacgtn", np.uint8), size=200_000)
    seps = rng.choice(np.frombuffer(b" \t\r", np.uint8), size=3000)
    pos = np.sort(rng.choice(len(seq), size=3000))
    body = np.insert(seq, pos, seps)
    lines = [bytes(body[i:i + 70]) + b"\n" for i in range(0, len(body), 70)]
    text = b"ACGTA CG\tT\r\n" + b"".join(lines[:1000]) + b">r1 x\n" + b"".join(lines[1000:]) + b">last"
    check(P, np.frombuffer(text, np.uint8), what="blanks")


def test_long_headers_across_tiles(P):
    rng = np.random.default_rng(7)
    parts = []
    for i in range(12):
        parts.append(b">" + bytes(rng.integers(32, 127, size=int(rng.integers(1, 40_000))).astype(np.uint8)) + b"\n")
        parts.append(bytes(rng.choice(np.frombuffer(b"ACGT", np.uint8), size=int(rng.integers(0, 30_000)))) + b"\n")
    text = np.frombuffer(b"".join(parts), np.uint8)
    check(P, text, what="long headers")
    # the same text cut inside a header and inside a sequence line
    for cut in (len(text) - 5, len(text) // 2 + 3):
        check(P, text[:cut], ks=(3, 6), what="cut at %d" % cut)


def test_records_without_bases_and_header_at_end(P):
    body = b"".join(b">h%d\n" % i + (b"ACGTTGCA" * 40 * (i % 5)) + b"\n" for i in range(5_000))
    check(P, np.frombuffer(body + b">tail-header-no-newline", np.uint8), ks=(2, 6))
    check(P, np.frombuffer(b"\n\n" + body, np.uint8), ks=(4,))  # an empty first record
    # records of 16 bases on average: denser than the direct kernel's record
    # window, which hands such slots to the general kernel
    dense = b"".join(b">h%d\n" % i + (b"ACGTTGCA" * (i % 5)) + b"\n" for i in range(20_000))
    check(P, np.frombuffer(dense, np.uint8), ks=(2, 6), direct_path=None)


def test_more_records_than_the_plan_takes(P):
    # 70,000 records: the scan hands the encode to the general kernel
    text = np.frombuffer(b"".join(b">\nAC%s\n" % (b"G" * (i % 3)) for i in range(70_000)), np.uint8)
    check(P, text, ks=(2, 3), what="70000 records", direct_path=0)


def test_too_few_id_offsets(P):
    """The records found exceed the id offsets' capacity: the entries past it
    are not written, the ids and the totals are complete (the scan hands
    the encode to the general kernel)."""
    text = np.frombuffer(b"".join(b">r\n" + b"ACGT" * 50 + b"\n" for _ in range(1000)), np.uint8)
    want = oracle.encode(text, oracle.KMER, k=6, fmt=oracle.FASTA)
    for direct in (True, False):
        gi, go = run(P, text, 6, direct=direct, offsets_capacity=500)
        assert run.path == (0 if direct else -1)
        assert len(go) == 500 and go.tolist() == want[1][:500].tolist()
        assert np.array_equal(gi, want[0])


def test_control_bytes_fall_back(P):
    text, _ = synth.fasta_stream(400_000, seed=8, rec_lo=1000, rec_hi=50_000)
    text = text.copy()
    rng = np.random.default_rng(8)
    pos = rng.choice(len(text), size=20)
    text[pos] = np.where(text[pos] == ord("\n"), text[pos], 0x0B)  # vertical tabs in sequence lines
    check(P, text, ks=(3, 6), what="control bytes", direct_path=0)


@pytest.mark.parametrize("pad", [1, 8])
def test_misaligned_input(P, pad):
    text, _ = synth.fasta_stream(300_000, seed=9 + pad, rec_lo=500, rec_hi=80_000)
    want = oracle.encode(text, oracle.KMER, k=6, fmt=oracle.FASTA)
    gi, go = run(P, text, 6, pad=pad)
    assert run.path == -1  # the compacted path wants 16-byte aligned text
    assert go.tolist() == want[1].tolist() and np.array_equal(gi, want[0])


def test_graph_replay(P):
    """Captured once, replayed over two texts of the same size, the second one
    with more records than the direct plan takes (the replay's general
    kernel runs and clears the switch for the next replay)."""
    import torch
    n = 300_000
    a, _ = synth.fasta_stream(n, seed=12, rec_lo=500, rec_hi=60_000)
    many = b"".join(b">\nA\n" for _ in range(n // 4 + 1))[:n]  # 75,000 records
    b = np.frombuffer(many, np.uint8)
    k = 6
    with P.Tokenizer(P.KMER, k=k, fmt=P.FASTA) as tok:
        tok.reserve(n, 1)
        d = torch.from_numpy(a.copy()).cuda()
        ids, o, tot = tok.alloc_outputs(n, 0)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            tok.encode(d, None, ids, o, tot, stream=s)  # warm-up outside the graph
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            tok.encode(d, None, ids, o, tot, stream=s)
        for text in (a, b, a):
            d.copy_(torch.from_numpy(text.copy()))
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            want = oracle.encode(text, oracle.KMER, k=k, fmt=oracle.FASTA)
            n_ids, n_rec = (int(x) for x in tot.cpu().tolist())
            assert o[: n_rec + 1].cpu().numpy().tolist() == want[1].tolist()
            assert np.array_equal(ids[:n_ids].cpu().numpy(), want[0])


def test_small_text_and_raw_paths(P):
    """Below 64 KiB FASTA text goes straight to the general kernel; a RAW
    encode reports its own direct path."""
    import torch
    text = synth.fuzz_fasta(3, n_records=5, max_len=300)
    check(P, text, ks=(6,), direct_path=-1)
    data, offs = synth.markov_batch([5000, 0, 70000], 0.4, seed=2)
    with P.Tokenizer(P.KMER, k=6) as tok:
        ids, o, tot = tok.encode(torch.from_numpy(data).cuda(), torch.from_numpy(offs).cuda())
        assert P.binding.dnatok_direct_ran(tok.h) == 1
        want = oracle.encode(data, oracle.KMER, k=6, seq_offsets=offs)
        assert np.array_equal(ids[: len(want[0])].cpu().numpy(), want[0])
        sep = data.copy()
        sep[100] = ord(" ")
        tok.encode(torch.from_numpy(sep).cuda(), torch.from_numpy(offs).cuda(), ids, o, tot)
        assert P.binding.dnatok_direct_ran(tok.h) == 0
