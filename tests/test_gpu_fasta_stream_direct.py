"""The host-streamed FASTA encode through the compacted path: chunks of 64 KiB
and more (k >= 2) are compacted on the device and tokenized by the direct
k-mer kernels, continuing the record left open by the chunk before from the
general kernel's carry (its symbols, ids, boundaries and line state), while
smaller chunks, and chunks the compacted path declines, take the general
kernel.  Ids and offsets must equal the oracle's on the whole text whatever
the chunking: seams inside headers, between CR and LF, right before a '>',
inside records shorter than k, whole chunks of header, chunks without a
base, control bytes in one chunk, and the direct path switched off."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

C = 65536  # the smallest chunk the compacted path takes


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    return torch, P


def stream(torch, P, text, k, chunk, pieces=None, direct=True):
    """Encode `text` through the stream API (chunk bytes per chunk, the text
    submitted in `pieces`, pinned) and return (ids, offsets)."""
    n = len(text)
    with P.Tokenizer(P.KMER, k=k, fmt=P.FASTA) as tok:
        P.binding.dnatok_set_direct(tok.h, direct)
        ids = torch.full((n + 16,), -9, dtype=torch.int32, device="cuda")
        offs = torch.full((n // 2 + 16,), -9, dtype=torch.int64, device="cuda")
        tok.stream_open(ids, offs, chunk_bytes=chunk, n_slots=3, overlap=True)
        host = torch.from_numpy(np.array(text, dtype=np.uint8)).pin_memory()
        cuts = [0, n] if pieces is None else pieces
        reqs = []
        for i in range(len(cuts) - 1):
            fl = P.HOST_PINNED | (P.END_OF_STREAM if i == len(cuts) - 2 else 0)
            reqs.append(tok.stream_submit(host[cuts[i]:cuts[i + 1]], fl))
        n_ids, n_rec, _ = tok.stream_wait(reqs[-1])
        tok.stream_close()
        return ids[:n_ids].cpu().numpy(), offs[: n_rec + 1].cpu().numpy()


def check(torch, P, text, ks, chunks, what="", pieces=None):
    text = np.ascontiguousarray(np.asarray(text, dtype=np.uint8))
    for k in ks:
        want = oracle.encode(text, oracle.KMER, k=k, fmt=oracle.FASTA)
        for chunk in chunks:
            for direct in (True, False):
                gi, go = stream(torch, P, text, k, chunk, pieces, direct)
                tag = "%s k=%d chunk=%d direct=%s" % (what, k, chunk, direct)
                assert go.tolist() == want[1].tolist(), "offsets differ " + tag
                if not np.array_equal(gi, want[0]):
                    m = min(len(gi), len(want[0]))
                    bad = np.nonzero(gi[:m] != want[0][:m])[0]
                    raise AssertionError("ids differ %s: len %d vs %d, first at %s" %
                                         (tag, len(gi), len(want[0]),
                                          int(bad[0]) if len(bad) else m))


def fuzz_concat(seed, n_bytes):
    parts, total, s = [], 0, seed * 1000 + 7
    while total < n_bytes:
        t = synth.fuzz_fasta(s, n_records=8, max_len=3000, crlf_p=0.3, blank_p=0.1)
        s += 1
        parts.append(t)
        total += len(t)
    return np.concatenate(parts)


def test_wrapped_records_many_chunk_sizes(env):
    torch, P = env
    text, _ = synth.fasta_stream(1_400_000, seed=71, rec_lo=300, rec_hi=200_000)
    check(torch, P, text, ks=(2, 6, 15), chunks=(C, C + 17, 200_003), what="wrapped")


@pytest.mark.parametrize("seed", range(4))
def test_fuzz_text_seams_everywhere(env, seed):
    torch, P = env
    text = fuzz_concat(seed, 300_000 + 100_000 * seed)
    check(torch, P, text, ks=(3, 6, 13), chunks=(C, C + 5 + 1000 * seed), what="seed %d" % seed)


def _seq(rng, n, alphabet=b"ACGTacgtN"):
    return bytes(rng.choice(np.frombuffer(alphabet, np.uint8), size=n))


def test_targeted_seams(env):
    """Seams at chosen bytes of the text, chunk size C."""
    torch, P = env
    rng = np.random.default_rng(17)
    parts = []

    def at(pos):  # pad the text with sequence lines up to `pos`
        cur = sum(len(p) for p in parts)
        assert cur <= pos
        body = _seq(rng, pos - cur)
        parts.append(body)

    parts.append(b">first record\n")
    at(C - 3)
    parts.append(b"\n>h2 spans the seam\n")  # header across chunk 1 -> 2
    at(2 * C - 1)
    parts.append(b"\r\nACGTACG\n")  # CR ends chunk 2, LF starts chunk 3
    at(3 * C - 1)
    parts.append(b"\n>h4 right at the seam\nAC")  # '>' is chunk 4's first byte
    at(4 * C - 2)
    parts.append(b"\n>h5\nAC\n>h6\nA")  # a 2-base record inside the seam region
    parts.append(b"\n>" + b"x" * (2 * C + 100) + b"\n")  # whole chunks of header
    at(8 * C + 11)
    parts.append(b"\n>h8\n>h9\n")  # records without bases
    at(9 * C)
    parts.append(b">h10 at a seam after a full sequence line\n")
    text = np.frombuffer(b"".join(parts), np.uint8)
    check(torch, P, text, ks=(2, 5, 6, 14), chunks=(C,), what="targeted")


def test_short_records_across_seams(env):
    """Records shorter than k whose bytes fall on both sides of a seam."""
    torch, P = env
    rng = np.random.default_rng(23)
    recs = []
    while sum(len(r) for r in recs) < 5 * C:
        recs.append(b">r\n" + _seq(rng, int(rng.integers(0, 20)), b"ACGT") + b"\n")
    text = np.frombuffer(b"".join(recs), np.uint8)
    check(torch, P, text, ks=(6, 15), chunks=(C, C + 3), what="short records")


def test_chunk_without_bases_and_control_bytes(env):
    """One chunk is a single header (the compacted path has nothing to
    encode there and declines), another holds control bytes (the direct
    kernel declines): the general kernel takes those chunks, the compacted
    path the others, and the carry passes between them."""
    torch, P = env
    text, _ = synth.fasta_stream(6 * C, seed=29, rec_lo=500, rec_hi=40_000)
    text = text.copy()
    hdr = b"\n>" + b"y" * (C + 200) + b"\n"
    text = np.concatenate([text[:2 * C + 100], np.frombuffer(hdr, np.uint8), text[2 * C + 100:]])
    pos = 4 * C + 1234
    while text[pos] in (ord("\n"), ord(">")):
        pos += 1
    text[pos] = 0x0B
    check(torch, P, text, ks=(4, 6), chunks=(C,), what="declines")


def test_pieces_smaller_than_chunks(env):
    """Pieces of random sizes: chunks below 64 KiB (general kernel) and above
    (compacted path) alternate along the stream."""
    torch, P = env
    text = fuzz_concat(9, 700_000)
    rng = np.random.default_rng(9)
    cuts = np.sort(rng.integers(0, len(text), size=12))
    pieces = [0] + [int(c) for c in cuts] + [len(text)]
    check(torch, P, text, ks=(6,), chunks=(2 * C,), what="pieces", pieces=pieces)
