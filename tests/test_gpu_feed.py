"""Parity of the fixed-shape model feed (left padding to token_len, int32 or
int64) and of the per-record reverse complement with the CPU oracle:
hand-worked fixtures, ragged batches with short (one warp per row) and long
(strip per CTA) rows, truncation, row windows, the two-stream micro-batch
pipeline with an embedding lookup as its consumer, misaligned and tiny
records for the reverse complement, and both at full 4096-sequence size."""
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


def dev(a, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype))).cuda()


# ------------------------------------------------------------------- feed

def test_feed_hand_examples(P):
    import torch
    from tests import _golden as G
    for tl, pad, toks, row in G.rows("feed_examples.txt"):
        t = np.array(G.ints(toks), np.int32)
        out = P.feed(dev(t if len(t) else np.zeros(1, np.int32)), dev([0, len(t)], np.int64),
                     int(tl), int(pad))
        torch.cuda.synchronize()
        assert out.cpu().numpy()[0].tolist() == G.ints(row), (tl, pad, toks)


@pytest.mark.parametrize("token_len", [1, 7, 100, 512, 513, 1000, 3000])
@pytest.mark.parametrize("width", [4, 8])
def test_feed_ragged(P, token_len, width):
    import torch
    rng = np.random.default_rng(token_len)
    lens = rng.integers(0, 2 * token_len + 2, size=300)
    lens[:5] = [0, token_len, token_len + 1, 1, 0]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ids = rng.integers(0, 4097, size=max(int(offs[-1]), 1)).astype(np.int32)
    dtype = torch.int64 if width == 8 else torch.int32
    out = P.feed(dev(ids), dev(offs), token_len, 4098, dtype=dtype)
    torch.cuda.synchronize()
    want = oracle.feed(ids, offs, token_len, 4098, dtype=np.int64 if width == 8 else np.int32)
    assert np.array_equal(out.cpu().numpy(), want)


def test_feed_row_window_and_negative_pad(P):
    import torch
    ids = np.arange(50, dtype=np.int32)
    offs = np.array([0, 3, 3, 20, 50], np.int64)
    out = P.feed(dev(ids), dev(offs), 10, -100, row_begin=1, n_rows=3)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.feed(ids, offs, 10, -100, 1, 3))


def test_feed_bad_arguments(P):
    import torch
    ids = dev(np.zeros(4, np.int32))
    offs = dev([0, 4], np.int64)
    with pytest.raises(P.DnatokError):
        P.feed(ids, offs, 4, 1 << 40, dtype=torch.int32)  # pad does not fit int32
    with pytest.raises(P.DnatokError):
        P.binding.dnatok_feed(ids.data_ptr(), offs.data_ptr(), 0, 1, 4, 0, 0, 2, 0)


def test_microbatch_rows_rule(P):
    # Algorithm 2: b = min(B_emb, max(1, floor(M / T')))
    assert P.microbatch_rows(64, 100_000, 1000) == 64
    assert P.microbatch_rows(64, 10_000, 1000) == 10
    assert P.microbatch_rows(64, 500, 1000) == 1


@pytest.mark.parametrize("rows_per_batch", [1, 7, 64, 1000])
def test_feed_pipeline_with_embedding_consumer(P, rows_per_batch):
    import torch
    rng = np.random.default_rng(rows_per_batch)
    T, n_rows = 300, 257
    lens = rng.integers(0, T + 50, size=n_rows)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ids = rng.integers(0, 4097, size=int(offs[-1])).astype(np.int32)
    emb = torch.randn(4099, 16, device="cuda")
    result = torch.empty(n_rows, T, 16, device="cuda")
    cs = torch.cuda.Stream()

    def consumer(row_begin, batch, stream):
        with torch.cuda.stream(stream):
            result[row_begin:row_begin + batch.shape[0]] = torch.nn.functional.embedding(batch, emb)

    bufs, fs = P.feed_pipeline(dev(ids), dev(offs), T, 4098, rows_per_batch, consumer,
                               consumer_stream=cs)
    cs.synchronize()
    want = torch.from_numpy(oracle.feed(ids, offs, T, 4098)).cuda()
    assert torch.equal(result, torch.nn.functional.embedding(want, emb))


def test_feed_pipeline_right_after_encode_no_sync(P):
    """encode() and then feed_pipeline() on the caller's current stream with no
    synchronize in between: the feed must see the finished ids."""
    import torch
    data, offs = synth.kmer_batch_4096(n_seq=512)
    want_ids, want_o = oracle.encode(data, oracle.KMER, k=6, seq_offsets=offs)
    T = 512
    emb = torch.randn(4099, 8, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):  # the caller works on its own stream
        with P.Tokenizer(P.KMER, k=6) as tok:
            ids, o, tot = tok.alloc_outputs(len(data), len(offs) - 1, device="cuda")
            ids.fill_(-7)
            tok.encode(dev(data), dev(offs), ids, o, tot, stream=side)
            result = torch.empty(len(offs) - 1, T, 8, device="cuda")

            def consumer(row_begin, batch, stream):
                with torch.cuda.stream(stream):
                    result[row_begin:row_begin + batch.shape[0]] = \
                        torch.nn.functional.embedding(batch, emb)

            P.feed_pipeline(ids, o[: len(offs)], T, 4097, 64, consumer)
            side.synchronize()
    want = torch.from_numpy(oracle.feed(want_ids, want_o, T, 4097)).cuda()
    assert torch.equal(result, torch.nn.functional.embedding(want, emb))


def test_feed_full_kmer_batch_4096(P):
    import torch
    data, offs = synth.kmer_batch_4096()
    ids, o = oracle.encode(data, oracle.KMER, k=6, seq_offsets=offs)
    T = 4096
    out = P.feed(dev(ids), dev(o), T, 4097)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want_rows = [0, 1, 2, 1000, 4095]
    want = oracle.feed(ids, o, T, 4097)
    assert np.array_equal(got, want)
    # the last column holds a record's last id, or its id T - 1 when cut
    assert got.shape == (4096, T) and all(
        got[r, -1] == ids[o[r] + min(o[r + 1] - o[r], T) - 1] for r in want_rows if o[r + 1] > o[r])


# ------------------------------------------------------ reverse complement

def gpu_rc(P, data, offs, pad_in=0, pad_out=0):
    import torch
    raw = np.zeros(len(data) + pad_in, np.uint8)
    raw[pad_in:] = data
    d = dev(raw)[pad_in:]
    out = torch.full((len(data) + pad_out + 1,), 0xEE, dtype=torch.uint8, device="cuda")
    P.reverse_complement(d, dev(offs, np.int64), out=out[pad_out:])
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert (o[:pad_out] == 0xEE).all() and o[pad_out + len(data)] == 0xEE
    return o[pad_out:pad_out + len(data)]


def test_revcomp_hand_examples(P):
    from tests import _golden as G
    for text, want in G.rows("revcomp_examples.txt"):
        d = np.frombuffer(G.unescape(text), np.uint8)
        got = gpu_rc(P, d, [0, len(d)])
        assert got.tobytes() == G.unescape(want), text


@pytest.mark.parametrize("pad_in,pad_out", [(0, 0), (1, 0), (3, 0), (0, 5), (7, 9), (0, 16)])
def test_revcomp_ragged(P, pad_in, pad_out):
    rng = np.random.default_rng(pad_in * 31 + pad_out)
    lens = rng.integers(0, 3000, size=200)
    lens[::7] = rng.integers(0, 20, size=len(lens[::7]))
    data = synth.random_bytes(int(lens.sum()), seed=pad_in + 5)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    got = gpu_rc(P, data, offs, pad_in, pad_out)
    assert np.array_equal(got, oracle.revcomp(data, offs))


def test_revcomp_tiny_records(P):
    # far more records per 4096-byte tile than the kernel's window holds
    rng = np.random.default_rng(4)
    lens = rng.integers(0, 6, size=20000)
    lens[5000:6000] = 0
    data = synth.random_bytes(int(lens.sum()), seed=4)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    assert np.array_equal(gpu_rc(P, data, offs), oracle.revcomp(data, offs))


def test_revcomp_involution_and_arguments(P):
    import torch
    data, offs = synth.markov_batch([5000, 0, 17, 40000], 0.4, seed=3)
    once = gpu_rc(P, data, offs)
    assert np.array_equal(gpu_rc(P, once, offs), data)
    d = dev(data)
    with pytest.raises(P.DnatokError):  # output overlapping the input
        P.binding.dnatok_reverse_complement(d.data_ptr(), len(data), dev(offs).data_ptr(),
                                            len(offs) - 1, d.data_ptr() + 10, 0)


def test_revcomp_full_kmer_batch_4096(P):
    data, offs = synth.kmer_batch_4096()
    assert np.array_equal(gpu_rc(P, data, offs), oracle.revcomp(data, offs))
