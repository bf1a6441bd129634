"""Host-streamed encode (pinned staging, device slot ring, copy/compute
streams, carry across chunks) against the CPU oracle run on the whole stream
at once: ids and offsets must be bit-identical whatever the piece sizes,
chunk size, slot count, overlap setting and host memory kind."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    return torch, P


def _cuts(n, seed, n_pieces, empty_p=0.1):
    """Random piece boundaries over [0, n], some pieces empty."""
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.integers(0, n + 1, size=max(n_pieces - 1, 0)))
    cuts = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    extra = rng.random(len(cuts)) < empty_p
    return np.sort(np.concatenate([cuts, cuts[extra]]))


def _stream(torch, P, tok, data, pieces, pinned=False, chunk=0, slots=0, overlap=True,
            raw_records=None, cap=None):
    """Feed data[pieces[i]:pieces[i+1]] in order; raw_records: set of piece
    indices flagged NEW_RECORD.  Returns (ids, offsets) trimmed."""
    n = len(data)
    cap = max(n, 1) if cap is None else cap
    ids = torch.full((cap,), -9, dtype=torch.int32, device="cuda")
    offs = torch.full((n + len(pieces) + 2,), -9, dtype=torch.int64, device="cuda")
    tok.stream_open(ids, offs, chunk_bytes=chunk, n_slots=slots, overlap=overlap)
    host = torch.from_numpy(np.ascontiguousarray(data))
    if pinned:
        host = host.pin_memory()
    reqs = []
    for i in range(len(pieces) - 1):
        a, b = int(pieces[i]), int(pieces[i + 1])
        fl = 0
        if raw_records is not None and i in raw_records:
            fl |= P.NEW_RECORD
        if i == len(pieces) - 2:
            fl |= P.END_OF_STREAM
        if pinned:
            reqs.append(tok.stream_submit(host[a:b], fl | P.HOST_PINNED))
        else:
            reqs.append(tok.stream_submit(data[a:b], fl))
    res = [tok.stream_wait(r) for r in reqs]
    n_ids, n_rec, bytes_in = res[-1]
    assert bytes_in == n
    # totals are cumulative and never decrease
    assert all(res[i][0] <= res[i + 1][0] for i in range(len(res) - 1))
    tok.stream_close()
    return ids[:n_ids].cpu().numpy(), offs[: n_rec + 1].cpu().numpy()


def _same(got, want, what):
    assert got[1].tolist() == want[1].tolist(), "offsets differ " + what
    assert np.array_equal(got[0], want[0]), "ids differ " + what


@pytest.mark.parametrize("mode,k", [(0, 1), (1, 3), (1, 6), (1, 15)])
def test_fasta_stream_matches_whole(env, mode, k):
    torch, P = env
    data, _ = synth.fasta_stream(1_500_000, seed=101 + k, rec_lo=1000, rec_hi=300_000)
    want = oracle.encode(data, mode, k=k, fmt=oracle.FASTA)
    with P.Tokenizer(mode, k=k, fmt=P.FASTA) as tok:
        for j, (chunk, slots, pinned, overlap, npieces) in enumerate(
                [(65536, 3, False, True, 7), (100_003, 2, True, True, 3),
                 (1 << 20, 4, False, False, 1), (4099, 3, True, True, 40)]):
            cuts = _cuts(len(data), 7 * j + k, npieces)
            got = _stream(torch, P, tok, data, cuts, pinned, chunk, slots, overlap)
            _same(got, want, "k=%d case %d" % (k, j))


def test_fasta_fuzz_small_chunks(env):
    torch, P = env
    for seed in range(12):
        data = synth.fuzz_fasta(seed, n_records=8, max_len=700)
        for mode, k in [(0, 1), (1, 4)]:
            want = oracle.encode(data, mode, k=k, fmt=oracle.FASTA)
            with P.Tokenizer(mode, k=k, fmt=P.FASTA) as tok:
                got = _stream(torch, P, tok, data, _cuts(len(data), seed, 6, 0.3),
                              chunk=17 + seed)
            _same(got, want, "seed %d mode %d" % (seed, mode))


@pytest.mark.parametrize("k", [1, 6, 11])
def test_raw_stream_records(env, k):
    torch, P = env
    rng = np.random.default_rng(300 + k)
    lens = rng.integers(0, 60_000, size=60)
    lens[rng.random(60) < 0.15] = 0
    data, offs = synth.markov_batch(lens, 0.4, seed=300 + k)
    want = oracle.encode(data, 1, k=k, seq_offsets=offs)
    # each record split into 1-3 pieces; the first piece of a record is
    # flagged NEW_RECORD
    cuts, flagged = [0], set()
    for r in range(len(lens)):
        a, b = int(offs[r]), int(offs[r + 1])
        inner = np.sort(rng.integers(a, b + 1, size=int(rng.integers(0, 3))))
        flagged.add(len(cuts) - 1)
        for c in list(inner) + [b]:
            cuts.append(int(c))
    cuts = np.array(cuts, dtype=np.int64)
    with P.Tokenizer(P.KMER, k=k) as tok:
        for chunk, pinned in [(8192, False), (250_001, True)]:
            got = _stream(torch, P, tok, data, cuts, pinned, chunk, raw_records=flagged)
            _same(got, want, "k=%d chunk %d" % (k, chunk))


def test_empty_streams(env):
    torch, P = env
    with P.Tokenizer(P.KMER, k=6) as tok:
        # RAW: one empty piece = one empty record
        got = _stream(torch, P, tok, np.zeros(0, np.uint8), np.array([0, 0]))
        _same(got, oracle.encode(np.zeros(0, np.uint8), 1, k=6,
                                 seq_offsets=np.array([0, 0], np.int64)), "raw empty")
        # three empty records
        got = _stream(torch, P, tok, np.zeros(0, np.uint8), np.array([0, 0, 0, 0]),
                      raw_records={0, 1, 2})
        assert got[1].tolist() == [0, 0, 0, 0] and len(got[0]) == 0
    with P.Tokenizer(P.KMER, k=6, fmt=P.FASTA) as tok:
        e = np.zeros(0, np.uint8)
        _same(_stream(torch, P, tok, e, np.array([0, 0])),
              oracle.encode(e, 1, k=6, fmt=oracle.FASTA), "fasta empty")
        d = np.frombuffer(b">h\nACGTACG\n", np.uint8)
        _same(_stream(torch, P, tok, d, np.array([0, 0, 0, 5, len(d), len(d)])),
              oracle.encode(d, 1, k=6, fmt=oracle.FASTA), "fasta with empty pieces")


def test_stream_errors(env):
    torch, P = env
    data, offs = synth.markov_batch([5000, 7000], 0.4, seed=5)
    with P.Tokenizer(P.KMER, k=1) as tok:
        ids = torch.empty(100, dtype=torch.int32, device="cuda")
        o = torch.empty(4, dtype=torch.int64, device="cuda")
        tok.stream_open(ids, o, chunk_bytes=4096)
        with pytest.raises(P.DnatokError) as ei:
            tok.stream_open(ids, o)
        assert ei.value.status == -9
        r = tok.stream_submit(data, P.END_OF_STREAM)
        with pytest.raises(P.DnatokError) as ei:
            tok.stream_wait(r)
        assert ei.value.status == -3  # ids_out too small
        with pytest.raises(P.DnatokError) as ei:
            tok.stream_submit(data[:10])
        assert ei.value.status == -9  # after END_OF_STREAM
        with pytest.raises(P.DnatokError) as ei:
            tok.stream_poll(r + 5)
        assert ei.value.status == -7
        tok.stream_close()
        with pytest.raises(P.DnatokError):
            tok.stream_close()
        # the handle still encodes normally afterwards
        got = tok.encode_host(data, offs)
        want = oracle.encode(data, 1, k=1, seq_offsets=offs)
        _same(got, want, "after stream")


def test_poll_pending_then_done(env):
    torch, P = env
    data, _ = synth.fasta_stream(8_000_000, seed=9)
    want = oracle.encode(data, 1, k=6, fmt=oracle.FASTA)
    with P.Tokenizer(P.KMER, k=6, fmt=P.FASTA) as tok:
        ids = torch.empty(len(data), dtype=torch.int32, device="cuda")
        o = torch.empty(len(data) + 2, dtype=torch.int64, device="cuda")
        tok.stream_open(ids, o, chunk_bytes=1 << 20)
        r = tok.stream_submit(data, P.END_OF_STREAM)
        res = None
        for _ in range(10_000_000):
            res = tok.stream_poll(r)
            if res is not None:
                break
        assert res is not None
        tok.stream_close()
        _same((ids[: res[0]].cpu().numpy(), o[: res[1] + 1].cpu().numpy()), want, "poll")


def test_full_size_fasta_stream_every_record(env):
    """The 8 GiB FASTA stream in pinned host memory, streamed in 64 MiB
    chunks through 3 slots as the benchmark runs it: every record's ids equal
    the oracle's encoding of that record, element by element, records cut by
    a chunk boundary included.  The oracle runs over ranges of about 128 MB
    in worker processes that regenerate their records from the seeded
    generator."""
    torch, P = env
    from tests import _oracle_pool as pool
    n = 8 << 30
    chunk = 64 << 20
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    _, lay = synth.fasta_stream(n, seed=47, out=host.numpy())
    n_rec = len(lay.rec_off)
    ids = torch.empty(n // 6 + 2 * n_rec + 1024, dtype=torch.int32, device="cuda")
    offs = torch.empty(n_rec + 2, dtype=torch.int64, device="cuda")
    with P.Tokenizer(P.KMER, k=6, fmt=P.FASTA) as tok:
        tok.stream_open(ids, offs, chunk_bytes=chunk, n_slots=3)
        r = tok.stream_submit(host, P.HOST_PINNED | P.END_OF_STREAM)
        n_ids, n_out_rec, bytes_in = tok.stream_wait(r)
        tok.stream_close()
    assert bytes_in == n and n_out_rec == n_rec
    o = offs[: n_rec + 1].cpu().numpy()
    assert o[0] == 0 and o[-1] == n_ids and np.all(np.diff(o) >= 0)
    got = ids[:n_ids].cpu().numpy()
    del ids, host
    starts = np.append(lay.rec_off, n)
    # record ranges of about 128 MB each
    cuts = np.searchsorted(starts, np.arange(0, n, 128 << 20), side="left")
    bounds = sorted(set(int(c) for c in cuts) | {0, n_rec})
    ranges = [(n, 47, 6, a, b) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    checked = 0
    for r0, r1, want, wo in pool.run(pool.fasta_stream_records, ranges):
        pool.compare(got, o, r0, want, wo, "8 GiB FASTA stream")
        checked += r1 - r0
    assert checked == n_rec
