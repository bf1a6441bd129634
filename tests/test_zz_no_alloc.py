"""The k-mer encode that allocates nothing (dnatok_encode_kmer_noalloc),
called through the C ABI and compared with dnatok_encode on the same inputs
and with the CPU oracle: ids, offsets and totals must be identical, on two
calls in a row (the second call finds the shared scratch array as the first
one left it).  Named so that pytest collects it last; it passes alone and
after the other tests."""
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
    torch.cuda.init()
    return torch, P


def _inputs(torch, seed, n_seq, lo, hi, pad):
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, size=n_seq)
    lens[rng.random(n_seq) < 0.1] = 0
    data, offs = synth.markov_batch(lens, 0.4, seed=seed)
    raw = np.zeros(len(data) + pad, dtype=np.uint8)
    raw[pad:] = data
    d = torch.from_numpy(raw).cuda()[pad:]
    so = torch.from_numpy(offs).cuda()
    return d, so, len(data), n_seq


def _oracle_same(got, d, so, n, n_seq, k):
    """The no-allocation results against the CPU oracle's encoding."""
    data = d.cpu().numpy()[:n] if n else np.zeros(0, np.uint8)
    want_ids, want_offs = oracle.encode(data, oracle.KMER, k=k, seq_offsets=so.cpu().numpy())
    ids, offs, tot = got[0].cpu(), got[1].cpu(), got[2].cpu().tolist()
    assert tot == [len(want_ids), n_seq], (tot, len(want_ids), n_seq)
    assert offs[: n_seq + 1].tolist() == want_offs.tolist()
    assert ids[: len(want_ids)].tolist() == want_ids.tolist()


def _outputs(torch, cap, n_seq):
    ids = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    offs = torch.full((n_seq + 1,), -7, dtype=torch.int64, device="cuda")
    tot = torch.full((2,), -7, dtype=torch.int64, device="cuda")
    return ids, offs, tot


def _with_handle(torch, P, k, d, so, n, n_seq):
    B = P.binding
    h = B.dnatok_create(P.KMER, k)
    try:
        cap = B.dnatok_max_tokens(h, n, n_seq)
        ids, offs, tot = _outputs(torch, cap, n_seq)
        s = torch.cuda.current_stream().cuda_stream
        B.dnatok_encode(h, d.data_ptr() if n else 0, n, so.data_ptr(), n_seq, ids.data_ptr(),
                        ids.numel(), offs.data_ptr(), offs.numel(), tot.data_ptr(), s)
        B.dnatok_sync(h, s)
    finally:
        B.dnatok_destroy(h)
    return ids, offs, tot, cap


def _noalloc(torch, P, k, d, so, n, n_seq, cap):
    B = P.binding
    ids, offs, tot = _outputs(torch, cap, n_seq)
    s = torch.cuda.current_stream().cuda_stream
    B.dnatok_encode_kmer_noalloc(k, d.data_ptr() if n else 0, n, so.data_ptr(), n_seq,
                                 ids.data_ptr(), ids.numel(), offs.data_ptr(), offs.numel(),
                                 tot.data_ptr(), s)
    torch.cuda.synchronize()
    return ids, offs, tot


def _same(a, b):
    ia, oa, ta = a[0].cpu(), a[1].cpu(), a[2].cpu().tolist()
    ib, ob, tb = b[0].cpu(), b[1].cpu(), b[2].cpu().tolist()
    assert ta == tb, (ta, tb)
    assert ta[0] >= 0
    assert oa.tolist() == ob.tolist()
    n_ids = ta[0]
    assert ia[:n_ids].tolist() == ib[:n_ids].tolist()


@pytest.mark.parametrize("k", [1, 3, 6, 15])
def test_noalloc_matches_encode_twice(env, k):
    torch, P = env
    # two different inputs back to back: the second call must not see the
    # first one's descriptors or counters
    cases = [_inputs(torch, 900 + k, 300, 0, 9000, pad=3),
             _inputs(torch, 950 + k, 40, 20000, 90000, pad=0)]
    for d, so, n, n_seq in cases:
        want = _with_handle(torch, P, k, d, so, n, n_seq)
        got = _noalloc(torch, P, k, d, so, n, n_seq, want[3])
        _same(got, want[:3])
        _oracle_same(got, d, so, n, n_seq, k)


def test_noalloc_same_input_twice_and_empty(env):
    torch, P = env
    d, so, n, n_seq = _inputs(torch, 77, 500, 0, 5000, pad=5)
    want = _with_handle(torch, P, 6, d, so, n, n_seq)
    for _ in range(2):
        got = _noalloc(torch, P, 6, d, so, n, n_seq, want[3])
        _same(got, want[:3])
        _oracle_same(got, d, so, n, n_seq, 6)
    # zero bytes in three empty records
    e = torch.zeros(1, dtype=torch.uint8, device="cuda")
    so0 = torch.zeros(4, dtype=torch.int64, device="cuda")
    want0 = _with_handle(torch, P, 6, e, so0, 0, 3)
    for _ in range(2):
        got = _noalloc(torch, P, 6, e, so0, 0, 3, want0[3])
        _same(got, want0[:3])
        _oracle_same(got, e, so0, 0, 3, 6)


def test_noalloc_rejects_oversize_before_launch(env):
    torch, P = env
    B = P.binding
    so = torch.zeros(2, dtype=torch.int64, device="cuda")
    offs = torch.zeros(2, dtype=torch.int64, device="cuda")
    n = B.NOALLOC_MAX_BYTES + 1
    # rejected on the host from the sizes alone: nothing is read or launched
    with pytest.raises(P.DnatokError) as ei:
        B.dnatok_encode_kmer_noalloc(6, so.data_ptr(), n, so.data_ptr(), 1, so.data_ptr(), n,
                                     offs.data_ptr(), 2, 0, 0)
    assert ei.value.status == -3
    with pytest.raises(P.DnatokError) as ei:
        B.dnatok_encode_kmer_noalloc(16, so.data_ptr(), 1, so.data_ptr(), 1, so.data_ptr(), 1,
                                     offs.data_ptr(), 2, 0, 0)
    assert ei.value.status == -1
