"""The serving loop: mixed-mode requests submitted while earlier batches run
(continuous batching) under a device-memory budget.  Every request's ids
must equal the oracle's encoding of that request alone, whatever batch it
landed in; the budget must hold at all times; releasing everything must give
all device memory back."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TABLE = "tests/golden/bpe_merges_markov45_seed45_4096.txt"


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


def _requests(seed, n, lo=1, hi=60_000):
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n)).astype(np.int64)
    sizes[rng.random(n) < 0.05] = 0
    modes = rng.choice(3, size=n, p=[0.3, 0.5, 0.2])
    data, offs = synth.markov_batch(sizes, 0.4, seed=seed)
    return [(int(modes[i]), data[offs[i]:offs[i + 1]].copy()) for i in range(n)]


def _want(mode, b, m):
    if mode == 0:
        return oracle.encode(b, oracle.CHAR)[0]
    if mode == 1:
        return oracle.encode(b, oracle.KMER, k=6)[0]
    return oracle.encode(b, oracle.BPE, merges=m)[0]


def _drain(B, srv, ids, timeout=60.0):
    res = {}
    t0 = time.time()
    while len(res) < len(ids):
        for r in ids:
            if r in res:
                continue
            out = B.dnatok_server_poll(srv, r)
            if out is not None:
                res[r] = out
        assert time.time() - t0 < timeout, "requests did not complete"
    return res


def test_mixed_requests_match_alone(env):
    torch, P = env
    B = P.binding
    m = np.loadtxt(TABLE, dtype=np.int32)
    reqs = _requests(11, 400)
    srv = B.dnatok_server_create(budget_bytes=256 << 20, host_arena_bytes=128 << 20,
                                 max_batch_bytes=4 << 20, max_batch_requests=64, n_slots=4,
                                 kmer_k=6, merges=m)
    try:
        ids = []
        for mode, b in reqs:
            r = B.dnatok_server_submit(srv, mode, b.ctypes.data if len(b) else 0, len(b))
            assert r is not None
            ids.append(r)
        res = _drain(B, srv, ids)
        st = B.dnatok_server_stats(srv)
        assert st["batches_launched"] < len(reqs)  # requests were batched
        for r, (mode, b) in zip(ids, reqs):
            _, n_ids, lat = res[r]
            got = B.dnatok_server_read(srv, r, n_ids)
            want = _want(mode, b, m)
            assert np.array_equal(got, want), (mode, len(b))
            assert lat > 0
            B.dnatok_server_release(srv, r)
        assert B.dnatok_server_stats(srv)["device_bytes_in_use"] == 0
    finally:
        B.dnatok_server_destroy(srv)


def test_budget_holds_and_requests_arrive_while_running(env):
    """A budget of a few batches: requests keep arriving from another thread
    while batches run; the arena never exceeds the budget; every result is
    still the alone result."""
    torch, P = env
    B = P.binding
    m = np.loadtxt(TABLE, dtype=np.int32)
    reqs = _requests(12, 300, hi=200_000)
    budget = 6 << 20
    srv = B.dnatok_server_create(budget_bytes=budget, host_arena_bytes=256 << 20,
                                 max_batch_bytes=1 << 20, max_batch_requests=16, n_slots=3,
                                 kmer_k=6, merges=m)
    try:
        ids = [None] * len(reqs)
        peak = [0]
        stop = [False]

        def watch():
            while not stop[0]:
                peak[0] = max(peak[0], B.dnatok_server_stats(srv)["device_bytes_in_use"])

        w = threading.Thread(target=watch)
        w.start()
        done = {}
        for i, (mode, b) in enumerate(reqs):
            while True:
                r = B.dnatok_server_submit(srv, mode, b.ctypes.data if len(b) else 0, len(b))
                if r is not None:
                    break
                time.sleep(0.001)
            ids[i] = r
            if i % 7 == 0:
                time.sleep(0.0005)
            # release finished requests as we go so the budget frees up
            for j in range(i + 1):
                rj = ids[j]
                if rj in done:
                    continue
                out = B.dnatok_server_poll(srv, rj)
                if out is not None:
                    done[rj] = B.dnatok_server_read(srv, rj, out[1])
                    B.dnatok_server_release(srv, rj)
        t0 = time.time()
        while len(done) < len(reqs):
            for rj in ids:
                if rj in done:
                    continue
                out = B.dnatok_server_poll(srv, rj)
                if out is not None:
                    done[rj] = B.dnatok_server_read(srv, rj, out[1])
                    B.dnatok_server_release(srv, rj)
            assert time.time() - t0 < 60
        stop[0] = True
        w.join()
        assert 0 < peak[0] <= budget
        for r, (mode, b) in zip(ids, reqs):
            assert np.array_equal(done[r], _want(mode, b, m)), (mode, len(b))
        assert B.dnatok_server_stats(srv)["device_bytes_in_use"] == 0
    finally:
        B.dnatok_server_destroy(srv)


def test_oversize_and_unknown(env):
    torch, P = env
    B = P.binding
    srv = B.dnatok_server_create(budget_bytes=16 << 20, host_arena_bytes=4 << 20,
                                 max_batch_bytes=1 << 20, max_batch_requests=8, n_slots=1)
    try:
        big = np.zeros(2 << 20, np.uint8)
        with pytest.raises(P.DnatokError) as ei:
            B.dnatok_server_submit(srv, 0, big.ctypes.data, len(big))
        assert ei.value.status == -3
        with pytest.raises(P.DnatokError) as ei:
            B.dnatok_server_poll(srv, 12345)
        assert ei.value.status == -7
    finally:
        B.dnatok_server_destroy(srv)


def _one(B, srv, mode, b, timeout=30.0):
    r = B.dnatok_server_submit(srv, mode, b.ctypes.data if len(b) else 0, len(b))
    assert r is not None
    t0 = time.time()
    while True:
        try:
            out = B.dnatok_server_poll(srv, r)
        except Exception as e:  # a failed request
            return r, e
        if out is not None:
            return r, out
        assert time.time() - t0 < timeout, "request did not complete"


@pytest.mark.parametrize("kind", [1, 2])
def test_failed_batch_then_next_request_exact(env, kind):
    """A batch that fails -- refused on the host (kind 1) or with a device-side
    error recorded by a kernel (kind 2), both injected -- completes with an
    error for its request; the next request, on the same slot and handle,
    comes back bit-exact against the oracle."""
    torch, P = env
    B = P.binding
    m = np.loadtxt(TABLE, dtype=np.int32)
    reqs = _requests(91, 6, lo=1000, hi=200_000)
    srv = B.dnatok_server_create(budget_bytes=64 << 20, host_arena_bytes=16 << 20,
                                 max_batch_bytes=1 << 20, max_batch_requests=8, n_slots=1,
                                 kmer_k=6, merges=m)
    try:
        for mode in (0, 1, 2):
            b = reqs[mode][1]
            B.dnatok_server_inject(srv, kind, 1)
            r, out = _one(B, srv, mode, b)
            assert isinstance(out, P.DnatokError) and out.status == -4, out
            B.dnatok_server_release(srv, r)
            r, out = _one(B, srv, mode, b)
            assert not isinstance(out, Exception), out
            got = B.dnatok_server_read(srv, r, out[1])
            assert np.array_equal(got, _want(mode, b, m)), (kind, mode)
            B.dnatok_server_release(srv, r)
        assert B.dnatok_server_stats(srv)["device_bytes_in_use"] == 0
    finally:
        B.dnatok_server_destroy(srv)


def test_budget_too_small_for_one_request(env):
    torch, P = env
    B = P.binding
    with pytest.raises(P.DnatokError) as ei:
        B.dnatok_server_create(budget_bytes=1 << 20, host_arena_bytes=4 << 20,
                               max_batch_bytes=1 << 20, max_batch_requests=8, n_slots=1)
    assert ei.value.status == -5
