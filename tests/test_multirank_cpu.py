"""The multi-process path on CPU with world_size 2 over gloo: each rank takes
its byte-balanced record shard (dnatok_shard_records), encodes it -- here
with the oracle standing in for the per-GPU encode, as the CPU has no GPU --
and turns its local id offsets into global ones with the single exchange the
path needs (global_id_offsets: an all_gather of one id count per rank).
The ranks' results, concatenated, must equal one encode of the whole batch;
no rank exchanges any data-path bytes."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, mode, k, out_q):
    import torch.distributed as dist
    import torch
    import paper_2601_05531_gb300 as P
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data, offs = synth.markov_batch(synth.log_uniform_lengths(300, 50, 20000, seed=9), 0.4,
                                        seed=9)
        b = P.shard_records(offs, world)
        r0, r1 = int(b[rank]), int(b[rank + 1])
        lo, hi = int(offs[r0]), int(offs[r1])
        ids, loc = oracle.encode(data[lo:hi], mode, k=k, seq_offsets=offs[r0:r1 + 1] - lo)
        g, total = P.global_id_offsets(torch.from_numpy(loc))
        out_q.put((rank, r0, r1, ids, g.numpy(), total))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode,k", [(oracle.KMER, 6), (oracle.CHAR, 1), (oracle.KMER_OVERLAP, 5)])
def test_two_ranks_match_one_encode(mode, k):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, mode, k, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    data, offs = synth.markov_batch(synth.log_uniform_lengths(300, 50, 20000, seed=9), 0.4, seed=9)
    want_ids, want_offs = oracle.encode(data, mode, k=k, seq_offsets=offs)
    (_, a0, a1, ids0, g0, t0), (_, b0, b1, ids1, g1, t1) = res
    assert a0 == 0 and a1 == b0 and b1 == len(offs) - 1  # the shards cover the records
    assert t0 == t1 == len(want_ids)
    assert np.array_equal(np.concatenate([ids0, ids1]), want_ids)
    assert np.array_equal(np.concatenate([g0[:-1], g1]), want_offs)


def _rank_main_small(rank, world, port, out_q):
    import torch.distributed as dist
    import torch
    import paper_2601_05531_gb300 as P
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # two records over three ranks: one rank's shard is empty
        data, offs = synth.markov_batch([900, 40], 0.4, seed=4)
        b = P.shard_records(offs, world)
        r0, r1 = int(b[rank]), int(b[rank + 1])
        lo, hi = int(offs[r0]), int(offs[r1])
        ids, loc = oracle.encode(data[lo:hi], oracle.KMER, k=3, seq_offsets=offs[r0:r1 + 1] - lo)
        g, total = P.global_id_offsets(torch.from_numpy(loc))
        out_q.put((rank, r0, r1, ids, g.numpy(), total))
    finally:
        dist.destroy_process_group()


def test_three_ranks_with_an_empty_shard():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main_small, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    data, offs = synth.markov_batch([900, 40], 0.4, seed=4)
    want_ids, want_offs = oracle.encode(data, oracle.KMER, k=3, seq_offsets=offs)
    assert any(r1 == r0 for _, r0, r1, _, _, _ in res)  # one shard holds no record
    ids = np.concatenate([x[3] for x in res])
    got_offs = [0]
    for _, r0, r1, _, g, _ in res:
        got_offs.extend(g[1:].tolist())
    assert np.array_equal(ids, want_ids)
    assert got_offs == want_offs.tolist()
    assert all(x[5] == len(want_ids) for x in res)


# ---------------------------------------------------------------- split stream
#
# encode_stream_part's exchanges over gloo with 2 to 4 processes.  A CPU has
# no GPU to encode the parts, so the two device calls are replaced by the
# scan element written out from its definition (tests.test_part_cpu) over a
# stream of symbols and record boundaries: what is tested is everything
# around them -- the all_gathers, the rank that starts the stream, the order
# of the host combines (the real dnatok_part_combine) -- and each rank must
# receive as its start state exactly the state of the whole stream before it.

def _stream_events(seed, world):
    rng = np.random.default_rng(seed)
    ev = [None if rng.random() < 0.03 else int(rng.integers(0, 5)) for _ in range(3000)]
    cuts = sorted(int(c) for c in rng.integers(0, len(ev) + 1, size=world - 1))
    if seed % 3 == 0:
        cuts[0] = 0  # an empty first part: the next rank starts the stream
    return ev, [0] + cuts + [len(ev)]


def _stream_rank_main(rank, world, port, seed, k, out_q):
    import torch
    import torch.distributed as dist
    import paper_2601_05531_gb300 as P
    from paper_2601_05531_gb300 import binding as B
    from tests.test_part_cpu import span_state
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ev, b = _stream_events(seed, world)
        mine = ev[b[rank]:b[rank + 1]]
        seen = {}

        def fake_map(h, addr, n, stream=0):
            return 0 | (1 << 2) | (2 << 4)  # every part keeps the line state

        def fake_encode(h, addr, n, before, last, *args):
            own = mine + ([None] if last else [])
            if before is None:
                st = span_state([None] + own, k) + [0]
            elif before.nb == 0:
                st = span_state(own, k) + [before.line_state]
            else:
                seen["before"] = before.as_list()
                st = B.dnatok_part_combine(k, before,
                                           B.PartState.from_list(span_state(own, k) + [0])).as_list()
            return B.PartState.from_list(st)

        B.dnatok_part_line_map = fake_map
        B.dnatok_part_encode = fake_encode

        class Tok:
            h = None
            mode = B.KMER

        Tok.k = k
        part = torch.zeros(len(mine), dtype=torch.uint8)  # only its length is read
        res = P.encode_stream_part(Tok(), part, torch.zeros(1, dtype=torch.int32),
                                   torch.zeros(1, dtype=torch.int64), stream=0)
        out_q.put((rank, tuple(int(x) for x in res), seen.get("before")))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,seed,k", [(2, 1, 6), (3, 3, 13), (4, 4, 2), (4, 6, 1)])
def test_split_stream_exchanges(world, seed, k):
    import multiprocessing as mp
    import __graft_entry__
    from tests.test_part_cpu import span_state
    __graft_entry__.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stream_rank_main, args=(r, world, port, seed, k, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=60) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ev, b = _stream_events(seed, world)
    lead = next((r for r in range(world) if b[r + 1] > b[r]), world - 1)
    total = span_state([None] + ev + [None], k)
    n_ids = n_recs = 0
    for rank, (ni, no, first_id, first_rec), before in got:
        if rank < lead:
            assert (ni, no, first_id, first_rec) == (0, 0, 0, 0)
            continue
        want_before = span_state([None] + ev[:b[rank]], k)
        if rank > lead:
            assert before == want_before + [0], rank  # the state of everything before it
        assert (first_id, first_rec) == (n_ids, n_recs) == (
            (want_before[2], want_before[0]) if rank > lead else (0, 0))
        n_ids += ni
        n_recs += no
    assert (n_ids, n_recs) == (total[2], total[0])
