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
