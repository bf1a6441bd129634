"""The batched form: CUDA-graph capture and replay of encodes (k-mer, char,
BPE), and the launch-shape autotuner with its cache -- results must stay
bit-identical to the oracle whatever the replay count or the chosen shape."""
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
    return torch, P


def _batch(seed, n_seq=300, hi=20_000):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, hi, size=n_seq)
    return synth.markov_batch(lens, 0.4, seed=seed)


def test_graph_replays_many_encodes(env):
    """Four independent encodes (two handles, two modes) captured into one
    graph; inputs rewritten in place between replays.  Odd replays hold
    newlines (the direct path hands over to the general kernel inside the
    graph), even ones do not, so each replay must start from a clean switch
    whatever the one before did."""
    torch, P = env
    B = P.binding
    s = torch.cuda.Stream()
    m = np.loadtxt(TABLE, dtype=np.int32)
    toks = [P.Tokenizer(P.KMER, k=6), P.Tokenizer(P.BPE, merges=m)]
    n_max, seq_max = 8_000_000, 400
    for t in toks:
        t.reserve(n_max, seq_max)
    slots = []
    for i in range(4):
        d = torch.zeros(n_max, dtype=torch.uint8, device="cuda")
        so = torch.zeros(seq_max + 1, dtype=torch.int64, device="cuda")
        ids = torch.empty(n_max, dtype=torch.int32, device="cuda")
        o = torch.empty(seq_max + 1, dtype=torch.int64, device="cuda")
        tot = torch.zeros(2, dtype=torch.int64, device="cuda")
        slots.append((d, so, ids, o, tot))
    # fixed sizes per slot (the graph bakes them in)
    shapes = []
    for i in range(4):
        data, offs = _batch(500 + i)
        shapes.append((len(data), len(offs) - 1))
    torch.cuda.synchronize()
    B.dnatok_graph_begin(toks[0].h, s.cuda_stream)
    for i, (d, so, ids, o, tot) in enumerate(slots):
        n, ns = shapes[i]
        t = toks[i % 2]
        B.dnatok_encode(t.h, d.data_ptr(), n, so.data_ptr(), ns, ids.data_ptr(), ids.numel(),
                        o.data_ptr(), o.numel(), tot.data_ptr(), s.cuda_stream)
    g = B.dnatok_graph_end(toks[0].h, s.cuda_stream)
    try:
        for rep in range(4):
            wants = []
            for i, (d, so, ids, o, tot) in enumerate(slots):
                n, ns = shapes[i]
                # same lengths, new bytes each replay
                rng = np.random.default_rng(1000 * rep + i)
                data, offs = _batch(500 + i)
                data = data.copy()
                flip = rng.choice(len(data), size=len(data) // 20, replace=False)
                alphabet = b"ACGTNacgt\n" if rep % 2 else b"ACGTNacgt"
                data[flip] = rng.choice(np.frombuffer(alphabet, np.uint8), size=len(flip))
                d[:n].copy_(torch.from_numpy(data))
                so[: ns + 1].copy_(torch.from_numpy(offs))
                mode = P.KMER if i % 2 == 0 else P.BPE
                wants.append(oracle.encode(data, mode, k=6 if mode == P.KMER else 1,
                                           seq_offsets=offs, merges=None if mode == P.KMER else m))
            torch.cuda.synchronize()
            B.dnatok_graph_launch(g, s.cuda_stream)
            s.synchronize()
            for t in toks:
                t.sync()
            for i, (d, so, ids, o, tot) in enumerate(slots):
                n_ids, n_rec = (int(x) for x in tot.cpu().tolist())
                wi, wo = wants[i]
                assert o[: n_rec + 1].cpu().numpy().tolist() == wo.tolist(), (rep, i)
                assert np.array_equal(ids[:n_ids].cpu().numpy(), wi), (rep, i)
    finally:
        B.dnatok_graph_destroy(g)
        for t in toks:
            t.close()


def test_graph_needs_reserved_workspace(env):
    torch, P = env
    B = P.binding
    s = torch.cuda.Stream()
    with P.Tokenizer(P.KMER, k=4) as tok:
        d = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
        so = torch.tensor([0, 1 << 20], dtype=torch.int64, device="cuda")
        ids, o, tot = tok.alloc_outputs(1 << 20, 1)
        torch.cuda.synchronize()
        B.dnatok_graph_begin(tok.h, s.cuda_stream)
        with pytest.raises(P.DnatokError) as ei:
            B.dnatok_encode(tok.h, d.data_ptr(), 1 << 20, so.data_ptr(), 1, ids.data_ptr(),
                            ids.numel(), o.data_ptr(), o.numel(), tot.data_ptr(), s.cuda_stream)
        assert ei.value.status == -9
        g = B.dnatok_graph_end(tok.h, s.cuda_stream)
        B.dnatok_graph_destroy(g)


@pytest.mark.parametrize("mode", ["kmer_direct", "kmer_general", "bpe"])
def test_autotune_picks_and_caches(env, tmp_path, mode):
    """The autotuner times the shapes of the kernel the encode takes (the
    direct k-mer kernel's slots, ring depth and CTAs per SM; the general
    kernel's tiles; the BPE segment), keeps the fastest, serves the second
    call from its cache file, and the tuned encode stays bit-exact."""
    torch, P = env
    B = P.binding
    data, offs = _batch(77, n_seq=200, hi=60_000)
    if mode.startswith("kmer"):
        tok = P.Tokenizer(P.KMER, k=6)
        if mode == "kmer_general":
            B.dnatok_set_direct(tok.h, 0)
        want = oracle.encode(data, oracle.KMER, k=6, seq_offsets=offs)
    else:
        m = np.loadtxt(TABLE, dtype=np.int32)
        tok = P.Tokenizer(P.BPE, merges=m)
        want = oracle.encode(data, oracle.BPE, seq_offsets=offs, merges=m)
    d = torch.from_numpy(data).cuda()
    so = torch.from_numpy(offs).cuda()
    ids, o, tot = tok.alloc_outputs(len(data), len(offs) - 1)
    cache = str(tmp_path / "tune.txt")
    best, ms = B.dnatok_autotune(tok.h, d.data_ptr(), len(data), so.data_ptr(), len(offs) - 1,
                                 ids.data_ptr(), ids.numel(), o.data_ptr(), o.numel(), 2, cache)
    assert ms > 0
    text = open(cache).read()
    assert " -> " in text and text.count("\n") == 1
    assert (" direct" in text) == (mode == "kmer_direct")
    best2, ms2 = B.dnatok_autotune(tok.h, d.data_ptr(), len(data), so.data_ptr(),
                                   len(offs) - 1, ids.data_ptr(), ids.numel(), o.data_ptr(),
                                   o.numel(), 2, cache)
    assert best2 == best and ms2 < 0  # served from the cache
    if mode == "kmer_general":
        assert tok.get_launch() == best
    if mode == "kmer_direct":
        slots, ring, ctas = B.dnatok_get_direct_launch(tok.h)
        assert best == (512 * slots, 256, ctas, ring)
    got = tok.encode_host(data, offs)
    assert got[1].tolist() == want[1].tolist()
    assert np.array_equal(got[0], want[0])


@pytest.mark.parametrize("shape", [(2, 4, 0), (1, 8, 0), (4, 2, 0), (2, 4, 1), (4, 2, 3), (1, 8, 2)])
@pytest.mark.parametrize("k", [3, 6, 11])
def test_direct_shapes_are_exact(env, shape, k):
    """Every supported shape of the direct k-mer kernel gives the oracle's ids
    and offsets: record boundaries at every phase, tiny and empty records,
    N runs and lowercase, a misaligned start."""
    torch, P = env
    B = P.binding
    rng = np.random.default_rng(k * 100 + shape[0] * 10 + shape[2])
    lens = np.concatenate([rng.integers(0, 40, size=300), rng.integers(1000, 30000, size=60)])
    rng.shuffle(lens)
    data, offs = synth.markov_batch(lens, 0.4, seed=int(lens.sum() % 1000))
    want = oracle.encode(data, oracle.KMER, k=k, seq_offsets=offs)
    with P.Tokenizer(P.KMER, k=k) as tok:
        B.dnatok_set_direct_launch(tok.h, *shape)
        assert B.dnatok_get_direct_launch(tok.h) == shape
        raw = np.zeros(len(data) + 5, np.uint8)
        raw[5:] = data
        d = torch.from_numpy(raw).cuda()[5:]
        so = torch.from_numpy(offs).cuda()
        ids, o, tot = tok.encode(d, so)
        tok.sync()
        n = int(tot[0])
        assert o[: len(offs)].cpu().tolist() == want[1].tolist()
        assert np.array_equal(ids[:n].cpu().numpy(), want[0])
    with P.Tokenizer(P.KMER, k=k) as tok:
        with pytest.raises(P.DnatokError):
            B.dnatok_set_direct_launch(tok.h, 3, 4, 0)


@pytest.mark.parametrize("fmt", [0, 1])
def test_lookback_wait_runs_out_and_handle_recovers(env, fmt):
    """A look-back wait that can never be satisfied (the chunk before it is
    left unprocessed by fault injection on the host) gives up after the
    handle's wait limit: dnatok_sync reports DNATOK_ERR_TIMEOUT within a few
    seconds, no trap, no hang, and the next encode on the same handle is
    bit-exact against the oracle again."""
    import time
    torch, P = env
    B = P.binding
    if fmt == 0:
        data, offs = synth.markov_batch([300_000, 1, 450_000, 500_000], 0.4, seed=5)
        want = oracle.encode(data, oracle.KMER, k=6, seq_offsets=offs)
    else:
        data, _ = synth.fasta_stream(1_500_000, seed=6, rec_lo=1000, rec_hi=200_000)
        offs = None
        want = oracle.encode(data, oracle.KMER, k=6, fmt=oracle.FASTA)
    with P.Tokenizer(P.KMER, k=6, fmt=fmt) as tok:
        B.dnatok_set_direct(tok.h, 0)  # the general kernel (the one that looks back)
        B.dnatok_set_wait_limit(tok.h, 2000)
        d = torch.from_numpy(data).cuda()
        so = torch.from_numpy(offs).cuda() if offs is not None else None
        ids, o, tot = tok.alloc_outputs(len(data), len(offs) - 1 if offs is not None else 1)
        tok.encode(d, so, ids, o, tot)  # warm: workspace and kernels
        tok.sync()
        B.dnatok_inject_lookback_stall(tok.h, 1)
        t0 = time.time()
        tok.encode(d, so, ids, o, tot)
        with pytest.raises(P.DnatokError) as ei:
            tok.sync()
        assert ei.value.status == -6, ei.value
        assert time.time() - t0 < 30
        B.dnatok_set_wait_limit(tok.h, 0)
        got = tok.encode_host(data, offs)
    assert got[1].tolist() == want[1].tolist()
    assert np.array_equal(got[0], want[0])
