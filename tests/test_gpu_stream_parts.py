"""One stream split into parts encoded by separate ranks (here simulated in
one process on one GPU, the exchanges done in place): each rank's line map,
summary and final encode (StreamPart, dnatok_part_*), then the ranks' ids and
offsets concatenated must equal the oracle's encode of the whole stream.
Cuts fall anywhere -- inside headers, between CR and LF, right before a '>',
inside N runs, inside records shorter than k -- with 1 to 6 ranks, FASTA and
RAW, k-mers and single nucleotides, parts above and below the 64 KiB where
FASTA k-mers take the compacted path, and empty parts (an empty first part
hands the stream start to the next rank)."""
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


def run_parts(torch, P, text, cuts, mode, k, fmt):
    """Encode text split at cuts by len(cuts) + 1 simulated ranks; returns
    the concatenated (ids, offsets) and each rank's (first id, first record)."""
    bounds = [0] + list(cuts) + [len(text)]
    world = len(bounds) - 1
    with P.Tokenizer(mode, k=k, fmt=fmt) as tok:
        parts = []
        for r in range(world):
            seg = np.ascontiguousarray(text[bounds[r]:bounds[r + 1]])
            n = len(seg)
            d = torch.from_numpy(seg).cuda() if n else torch.empty(0, dtype=torch.uint8,
                                                                  device="cuda")
            ids = torch.full((n + 8,), -9, dtype=torch.int32, device="cuda")
            offs = torch.full((n + 4,), -9, dtype=torch.int64, device="cuda")
            parts.append(P.StreamPart(tok, d, ids, offs, r, world))
        maps = [p.line_map() for p in parts]
        states = [p.summary(maps) for p in parts]
        res = [p.finish(states) for p in parts]
        ids = np.concatenate([p.ids[:r[0]].cpu().numpy() for p, r in zip(parts, res)])
        offs = np.concatenate([p.offsets[:r[1]].cpu().numpy() for p, r in zip(parts, res)])
        return ids, offs, [(r[2], r[3]) for r in res], [(r[0], r[1]) for r in res]


def check(torch, P, text, cuts, mode, k, fmt, what=""):
    text = np.ascontiguousarray(np.asarray(text, dtype=np.uint8))
    om = {P.KMER: oracle.KMER, P.CHAR: oracle.CHAR}[mode]
    if fmt == P.FASTA:
        want_ids, want_offs = oracle.encode(text, om, k=k, fmt=oracle.FASTA)
    else:
        want_ids, want_offs = oracle.encode(text, om, k=k,
                                            seq_offsets=np.array([0, len(text)], np.int64))
    ids, offs, firsts, counts = run_parts(torch, P, text, cuts, mode, k, fmt)
    tag = "%s k=%d cuts=%s" % (what, k, list(cuts)[:8])
    assert offs.tolist() == want_offs.tolist(), "offsets differ " + tag
    if not np.array_equal(ids, want_ids):
        m = min(len(ids), len(want_ids))
        bad = np.nonzero(ids[:m] != want_ids[:m])[0]
        raise AssertionError("ids differ %s: %d vs %d, first at %s" %
                             (tag, len(ids), len(want_ids), int(bad[0]) if len(bad) else m))
    # each rank's first id and record are the sums over the ranks before it
    run_ids = run_recs = 0
    for (fi, fr), (ni, no) in zip(firsts, counts):
        assert (fi, fr) == (run_ids, run_recs), tag
        run_ids += ni
        run_recs += no


def fuzz_text(seed, n_bytes):
    parts, total, s = [], 0, seed * 1000 + 3
    while total < n_bytes:
        t = synth.fuzz_fasta(s, n_records=6, max_len=2500, crlf_p=0.3, blank_p=0.1)
        s += 1
        parts.append(t)
        total += len(t)
    return np.concatenate(parts)


@pytest.mark.parametrize("seed", range(5))
def test_fasta_random_cuts(env, seed):
    torch, P = env
    text = fuzz_text(seed, 200_000 + 50_000 * seed)
    rng = np.random.default_rng(seed)
    for world in (1, 2, 3, 6):
        cuts = sorted(int(c) for c in rng.integers(0, len(text) + 1, size=world - 1))
        for k in (2, 6, 13):
            check(torch, P, text, cuts, P.KMER, k, P.FASTA, "seed %d world %d" % (seed, world))
    cuts = sorted(int(c) for c in rng.integers(0, len(text) + 1, size=3))
    check(torch, P, text, cuts, P.CHAR, 1, P.FASTA, "single nucleotides")


def test_fasta_cuts_at_chosen_bytes(env):
    torch, P = env
    text = np.frombuffer(b">r1 first\r\nACGTNNACGTacgt\r\n>r2\nAC\n>r3 x\nACGTACGTAC\nGTACGTA\n"
                         b">r4\n\n>r5\nNNNNNACGTTTT\n", np.uint8).copy()
    cr = bytes(text).index(b"\r\n")
    gt = bytes(text).index(b">r2")
    cuts_sets = [
        [3],                 # inside the first header
        [cr + 1],            # between CR and LF
        [gt],                # right before a '>'
        [gt + 5],            # inside a record shorter than k
        [1, 2, 3, 4, 5],     # one-byte parts
        [10, 10, 10],        # empty parts
        [len(text)],         # an empty last part
        [0],                 # an empty first part
    ]
    for cuts in cuts_sets:
        for k in (1, 3, 6):
            mode = P.CHAR if k == 1 else P.KMER
            check(torch, P, text, cuts, mode, k, P.FASTA, "chosen")


def test_fasta_large_parts_compacted_path(env):
    # parts of several MiB: the compacted FASTA path with a carried state
    torch, P = env
    text, _ = synth.fasta_stream(6_000_000, seed=81, rec_lo=500, rec_hi=400_000)
    rng = np.random.default_rng(81)
    cuts = sorted(int(c) for c in rng.integers(0, len(text), size=3))
    for k in (4, 6):
        check(torch, P, text, cuts, P.KMER, k, P.FASTA, "large parts")


def test_raw_one_record_stream(env):
    torch, P = env
    data = synth.iid_sequence(700_001, 5)
    data = data.copy()
    data[::997] = ord("\n")  # separators inside the record are dropped
    rng = np.random.default_rng(5)
    for world in (2, 4):
        cuts = sorted(int(c) for c in rng.integers(0, len(data) + 1, size=world - 1))
        for k in (1, 5, 6):
            mode = P.CHAR if k == 1 else P.KMER
            check(torch, P, data, cuts, mode, k, P.RAW, "raw world %d" % world)


def test_every_part_empty(env):
    # the last rank starts and ends the stream: FASTA text of no bytes has
    # no record, a RAW stream one empty record
    torch, P = env
    e = np.zeros(0, np.uint8)
    for fmt in (P.FASTA, P.RAW):
        for cuts in ([], [0], [0, 0]):
            check(torch, P, e, cuts, P.KMER, 6, fmt, "empty")


def test_refused_for_other_modes(env):
    torch, P = env
    lut, base = synth.kmer_vocab(3, seed=1)
    with P.Tokenizer(P.KMER_TABLE, k=3, kmer_lut=lut, base_ids=base) as tok:
        d = torch.zeros(16, dtype=torch.uint8, device="cuda")
        ids = torch.zeros(64, dtype=torch.int32, device="cuda")
        offs = torch.zeros(8, dtype=torch.int64, device="cuda")
        with pytest.raises(P.DnatokError):
            P.binding.dnatok_part_encode(tok.h, d.data_ptr(), 16, None, True, ids.data_ptr(), 64,
                                         offs.data_ptr(), 8)
