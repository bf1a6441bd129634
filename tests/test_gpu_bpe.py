"""BPE merge application on the GPU against the CPU oracle (greedy lowest
rank, leftmost first; C7/C8): ids and offsets bit-identical.  Random small
tables on short words (every segment / halo setting, including a halo of 0
that sends every mid-word segment through the exact repair pass), the
4096-merge table on Markov DNA with N runs, separators, lowercase and many
records, FASTA input, table validation, and the 1 GiB workload (512 x 2 Mb)
on every record."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import _tables

pytestmark = pytest.mark.gpu

TABLE = "tests/golden/bpe_merges_markov45_seed45_4096.txt"


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    return P


@pytest.fixture(scope="module")
def merges4096():
    return np.loadtxt(TABLE, dtype=np.int32)


def gpu_bpe(P, data, merges, offs=None, fmt=0, launch=None):
    with P.Tokenizer(P.BPE, merges=merges, fmt=fmt) as tok:
        if launch:
            P.binding.dnatok_set_bpe_launch(tok.h, *launch)
        return tok.encode_host(data, offs)


def check(got, want, what=""):
    gi, go = got
    wi, wo = want
    assert go.tolist() == wo.tolist(), "offsets differ " + what
    if not np.array_equal(gi, wi):
        n = min(len(gi), len(wi))
        bad = np.nonzero(gi[:n] != wi[:n])[0]
        first = int(bad[0]) if len(bad) else n
        raise AssertionError("ids differ %s: len %d vs %d, first mismatch at %d" %
                             (what, len(gi), len(wi), first))


def test_random_tables_short_words(P):
    rng = np.random.default_rng(61)
    for ti, merges in enumerate(_tables(16, seed=62)):
        m = np.array(merges, dtype=np.int32).reshape(-1, 2)
        ln = [1, 1, 1, 1]
        for a, b in merges:
            ln.append(ln[a] + ln[b])
        if max(ln) > 32:
            continue  # longer tokens are refused at create (test_table_validation)
        lens = rng.integers(0, 40, size=50)
        data, offs = synth.markov_batch(lens, 0.5, seed=100 + ti)
        want = oracle.encode(data, oracle.BPE, seq_offsets=offs, merges=m)
        for launch in [None, (64, 0), (64, 16), (128, 64)]:
            got = gpu_bpe(P, data, m, offs, launch=launch)
            check(got, want, "table %d launch %s" % (ti, launch))


def test_no_merges_is_char(P):
    data, offs = synth.markov_batch([0, 5, 3000, 17], 0.4, seed=3)
    got = gpu_bpe(P, data, np.zeros((0, 2), np.int32), offs)
    want = oracle.encode(data, oracle.CHAR, seq_offsets=offs)
    check(got, want)


@pytest.mark.parametrize("launch", [None, (64, 0), (128, 16), (1024, 0), (4096, 128),
                                    (16384, 256)])
def test_table4096_markov_records(P, merges4096, launch):
    rng = np.random.default_rng(71)
    lens = np.exp(rng.uniform(np.log(1), np.log(200_000), size=40)).astype(np.int64)
    lens[rng.random(40) < 0.1] = 0
    data, offs = synth.markov_batch(lens, 0.45, seed=72)  # N runs, soft-masking
    want = oracle.encode(data, oracle.BPE, seq_offsets=offs, merges=merges4096)
    got = gpu_bpe(P, data, merges4096, offs, launch=launch)
    check(got, want, "launch %s" % (launch,))


def test_separators_and_iupac(P, merges4096):
    rng = np.random.default_rng(81)
    data, offs = synth.markov_batch([30_000, 1, 0, 9_000], 0.45, seed=82)
    # insert separators and IUPAC letters, keeping record offsets consistent
    pieces, new_offs = [], [0]
    for r in range(len(offs) - 1):
        rec = data[offs[r]:offs[r + 1]].copy()
        pos = np.sort(rng.choice(len(rec) + 1, size=len(rec) // 50))
        rec = np.insert(rec, pos, rng.choice(np.frombuffer(b"\n\r \tRYKMN", np.uint8), size=len(pos)))
        pieces.append(rec)
        new_offs.append(new_offs[-1] + len(rec))
    data2 = np.concatenate(pieces)
    offs2 = np.array(new_offs, dtype=np.int64)
    want = oracle.encode(data2, oracle.BPE, seq_offsets=offs2, merges=merges4096)
    for launch in [None, (64, 0)]:
        check(gpu_bpe(P, data2, merges4096, offs2, launch=launch), want, str(launch))


def test_fasta_bpe(P, merges4096):
    data, _ = synth.fasta_stream(3_000_000, seed=91, rec_lo=100, rec_hi=200_000)
    want = oracle.encode(data, oracle.BPE, fmt=oracle.FASTA, merges=merges4096)
    got = gpu_bpe(P, data, merges4096, fmt=P.FASTA)
    check(got, want)
    for seed in range(6):
        d = synth.fuzz_fasta(seed, n_records=6, max_len=500)
        check(gpu_bpe(P, d, merges4096, fmt=P.FASTA),
              oracle.encode(d, oracle.BPE, fmt=oracle.FASTA, merges=merges4096), "fuzz %d" % seed)


def test_empty_inputs(P, merges4096):
    e = np.zeros(0, np.uint8)
    check(gpu_bpe(P, e, merges4096, np.array([0], np.int64)),
          oracle.encode(e, oracle.BPE, seq_offsets=np.array([0], np.int64), merges=merges4096))
    check(gpu_bpe(P, e, merges4096, np.array([0, 0, 0], np.int64)),
          oracle.encode(e, oracle.BPE, seq_offsets=np.array([0, 0, 0], np.int64),
                        merges=merges4096))
    check(gpu_bpe(P, e, merges4096, fmt=P.FASTA),
          oracle.encode(e, oracle.BPE, fmt=oracle.FASTA, merges=merges4096))


def test_table_validation(P):
    with pytest.raises(P.DnatokError) as ei:
        P.Tokenizer(P.BPE, merges=np.array([[0, 4]], np.int32))  # operand not yet defined
    assert ei.value.status == -2
    with pytest.raises(P.DnatokError) as ei:
        P.Tokenizer(P.BPE, merges=np.array([[0, 1], [2, 3], [0, 1]], np.int32))
    assert ei.value.status == -2
    # (A,A), (AA,AA), ... doubles the token length: 64 bases after 6 merges
    chain = np.array([[0, 0]] + [[4 + i, 4 + i] for i in range(5)], np.int32)
    with pytest.raises(P.DnatokError) as ei:
        P.Tokenizer(P.BPE, merges=chain)
    assert ei.value.status == -2


def test_periodic_runs_force_repair(P):
    """Long runs of A under (A,A), (AA,AA), (AAAA,AAAA): the tokens repeat
    every 8 bases from the word start, and a word starting at an odd offset
    puts every mid-word pass out of phase, so its halo never agrees and the
    segments go through the exact repair, run after run (regions of several
    records in parallel).  Ids and offsets must still equal the oracle's."""
    m = np.array([[0, 0], [4, 4], [5, 5], [1, 0], [2, 3]], np.int32)
    rng = np.random.default_rng(17)
    recs = []
    for i in range(12):
        head = bytes(rng.choice(np.frombuffer(b"CGT", np.uint8), size=int(rng.integers(1, 8))))
        recs.append(head + b"A" * int(rng.integers(3000, 40000)) + b"GTCA" * int(rng.integers(0, 50)))
    recs.append(b"A" * 70001)
    data = np.frombuffer(b"".join(recs), np.uint8)
    offs = np.concatenate([[0], np.cumsum([len(r) for r in recs])]).astype(np.int64)
    want = oracle.encode(data, oracle.BPE, seq_offsets=offs, merges=m)
    for launch in [None, (64, 16), (256, 64), (1024, 0)]:
        with P.Tokenizer(P.BPE, merges=m) as tok:
            if launch:
                P.binding.dnatok_set_bpe_launch(tok.h, *launch)
            got = tok.encode_host(data, offs)
            stats = P.binding.dnatok_bpe_stats(tok.h)
        check(got, want, "launch %s" % (launch,))
        assert stats["repaired_segments"] > 0, stats


def test_full_size_1gib_every_record(P, merges4096):
    """512 x 2 Mb uppercase ACGT (1 GiB), the default launch: every record's
    ids equal the oracle's encoding of that record, element by element, and
    the offsets agree.  The oracle runs over ranges of 8 records in worker
    processes that regenerate their records from the seeded generator."""
    import torch

    from tests import _oracle_pool as pool
    data, offs = synth.bpe_apply_corpus()
    n_seq = len(offs) - 1
    with P.Tokenizer(P.BPE, merges=merges4096) as tok:
        d = torch.from_numpy(data).cuda()
        so = torch.from_numpy(offs).cuda()
        ids, o, tot = tok.encode(d, so)
        tok.sync()
        n_ids, n_rec = (int(x) for x in tot.cpu().tolist())
        o = o[: n_rec + 1].cpu().numpy()
        got = ids[:n_ids].cpu().numpy()
        del d, so, ids
    assert n_rec == n_seq and o[0] == 0 and o[-1] == n_ids and np.all(np.diff(o) > 0)
    del data
    ranges = [(r, min(r + 8, n_seq)) for r in range(0, n_seq, 8)]
    checked = 0
    for r0, r1, want, wo in pool.run(pool.bpe_corpus_records, ranges):
        pool.compare(got, o, r0, want, wo, "1 GiB BPE")
        checked += r1 - r0
    assert checked == n_seq
