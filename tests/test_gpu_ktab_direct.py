"""The single pass of table-driven k-mers over RAW bytes (window plan, then
one look-back kernel that reads the bytes once and writes the ids once):
ids, offsets and totals bit-identical with the oracle on inputs that stress
its parts -- one long record across thousands of tiles (look-back over many
predecessors), records ending exactly on tile boundaries, more records than
one pass of the plan takes, misaligned ids buffers (the staged tile's
16-byte stores), tables where no window has an entry (tiles too large to
stage), and that it is the path that ran, while a separator anywhere sends
the encode to the general path behind it."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import random_ktab

pytestmark = pytest.mark.gpu

KW = 2048  # windows per tile of the single pass


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    return P


def run(P, data, offs, k, lut, base, ids_shift=0, direct=True):
    """Encode through the C ABI with the ids written `ids_shift` int32s into
    a larger buffer; returns (ids, offsets, totals, direct_ran, nothing
    written outside [0, capacity))."""
    import torch
    n, n_seq = len(data), len(offs) - 1
    with P.Tokenizer(P.KMER_TABLE, k=k, kmer_lut=lut, base_ids=base) as tok:
        P.binding.dnatok_set_direct(tok.h, direct)
        d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
        so = torch.from_numpy(np.asarray(offs, dtype=np.int64)).cuda()
        cap = tok.max_tokens(n, n_seq)
        buf = torch.full((cap + ids_shift + 8,), -7, dtype=torch.int32, device="cuda")
        ids = buf[ids_shift:ids_shift + cap]
        o = torch.full((n_seq + 1,), -7, dtype=torch.int64, device="cuda")
        tot = torch.zeros(2, dtype=torch.int64, device="cuda")
        P.binding.dnatok_encode(tok.h, d.data_ptr(), n, so.data_ptr(), n_seq, ids.data_ptr(), cap,
                                o.data_ptr(), n_seq + 1, tot.data_ptr(), P._stream_ptr(None))
        tok.sync()
        ran = P.binding.dnatok_direct_ran(tok.h)
        n_ids, n_rec = (int(x) for x in tot.cpu().tolist())
        b = buf.cpu().numpy()
        # entries past the ids produced are scratch up to the capacity
        guard = (b[:ids_shift] == -7).all() and (b[ids_shift + cap:] == -7).all()
        return b[ids_shift:ids_shift + n_ids], o.cpu().numpy(), (n_ids, n_rec), ran, guard


def check(P, data, offs, k, lut, base, what, ids_shift=0, expect_direct=1):
    wi, wo = oracle.encode_ktab(data, k, lut, base, seq_offsets=offs)
    gi, go, tot, ran, guard = run(P, data, offs, k, lut, base, ids_shift)
    assert tot == (len(wi), len(offs) - 1), "totals %s" % what
    assert go.tolist() == wo.tolist(), "offsets differ " + what
    if not np.array_equal(gi, wi):
        bad = np.nonzero(gi != wi)[0]
        raise AssertionError("ids differ %s at %d of %d" % (what, int(bad[0]), len(wi)))
    assert guard, "ids written outside the buffer " + what
    assert ran == expect_direct, "direct_ran %d, wanted %d (%s)" % (ran, expect_direct, what)


@pytest.mark.parametrize("k", [1, 3, 6, 7, 10])
def test_one_long_record(P, k):
    # about 3 MB in one record: thousands of tiles, each looking back over
    # predecessors still being counted
    data = synth.iid_sequence(3_000_017, 11 + k)
    offs = np.array([0, len(data)], np.int64)
    rng = np.random.default_rng(k)
    lut, base = (synth.kmer_vocab(k, seed=k) if k <= 7 else random_ktab(rng, k, hole_p=0.1))
    check(P, data, offs, k, lut, base, "k=%d" % k)


@pytest.mark.parametrize("k", [2, 6])
def test_records_on_tile_boundaries(P, k):
    # records of exactly one tile of windows, and one window more or less,
    # plus tails of every length
    rng = np.random.default_rng(30 + k)
    lens = []
    for _ in range(40):
        w = KW * int(rng.integers(1, 3)) + int(rng.integers(-1, 2))
        lens.append(w * k + int(rng.integers(0, k)))
    lens = np.array(lens, np.int64)
    data, offs = synth.markov_batch(lens, 0.4, seed=30 + k)
    lut, base = random_ktab(rng, k, hole_p=0.2)
    check(P, data, offs, k, lut, base, "k=%d" % k)


def test_many_records_several_plan_passes(P):
    # 9000 records (the plan stages 4096 per pass), empty ones included
    rng = np.random.default_rng(41)
    lens = rng.integers(50, 2500, size=9000)
    lens[rng.random(9000) < 0.05] = 0
    data, offs = synth.markov_batch(lens, 0.4, seed=41)
    for k in (4, 6):
        lut, base = synth.kmer_vocab(k, seed=40 + k)
        check(P, data, offs, k, lut, base, "k=%d" % k)


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_misaligned_ids_buffer(P, shift):
    data, offs = synth.markov_batch(np.random.default_rng(5).integers(0, 9000, size=120), 0.4,
                                    seed=5)
    lut, base = synth.kmer_vocab(6, seed=5)
    check(P, data, offs, 6, lut, base, "shift %d" % shift, ids_shift=shift)


def test_no_entries_tiles_too_large_to_stage(P):
    # every whole window falls back to its k symbols: 6 ids per window, more
    # than a tile stages, so the ids go straight to the output
    data, offs = synth.markov_batch(np.random.default_rng(6).integers(0, 20000, size=60), 0.4,
                                    seed=6)
    lut = np.full(5 ** 6, -1, np.int32)
    base = np.array([11, 12, 13, 14, 15], np.int32)
    check(P, data, offs, 6, lut, base, "no entries", ids_shift=1)


def test_separator_sends_to_general_path(P):
    # one newline in the last record: the single pass raises the gate and
    # the general path (which drops the separator) gives the oracle's ids
    data, offs = synth.markov_batch(np.random.default_rng(7).integers(100, 5000, size=50), 0.4,
                                    seed=7)
    data = data.copy()
    data[len(data) - 3] = ord("\n")
    lut, base = synth.kmer_vocab(6, seed=7)
    check(P, data, offs, 6, lut, base, "newline", expect_direct=0)


def test_direct_off_and_malformed_offsets(P):
    import torch
    data, offs = synth.markov_batch(np.random.default_rng(8).integers(0, 3000, size=30), 0.4, seed=8)
    lut, base = synth.kmer_vocab(5, seed=8)
    wi, wo = oracle.encode_ktab(data, 5, lut, base, seq_offsets=offs)
    gi, go, tot, ran, guard = run(P, data, offs, 5, lut, base, direct=False)
    assert go.tolist() == wo.tolist() and np.array_equal(gi, wi) and guard
    # offsets that decrease, between two good encodes on one handle: the plan
    # declines, nothing behind it reads the window offsets it left unwritten,
    # the general path reports the error, and the handle works again after
    bad = offs.copy()
    bad[5], bad[6] = offs[6] + 1, offs[5]
    with P.Tokenizer(P.KMER_TABLE, k=5, kmer_lut=lut, base_ids=base) as tok:
        d = torch.from_numpy(data).cuda()
        so = torch.from_numpy(offs).cuda()
        for good in (True, False, True):
            ids, o, tot = tok.encode(d, so if good else torch.from_numpy(bad).cuda())
            if not good:
                with pytest.raises(P.DnatokError):
                    tok.sync()
                continue
            tok.sync()
            n_ids = int(tot[0])
            assert o.cpu().numpy().tolist() == wo.tolist()
            assert np.array_equal(ids[:n_ids].cpu().numpy(), wi)


def test_more_records_than_the_plan_takes(P):
    # 70000 short records: past the 65536 the direct plans take, so the
    # general path encodes them on its own
    rng = np.random.default_rng(12)
    data, offs = synth.markov_batch(rng.integers(0, 60, size=70000), 0.4, seed=12)
    lut, base = synth.kmer_vocab(4, seed=12)
    check(P, data, offs, 4, lut, base, "70000 records", expect_direct=-1)
