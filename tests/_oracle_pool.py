"""The oracle over record ranges of the full-size workloads, in worker
processes (started with ``spawn``, so they inherit no CUDA state).  Each
worker regenerates its records from the seeded generators (every record is
seeded by its own index, so a range equals that slice of the whole input)
and returns the oracle's ids and offsets for them; the test compares them
element by element with the GPU's output."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

BPE_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                         "bpe_merges_markov45_seed45_4096.txt")


def bpe_corpus_records(r0: int, r1: int):
    """Records r0..r1-1 of the 1 GiB BPE corpus (512 x 2 Mb) through the
    oracle's BPE with the 4096-merge table."""
    import oracle
    import synth
    data, offs = synth.bpe_apply_corpus(records=(r0, r1), threads=1)
    merges = np.loadtxt(BPE_TABLE, dtype=np.int32)
    ids, o = oracle.encode(data, oracle.BPE, seq_offsets=offs, merges=merges)
    return r0, r1, ids, o


def fasta_stream_records(n_total: int, seed: int, k: int, r0: int, r1: int):
    """Records r0..r1-1 of the seeded FASTA stream through the oracle's
    k-mer tokenizer (FASTA format: the slice starts at a header)."""
    import oracle
    import synth
    data, _ = synth.fasta_stream(n_total, seed=seed, records=(r0, r1), threads=1)
    ids, o = oracle.encode(data, oracle.KMER, k=k, fmt=oracle.FASTA)
    return r0, r1, ids, o


def workers() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def run(fn, arg_tuples):
    """fn(*args) for every tuple, in spawned worker processes; yields the
    results in order."""
    with cf.ProcessPoolExecutor(min(workers(), len(arg_tuples)) or 1,
                                mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(fn, *a) for a in arg_tuples]
        for f in futs:
            yield f.result()


def compare(got_ids: np.ndarray, got_offs: np.ndarray, r0: int, want_ids, want_offs, what: str):
    """Records r0.. of the GPU output (ids, offsets of the whole input) against
    the oracle's ids and offsets of those records alone, element by element;
    raises with the first mismatch."""
    n = len(want_offs) - 1
    g0 = int(got_offs[r0])
    counts_got = np.diff(got_offs[r0:r0 + n + 1])
    counts_want = np.diff(want_offs)
    if not np.array_equal(counts_got, counts_want):
        bad = int(np.nonzero(counts_got != counts_want)[0][0])
        raise AssertionError("%s: record %d has %d ids, the oracle %d" %
                             (what, r0 + bad, counts_got[bad], counts_want[bad]))
    seg = got_ids[g0:g0 + len(want_ids)]
    if not np.array_equal(seg, want_ids):
        i = int(np.nonzero(seg != want_ids)[0][0])
        rec = r0 + int(np.searchsorted(want_offs, i, side="right")) - 1
        raise AssertionError("%s: id %d (record %d) is %d, the oracle's %d" %
                             (what, g0 + i, rec, seg[i], want_ids[i]))
