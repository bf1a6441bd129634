"""Seeded synthetic inputs for the DNA byte -> token-ID path.

This module only produces input bytes and their layout (sequence offsets,
FASTA record positions, request arrival schedules).  It holds none of the
tokenizer's arithmetic, so both the CPU oracle tests and the CUDA-path tests
can draw from it.

The recipes (all seeded, all synthetic):

* order-3 Markov DNA: for each of the 64 contexts the next-base distribution
  is drawn from Dirichlet(alpha * pi), pi = ((1-g)/2, g/2, g/2, (1-g)/2) for
  A, C, G, T and alpha = 20; the C/G weights are then tilted so that the
  stationary GC fraction equals g;
* N runs: run lengths uniform in 1..50, start rate set for ~1% N overall;
* soft-masking: lowercase stretches with log-uniform lengths in 10..1000,
  start rate set for ~5% coverage;
* FASTA: '>' header lines of 20..80 printable characters, sequence lines
  wrapped at 60 or 80 (coin flip per record), record lengths log-uniform in
  10 kb..10 Mb.

The heavy loops run in ``synth.c`` (splitmix64 streams keyed by seed and
sequence index, so the bytes do not depend on the thread count).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_libsynth.so")
_lib = None

N_FRACTION = 0.01
N_RUN = (1, 50)
LOWER_FRACTION = 0.05
LOWER_LEN = (10, 1000)


def build(force: bool = False) -> str:
    """Compile synth.c into an in-tree shared library (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64, u32, u64, cint = ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        lib.synth_iid_sequence.argtypes = [u8p, i64, u32, cint, cint, u32, u64]
        lib.synth_markov_batch.argtypes = [u8p, i64p, i64, u32p, u32, cint, cint, u32, i32p,
                                           u64, cint, i64, i64]
        lib.synth_fasta.argtypes = [u8p, i64, i64, i64p, i32p, i32p, i64p, u32p, u32, cint,
                                    cint, u32, i32p, u64, cint, i64, i64]
        lib.synth_random_bytes.argtypes = [u8p, i64, u64]
        for f in (lib.synth_iid_sequence, lib.synth_markov_batch, lib.synth_fasta,
                  lib.synth_random_bytes):
            f.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _threads() -> int:
    try:
        return max(1, min(64, len(os.sched_getaffinity(0))))
    except AttributeError:  # pragma: no cover
        return max(1, min(64, os.cpu_count() or 1))


def _p32(p: float) -> int:
    return int(min(max(p, 0.0), 1.0) * 4294967295.0)


def _run_start_p(fraction: float, mean_len: float) -> float:
    # A start check either consumes one position (no start) or a whole run.
    return fraction / (mean_len * (1.0 - fraction) + fraction)


def _lower_len_table() -> np.ndarray:
    lo, hi = LOWER_LEN
    q = (np.arange(4096) + 0.5) / 4096.0
    return np.floor(np.exp(math.log(lo) + q * (math.log(hi) - math.log(lo)))).astype(np.int32)


_LOWER_MEAN = (LOWER_LEN[1] - LOWER_LEN[0]) / math.log(LOWER_LEN[1] / LOWER_LEN[0])
_NRUN_P = _p32(_run_start_p(N_FRACTION, (N_RUN[0] + N_RUN[1]) / 2.0))
_LOWER_P = _p32(_run_start_p(LOWER_FRACTION, _LOWER_MEAN))


# ----------------------------------------------------------------- Markov model

def _stationary_gc(q: np.ndarray) -> float:
    trans = np.zeros((64, 64))
    for ctx in range(64):
        for b in range(4):
            trans[ctx, ((ctx << 2) | b) & 63] += q[ctx, b]
    p = np.full(64, 1.0 / 64)
    for _ in range(3000):
        p = p @ trans
    last = np.arange(64) & 3
    return float(p[(last == 1) | (last == 2)].sum())


def markov_model(gc: float, seed: int, alpha: float = 20.0):
    """Return (probabilities [64,4], cdf thresholds uint32 [64,3], achieved GC)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pi = np.array([(1 - gc) / 2, gc / 2, gc / 2, (1 - gc) / 2])
    base = rng.dirichlet(alpha * pi, size=64)

    def tilt(lam):
        q = base * np.array([1.0, lam, lam, 1.0])
        return q / q.sum(axis=1, keepdims=True)

    lo, hi = 0.05, 20.0
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        if _stationary_gc(tilt(mid)) < gc:
            lo = mid
        else:
            hi = mid
    q = tilt(math.sqrt(lo * hi))
    cum = np.cumsum(q, axis=1)[:, :3]
    cdf = np.minimum(np.floor(cum * 4294967296.0), 4294967295.0).astype(np.uint32)
    return q, np.ascontiguousarray(cdf), _stationary_gc(q)


# ------------------------------------------------------------------ generators

def iid_sequence(n: int, seed: int, n_fraction: float = N_FRACTION,
                 lower_fraction: float = 0.05) -> np.ndarray:
    """i.i.d. uppercase ACGT (p = 1/4 each), N runs of 1..50 covering
    ~n_fraction, then each byte lowercased independently with probability
    lower_fraction."""
    out = np.empty(n, dtype=np.uint8)
    nrun_p = _p32(_run_start_p(n_fraction, (N_RUN[0] + N_RUN[1]) / 2.0)) if n_fraction > 0 else 0
    _load().synth_iid_sequence(_ptr(out, ctypes.c_uint8), n, nrun_p, N_RUN[0], N_RUN[1],
                               _p32(lower_fraction), seed)
    return out


def markov_batch(lengths, gc: float, seed: int, n_runs: bool = True, soft_mask: bool = True,
                 model_seed: int | None = None, out: np.ndarray | None = None,
                 records: tuple | None = None, threads: int | None = None):
    """Back-to-back Markov sequences.  Returns (bytes uint8, offsets int64[n+1]).
    ``records=(r0, r1)`` writes only sequences r0..r1-1 (the same bytes as
    that slice of the whole batch, each sequence seeded by its index) and
    returns them with their offsets rebased to 0."""
    lengths = np.asarray(lengths, dtype=np.int64)
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    r0, r1 = (0, len(lengths)) if records is None else (int(records[0]), int(records[1]))
    assert 0 <= r0 <= r1 <= len(lengths)
    total = int(offsets[r1] - offsets[r0])
    if out is None:
        out = np.empty(max(total, 1), dtype=np.uint8)
    assert out.size >= total and out.dtype == np.uint8
    _, cdf, _ = markov_model(gc, seed if model_seed is None else model_seed)
    table = _lower_len_table()
    _load().synth_markov_batch(_ptr(out, ctypes.c_uint8), _ptr(offsets, ctypes.c_int64),
                               len(lengths), _ptr(cdf, ctypes.c_uint32),
                               _NRUN_P if n_runs else 0, N_RUN[0], N_RUN[1],
                               _LOWER_P if soft_mask else 0, _ptr(table, ctypes.c_int32),
                               seed, threads or _threads(), r0, r1)
    if records is not None:
        return out[:total], offsets[r0:r1 + 1] - offsets[r0]
    return out[:total], offsets


def log_uniform_lengths(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(n)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def random_bytes(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint8)
    _load().synth_random_bytes(_ptr(out, ctypes.c_uint8), n, seed)
    return out


def kmer_vocab(k: int, seed: int, n_specials: int = 5):
    """A vocabulary laid out like a blocked k-mer model's: every k-mer of
    A/C/G/T gets its own id (a seeded permutation after ``n_specials``
    special ids), windows holding the fifth digit (N) have no entry (-1), and
    the five single symbols A C G T N get the ids after the k-mers.  Returns
    (kmer_lut over the 5^k base-5 window indices, base_ids[5]).  Input data
    only: which windows hold the digit 4 is read off their base-5 index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.arange(5 ** k)
    has_n = np.zeros(5 ** k, dtype=bool)
    x = idx.copy()
    for _ in range(k):
        has_n |= (x % 5) == 4
        x //= 5
    lut = np.full(5 ** k, -1, dtype=np.int32)
    n_free = int((~has_n).sum())
    lut[~has_n] = (rng.permutation(n_free) + n_specials).astype(np.int32)
    base = np.arange(5, dtype=np.int32) + n_specials + n_free
    return lut, base


# ------------------------------------------------------------- named workloads

def single_sequence_1mb(seed: int = 43, n: int = 1_000_000):
    """One 1 MB sequence: i.i.d. ACGT, 1% N in runs of 1..50, 5% lowercase
    per byte.  Returns (bytes, offsets=[0, n])."""
    b = iid_sequence(n, seed)
    return b, np.array([0, n], dtype=np.int64)


def kmer_batch_4096(seed: int = 44, n_seq: int = 4096, lo: int = 1000, hi: int = 128000,
                    uniform: bool = False):
    """4096 sequences, lengths log-uniform in [1 kb, 128 kb] (uniform if
    ``uniform``), order-3 Markov at 40% GC with N runs and soft-masked
    stretches."""
    if uniform:
        rng = np.random.Generator(np.random.PCG64(seed))
        lengths = rng.integers(lo, hi + 1, size=n_seq).astype(np.int64)
    else:
        lengths = log_uniform_lengths(n_seq, lo, hi, seed)
    return markov_batch(lengths, 0.40, seed)


def bpe_training_corpus(seed: int = 45, n: int = 10_000_000) -> np.ndarray:
    """One uppercase ACGT Markov sequence at 45% GC (the BPE trainer input)."""
    b, _ = markov_batch([n], 0.45, seed, n_runs=False, soft_mask=False)
    return b


def bpe_apply_corpus(seed: int = 46, n_seq: int = 512, length: int = 2_097_152,
                     model_seed: int = 45, records: tuple | None = None,
                     threads: int | None = None):
    """512 sequences of 2 Mb, uppercase ACGT, drawn from the same Markov
    model as the trainer corpus (model parameters from ``model_seed``) with a
    fresh chain seed.  ``records=(r0, r1)``: only those sequences."""
    return markov_batch([length] * n_seq, 0.45, seed, n_runs=False, soft_mask=False,
                        model_seed=model_seed, records=records, threads=threads)


@dataclass
class FastaLayout:
    rec_off: np.ndarray     # byte offset of each record's '>'
    hdr_len: np.ndarray     # header characters including '>'
    wrap: np.ndarray        # line width
    seq_len: np.ndarray     # bases per record (the last record may be cut short)
    n_total: int


def fasta_layout(n_total: int, seed: int, rec_lo: float = 10_000, rec_hi: float = 10_000_000,
                 hdr_lo: int = 20, hdr_hi: int = 80) -> FastaLayout:
    rng = np.random.Generator(np.random.PCG64(seed))
    offs, hdrs, wraps, lens = [], [], [], []
    pos = 0
    while pos < n_total:
        sl = int(math.exp(math.log(rec_lo) + rng.random() * (math.log(rec_hi) - math.log(rec_lo))))
        hl = int(rng.integers(hdr_lo, hdr_hi + 1))
        wr = 60 if rng.random() < 0.5 else 80
        size = hl + 1 + sl + (sl + wr - 1) // wr
        offs.append(pos); hdrs.append(hl); wraps.append(wr); lens.append(sl)
        pos += size
    return FastaLayout(np.array(offs, dtype=np.int64), np.array(hdrs, dtype=np.int32),
                       np.array(wraps, dtype=np.int32), np.array(lens, dtype=np.int64), n_total)


def fasta_stream(n_total: int, seed: int = 47, out: np.ndarray | None = None,
                 records: tuple | None = None, threads: int | None = None, **layout_kw):
    """FASTA text of exactly n_total bytes (the last record is cut at the
    end), Markov 40% GC with N runs and soft-masked stretches.  ``out`` may
    be a pinned host buffer.  Returns (bytes, layout).  ``records=(r0, r1)``
    writes only records r0..r1-1 (the same bytes as that slice of the whole
    stream, each record seeded by its index)."""
    lay = fasta_layout(n_total, seed, **layout_kw)
    n_rec = len(lay.rec_off)
    r0, r1 = (0, n_rec) if records is None else (int(records[0]), int(records[1]))
    assert 0 <= r0 <= r1 <= n_rec
    starts = np.append(lay.rec_off, n_total)
    size = int(starts[r1] - starts[r0])
    if out is None:
        out = np.empty(max(size, 1), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size >= size
    _, cdf, _ = markov_model(0.40, seed)
    table = _lower_len_table()
    _load().synth_fasta(_ptr(out, ctypes.c_uint8), n_total, n_rec,
                        _ptr(lay.rec_off, ctypes.c_int64), _ptr(lay.hdr_len, ctypes.c_int32),
                        _ptr(lay.wrap, ctypes.c_int32), _ptr(lay.seq_len, ctypes.c_int64),
                        _ptr(cdf, ctypes.c_uint32), _NRUN_P, N_RUN[0], N_RUN[1], _LOWER_P,
                        _ptr(table, ctypes.c_int32), seed, threads or _threads(), r0, r1)
    return out[:size], lay


@dataclass
class RequestTrace:
    arrival_s: np.ndarray   # seconds from trace start
    sizes: np.ndarray       # bytes per request
    modes: np.ndarray       # 0 = single-nucleotide, 1 = 6-mer, 2 = BPE
    data: np.ndarray        # all payloads back to back
    offsets: np.ndarray     # payload r = data[offsets[r]:offsets[r+1]]


def request_trace(seed: int = 48, rate: float = 2000.0, duration_s: float = 10.0,
                  size_lo: float = 200, size_hi: float = 1_000_000,
                  mode_p=(0.3, 0.5, 0.2)) -> RequestTrace:
    """Poisson arrivals, log-uniform request sizes, mixed modes; payloads are
    Markov 40% GC sequences with N runs and soft-masking."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, arr = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        arr.append(t)
    n = len(arr)
    u = rng.random(n)
    sizes = np.floor(np.exp(math.log(size_lo) + u * (math.log(size_hi) - math.log(size_lo))))
    sizes = sizes.astype(np.int64)
    modes = rng.choice(3, size=n, p=np.asarray(mode_p)).astype(np.int32)
    data, offsets = markov_batch(sizes, 0.40, seed)
    return RequestTrace(np.array(arr), sizes, modes, data, offsets)


# ---------------------------------------------------------- small fuzz inputs

def fuzz_fasta(seed: int, n_records: int = 5, max_len: int = 300, crlf_p: float = 0.2,
               blank_p: float = 0.1, iupac_p: float = 0.05, lower_p: float = 0.2,
               leading_junk: bool | None = None) -> np.ndarray:
    """Small FASTA-like text with the awkward cases: CRLF line ends, blank
    lines, '>' inside sequence lines, IUPAC letters, lowercase, empty
    records, sequence bytes before the first header."""
    rng = np.random.Generator(np.random.PCG64(seed))
    alpha = np.frombuffer(b"ACGT", dtype=np.uint8)
    iupac = np.frombuffer(b"NRYKMSWBDHVnx>-.*0", dtype=np.uint8)
    parts = []

    def eol():
        return b"\r\n" if rng.random() < crlf_p else b"\n"

    if leading_junk is None:
        leading_junk = rng.random() < 0.3
    if leading_junk:
        parts.append(bytes(rng.choice(alpha, size=int(rng.integers(0, 20)))) + eol())
    for _ in range(n_records):
        hl = int(rng.integers(0, 30))
        hdr = bytes(rng.integers(32, 127, size=hl).astype(np.uint8))
        parts.append(b">" + hdr + eol())
        L = int(rng.integers(0, max_len + 1))
        seq = rng.choice(alpha, size=L)
        m = rng.random(L)
        seq = np.where(m < iupac_p, rng.choice(iupac, size=L), seq)
        low = rng.random(L) < lower_p
        seq = np.where(low & (seq >= 65) & (seq <= 90), seq + 32, seq).astype(np.uint8)
        wrap = int(rng.integers(1, 90))
        for i in range(0, L, wrap):
            parts.append(bytes(seq[i:i + wrap]) + eol())
            if rng.random() < blank_p:
                parts.append(eol())
    text = b"".join(parts)
    if text and rng.random() < 0.3:
        text = text[: int(rng.integers(0, len(text) + 1))]  # cut mid-record
    return np.frombuffer(text, dtype=np.uint8).copy()
