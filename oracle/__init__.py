"""CPU oracle for the DNA byte -> token-ID path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it
and shares no code with it.

``dnatok_oracle.c`` is the plain single-threaded statement of the method
(record split, byte classes, single-nucleotide / k-mer / BPE / overlapping
and table-driven k-mer tokenization, offsets, the BPE trainer, decoders and
the reverse complement); ``feed`` below is the fixed-shape model feed in
plain numpy; ``literal.py`` holds even simpler
pure-Python definitions used to brute-force check the C oracle on tiny
inputs.  The conventions the paper leaves open (C1-C18) are listed at the
top of ``dnatok_oracle.c``; C19 (the feed) is stated at ``feed``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dnatok_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

CHAR, KMER, BPE, KMER_OVERLAP, KMER_TABLE = 0, 1, 2, 3, 4
RAW, FASTA = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library (gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64, i32, cint = ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        lib.oracle_encode.argtypes = [cint, cint, i32p, i32p, i32, cint, u8p, i64, i64p, i64,
                                      i32p, i64, i64p, i64, i64p, i64p]
        lib.oracle_encode.restype = cint
        lib.oracle_bpe_word.argtypes = [i32p, i32, i32p, i64, i32p]
        lib.oracle_bpe_word.restype = i64
        lib.oracle_bpe_train.argtypes = [u8p, i64, i32, i32p]
        lib.oracle_bpe_train.restype = i32
        lib.oracle_decode.argtypes = [cint, cint, i32p, i32, i32p, i64, ctypes.c_char_p, i64]
        lib.oracle_decode.restype = i64
        lib.oracle_default_lut.argtypes = [i32p]
        lib.oracle_default_lut.restype = None
        lib.oracle_encode_ktab.argtypes = [cint, i32p, i32p, cint, u8p, i64, i64p, i64, i32p,
                                           i64, i64p, i64, i64p, i64p]
        lib.oracle_encode_ktab.restype = cint
        lib.oracle_revcomp.argtypes = [u8p, i64, i64p, i64, u8p]
        lib.oracle_revcomp.restype = cint
        lib.oracle_decode_lut.argtypes = [i32p, i32p, i64, ctypes.c_char_p, i64]
        lib.oracle_decode_lut.restype = i64
        lib.oracle_decode_ktab.argtypes = [cint, i32p, i32p, i32p, i64, ctypes.c_char_p, i64]
        lib.oracle_decode_ktab.restype = i64
        _lib = lib
    return _lib


def _p(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _merges_array(merges):
    if merges is None:
        return np.zeros((0, 2), dtype=np.int32)
    return np.ascontiguousarray(np.asarray(merges, dtype=np.int32).reshape(-1, 2))


def default_lut() -> np.ndarray:
    lut = np.empty(256, dtype=np.int32)
    _load().oracle_default_lut(_p(lut, ctypes.c_int32))
    return lut


def encode(data, mode: int, k: int = 1, seq_offsets=None, fmt: int = RAW, lut=None,
           merges=None, ids_capacity: int | None = None):
    """Tokenize ``data`` (bytes or uint8 array).  RAW: ``seq_offsets`` gives
    the records (default: one record).  Returns (ids int32, offsets int64)."""
    if isinstance(data, (bytes, bytearray)):
        data = np.frombuffer(bytes(data), dtype=np.uint8)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    n = data.size
    if fmt == RAW:
        if seq_offsets is None:
            seq_offsets = np.array([0, n], dtype=np.int64)
        seq_offsets = np.ascontiguousarray(seq_offsets, dtype=np.int64)
        n_seq = seq_offsets.size - 1
        offs_cap = n_seq + 1
    else:
        seq_offsets = None
        n_seq = 0
        offs_cap = n + 2
    m = _merges_array(merges)
    if lut is not None:
        lut = np.ascontiguousarray(lut, dtype=np.int32)
        assert lut.size == 256
    cap = n if ids_capacity is None else ids_capacity
    ids = np.empty(max(cap, 1), dtype=np.int32)
    offs = np.empty(offs_cap, dtype=np.int64)
    n_ids = ctypes.c_int64(0)
    n_rec = ctypes.c_int64(0)
    st = _load().oracle_encode(mode, k, _p(lut, ctypes.c_int32), _p(m, ctypes.c_int32),
                               m.shape[0], fmt, _p(data, ctypes.c_uint8), n,
                               _p(seq_offsets, ctypes.c_int64), n_seq, _p(ids, ctypes.c_int32),
                               cap, _p(offs, ctypes.c_int64), offs_cap, ctypes.byref(n_ids),
                               ctypes.byref(n_rec))
    if st != 0:
        raise RuntimeError("oracle_encode failed with status %d" % st)
    return ids[: n_ids.value].copy(), offs[: n_rec.value + 1].copy()


def bpe_word(codes, merges) -> np.ndarray:
    codes = np.ascontiguousarray(codes, dtype=np.int32)
    m = _merges_array(merges)
    out = np.empty(max(codes.size, 1), dtype=np.int32)
    n = _load().oracle_bpe_word(_p(m, ctypes.c_int32), m.shape[0], _p(codes, ctypes.c_int32),
                                codes.size, _p(out, ctypes.c_int32))
    if n < 0:
        raise RuntimeError("oracle_bpe_word failed")
    return out[:n].copy()


def bpe_train(codes, n_merges: int) -> np.ndarray:
    """Train a merge table on one word of base codes (0..3, uint8)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.empty(2 * max(n_merges, 1), dtype=np.int32)
    r = _load().oracle_bpe_train(_p(codes, ctypes.c_uint8), codes.size, n_merges,
                                 _p(out, ctypes.c_int32))
    if r < 0:
        raise RuntimeError("oracle_bpe_train failed")
    return out[: 2 * r].reshape(-1, 2).copy()


def decode(ids, mode: int, k: int = 1, merges=None) -> bytes:
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    m = _merges_array(merges)
    cap = max(16, ids.size * 64 if mode == BPE else ids.size * max(k, 1))
    buf = ctypes.create_string_buffer(cap)
    n = _load().oracle_decode(mode, k, _p(m, ctypes.c_int32), m.shape[0],
                              _p(ids, ctypes.c_int32), ids.size, buf, cap)
    if n < 0:
        raise RuntimeError("oracle_decode failed")
    return buf.raw[:n]


def codes_of(text) -> np.ndarray:
    """Uppercase ACGT text -> base codes (A0 C1 G2 T3); input-side helper."""
    if isinstance(text, str):
        text = text.encode()
    a = np.frombuffer(bytes(text), dtype=np.uint8)
    table = np.full(256, 255, dtype=np.uint8)
    for c, v in zip(b"ACGT", range(4)):
        table[c] = v
    out = table[a]
    assert (out < 4).all(), "codes_of expects uppercase ACGT only"
    return out


def _records(data, seq_offsets):
    if isinstance(data, (bytes, bytearray)):
        data = np.frombuffer(bytes(data), dtype=np.uint8)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    if seq_offsets is None:
        seq_offsets = np.array([0, data.size], dtype=np.int64)
    return data, np.ascontiguousarray(seq_offsets, dtype=np.int64)


def encode_ktab(data, k: int, kmer_lut, base_ids, seq_offsets=None, fmt: int = RAW):
    """Table-driven k-mers (reading C16).  Returns (ids int32, offsets int64)."""
    data, so = _records(data, seq_offsets)
    n = data.size
    kl = np.ascontiguousarray(kmer_lut, dtype=np.int32)
    bi = np.ascontiguousarray(base_ids, dtype=np.int32)
    assert kl.size == 5 ** k and bi.size == 5
    if fmt == RAW:
        n_seq, offs_cap, sop = so.size - 1, so.size, _p(so, ctypes.c_int64)
    else:
        n_seq, offs_cap, sop = 0, n + 2, None
    ids = np.empty(max(n, 1), dtype=np.int32)
    offs = np.empty(offs_cap, dtype=np.int64)
    n_ids, n_rec = ctypes.c_int64(0), ctypes.c_int64(0)
    st = _load().oracle_encode_ktab(k, _p(kl, ctypes.c_int32), _p(bi, ctypes.c_int32), fmt,
                                    _p(data, ctypes.c_uint8), n, sop, n_seq,
                                    _p(ids, ctypes.c_int32), n, _p(offs, ctypes.c_int64),
                                    offs_cap, ctypes.byref(n_ids), ctypes.byref(n_rec))
    if st != 0:
        raise RuntimeError("oracle_encode_ktab failed with status %d" % st)
    return ids[: n_ids.value].copy(), offs[: n_rec.value + 1].copy()


def revcomp(data, seq_offsets=None) -> np.ndarray:
    """Reverse complement of every record (reading C18)."""
    data, so = _records(data, seq_offsets)
    out = np.empty(max(data.size, 1), dtype=np.uint8)
    st = _load().oracle_revcomp(_p(data, ctypes.c_uint8), data.size, _p(so, ctypes.c_int64),
                                so.size - 1, _p(out, ctypes.c_uint8))
    if st != 0:
        raise RuntimeError("oracle_revcomp failed with status %d" % st)
    return out[: data.size].copy()


def decode_lut(ids, lut) -> bytes:
    """Single-nucleotide ids through the inverse of ``lut`` (reading C17)."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    lut = np.ascontiguousarray(lut, dtype=np.int32)
    buf = ctypes.create_string_buffer(max(ids.size, 1))
    n = _load().oracle_decode_lut(_p(lut, ctypes.c_int32), _p(ids, ctypes.c_int32), ids.size,
                                  buf, ids.size)
    if n < 0:
        raise RuntimeError("oracle_decode_lut: an id has no inverse")
    return buf.raw[:n]


def decode_ktab(ids, k: int, kmer_lut, base_ids) -> bytes:
    """Table-driven k-mer ids back to text (reading C17)."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    kl = np.ascontiguousarray(kmer_lut, dtype=np.int32)
    bi = np.ascontiguousarray(base_ids, dtype=np.int32)
    cap = max(ids.size * k, 1)
    buf = ctypes.create_string_buffer(cap)
    n = _load().oracle_decode_ktab(k, _p(kl, ctypes.c_int32), _p(bi, ctypes.c_int32),
                                   _p(ids, ctypes.c_int32), ids.size, buf, cap)
    if n < 0:
        raise RuntimeError("oracle_decode_ktab: an id has no inverse")
    return buf.raw[:n]


def feed(ids, id_offsets, token_len: int, id_pad: int, row_begin: int = 0, n_rows=None,
         dtype=np.int64) -> np.ndarray:
    """Fixed-shape model feed (reading C19 of Algorithm 2's left padding):
    row i holds record row_begin + i; a record of m <= token_len tokens is
    right-aligned after token_len - m copies of id_pad; a longer record keeps
    its first token_len tokens.  Plain per-row loop."""
    ids = np.asarray(ids)
    offs = np.asarray(id_offsets, dtype=np.int64)
    if n_rows is None:
        n_rows = offs.size - 1 - row_begin
    out = np.empty((n_rows, token_len), dtype=dtype)
    for i in range(n_rows):
        r = row_begin + i
        toks = ids[offs[r]:offs[r + 1]][:token_len]
        pad = token_len - toks.size
        out[i, :pad] = id_pad
        out[i, pad:] = toks
    return out
