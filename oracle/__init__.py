"""CPU oracle for the DNA byte -> token-ID path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it
and shares no code with it.

``dnatok_oracle.c`` is the plain single-threaded statement of the method
(record split, byte classes, single-nucleotide / k-mer / BPE tokenization,
offsets, the BPE trainer and a decoder); ``literal.py`` holds even simpler
pure-Python definitions used to brute-force check the C oracle on tiny
inputs.  The conventions the paper leaves open (C1-C10) are listed at the
top of ``dnatok_oracle.c``.
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

CHAR, KMER, BPE, KMER_OVERLAP = 0, 1, 2, 3
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
