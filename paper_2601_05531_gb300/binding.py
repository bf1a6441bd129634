"""Thin ctypes binding of libdnatok.so.

Every function here has the name of the C entry point it calls and only
marshals arguments (integers are raw device / host addresses, streams are
``cudaStream_t`` values such as ``torch.cuda.Stream.cuda_stream``).  All work
happens in the CUDA library; there is no Python or CPU fallback -- if the
library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

CHAR, KMER, BPE, KMER_OVERLAP, KMER_TABLE = 0, 1, 2, 3, 4  # dnatok_mode
RAW, FASTA = 0, 1

OK, PENDING = 0, 1
STATUS_NAMES = {
    0: "OK", 1: "PENDING", -1: "ERR_ARG", -2: "ERR_TABLE", -3: "ERR_CAPACITY", -4: "ERR_CUDA",
    -5: "ERR_BUDGET", -6: "ERR_TIMEOUT", -7: "ERR_UNKNOWN_REQ", -8: "ERR_NOMEM",
    -9: "ERR_STATE", -10: "ERR_DEVICE_DATA",
}

END_OF_STREAM = 1
NEW_RECORD = 2
HOST_PINNED = 4


class DnatokError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


class StreamCfg(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_int64), ("n_slots", ctypes.c_int32),
                ("overlap", ctypes.c_int32)]


class StreamResult(ctypes.Structure):
    _fields_ = [("n_ids", ctypes.c_int64), ("n_records", ctypes.c_int64),
                ("bytes_in", ctypes.c_int64)]


class PartState(ctypes.Structure):
    """dnatok_part_state: the state at a part boundary of a split stream."""
    _fields_ = [("nb", ctypes.c_int64), ("h", ctypes.c_int64), ("d", ctypes.c_int64),
                ("t", ctypes.c_int64), ("codes", ctypes.c_uint64),
                ("line_state", ctypes.c_uint32), ("pad", ctypes.c_uint32)]

    def as_list(self):
        return [self.nb, self.h, self.d, self.t, self.codes, self.line_state]

    @classmethod
    def from_list(cls, v):
        return cls(int(v[0]), int(v[1]), int(v[2]), int(v[3]), int(v[4]) & ((1 << 64) - 1),
                   int(v[5]), 0)


class ServerCfg(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("host_arena_bytes", ctypes.c_int64),
                ("max_batch_bytes", ctypes.c_int64), ("max_batch_requests", ctypes.c_int32),
                ("n_slots", ctypes.c_int32), ("kmer_k", ctypes.c_int32),
                ("n_merges", ctypes.c_int32), ("merges", ctypes.POINTER(ctypes.c_int32))]


class ServerResult(ctypes.Structure):
    _fields_ = [("ids_d", ctypes.c_void_p), ("n_ids", ctypes.c_int64),
                ("latency_us", ctypes.c_double)]


class ServerCounters(ctypes.Structure):
    _fields_ = [("device_bytes_in_use", ctypes.c_int64), ("batches_launched", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("batches_running", ctypes.c_int64)]


class LaunchCfg(ctypes.Structure):
    _fields_ = [("tile_bytes", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("chunk_tiles", ctypes.c_int32)]


class Tables(ctypes.Structure):
    _fields_ = [("ascii_lut256", ctypes.POINTER(ctypes.c_int32)),
                ("merges", ctypes.POINTER(ctypes.c_int32)), ("n_merges", ctypes.c_int32),
                ("kmer_lut", ctypes.POINTER(ctypes.c_int32)),
                ("base_ids", ctypes.POINTER(ctypes.c_int32))]


# int consumer(void *user, int64 row_begin, int64 n_rows, void *batch_d, cudaStream_t stream)
FEED_CONSUMER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_void_p, ctypes.c_void_p)


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_ST = ctypes.c_int


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libdnatok.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libdnatok.so is not built (%s): run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        sig = {
            "dnatok_create": (_ST, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(Tables), ctypes.c_int]),
            "dnatok_destroy": (None, [_P]),
            "dnatok_max_tokens": (_ST, [_P, _I64, _I64, ctypes.POINTER(_I64)]),
            "dnatok_reserve": (_ST, [_P, _I64, _I64]),
            "dnatok_encode": (_ST, [_P, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _P]),
            "dnatok_encode_host": (_ST, [_P, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _P]),
            "dnatok_sync": (_ST, [_P, _P]),
            "dnatok_last_error": (_ST, [_P, ctypes.c_char_p, ctypes.c_size_t]),
            "dnatok_get_launch": (_ST, [_P, ctypes.POINTER(LaunchCfg)]),
            "dnatok_set_launch": (_ST, [_P, ctypes.POINTER(LaunchCfg)]),
            "dnatok_stream_open": (_ST, [_P, ctypes.POINTER(StreamCfg), _P, _I64, _P, _I64]),
            "dnatok_stream_submit": (_ST, [_P, _P, _I64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_uint64)]),
            "dnatok_stream_poll": (_ST, [_P, ctypes.c_uint64, ctypes.POINTER(StreamResult)]),
            "dnatok_stream_wait": (_ST, [_P, ctypes.c_uint64, ctypes.POINTER(StreamResult)]),
            "dnatok_stream_close": (_ST, [_P]),
            "dnatok_set_bpe_launch": (_ST, [_P, ctypes.c_int32, ctypes.c_int32]),
            "dnatok_set_direct": (_ST, [_P, ctypes.c_int32]),
            "dnatok_direct_ran": (_ST, [_P, _P, ctypes.POINTER(ctypes.c_int32)]),
            "dnatok_set_kernel_timing": (_ST, [_P, ctypes.c_int32]),
            "dnatok_kernel_time_ms": (_ST, [_P, _P, ctypes.POINTER(ctypes.c_float)]),
            "dnatok_get_bpe_launch": (_ST, [_P, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]),
            "dnatok_bpe_stats": (_ST, [_P, ctypes.POINTER(_I64), _P]),
            "dnatok_set_wait_limit": (_ST, [_P, _I64]),
            "dnatok_set_direct_launch": (_ST, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
            "dnatok_get_direct_launch": (_ST, [_P, ctypes.POINTER(ctypes.c_int32)]),
            "dnatok_inject_lookback_stall": (_ST, [_P, _I64]),
            "dnatok_graph_begin": (_ST, [_P, _P]),
            "dnatok_graph_end": (_ST, [_P, _P, ctypes.POINTER(_P)]),
            "dnatok_graph_launch": (_ST, [_P, _P]),
            "dnatok_graph_destroy": (None, [_P]),
            "dnatok_autotune": (_ST, [_P, _P, _I64, _P, _I64, _P, _I64, _P, _I64, ctypes.c_int32,
                                      ctypes.c_char_p, ctypes.POINTER(LaunchCfg),
                                      ctypes.POINTER(ctypes.c_float)]),
            "dnatok_server_create": (_ST, [ctypes.POINTER(ServerCfg), ctypes.POINTER(_P)]),
            "dnatok_server_submit": (_ST, [_P, ctypes.c_int32, _P, _I64,
                                           ctypes.POINTER(ctypes.c_uint64)]),
            "dnatok_server_poll": (_ST, [_P, ctypes.c_uint64, ctypes.POINTER(ServerResult)]),
            "dnatok_server_read": (_ST, [_P, ctypes.c_uint64, _P, _I64, ctypes.POINTER(_I64)]),
            "dnatok_server_release": (_ST, [_P, ctypes.c_uint64]),
            "dnatok_server_stats": (_ST, [_P, ctypes.POINTER(ServerCounters)]),
            "dnatok_server_inject": (_ST, [_P, ctypes.c_int32, ctypes.c_int32]),
            "dnatok_server_destroy": (None, [_P]),
            "dnatok_encode_kmer_noalloc": (_ST, [ctypes.c_int, _P, _I64, _P, _I64, _P, _I64, _P,
                                                 _I64, _P, _P]),
            "dnatok_max_decoded_bytes": (_ST, [_P, _I64, _I64, ctypes.POINTER(_I64)]),
            "dnatok_decode": (_ST, [_P, _P, _I64, _P, _I64, _P, _I64, _P, _P, _P]),
            "dnatok_reverse_complement": (_ST, [_P, _I64, _P, _I64, _P, _P]),
            "dnatok_feed": (_ST, [_P, _P, _I64, _I64, _I64, _I64, _P, ctypes.c_int32, _P]),
            "dnatok_microbatch_rows": (_ST, [_I64, _I64, _I64, ctypes.POINTER(_I64)]),
            "dnatok_shard_records": (_ST, [_P, _I64, ctypes.c_int32, _P]),
            "dnatok_feed_pipeline": (_ST, [_P, _P, _I64, _I64, _I64, ctypes.c_int32, _I64, _P, _P,
                                           _P, _P, FEED_CONSUMER, _P]),
            "dnatok_part_line_map": (_ST, [_P, _P, _I64, ctypes.POINTER(ctypes.c_int32), _P]),
            "dnatok_part_encode": (_ST, [_P, _P, _I64, ctypes.POINTER(PartState), ctypes.c_int32,
                                         _P, _I64, _P, _I64, ctypes.POINTER(PartState), _P]),
            "dnatok_part_combine": (_ST, [ctypes.c_int32, ctypes.POINTER(PartState),
                                          ctypes.POINTER(PartState), ctypes.POINTER(PartState)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error(h) -> str:
    buf = ctypes.create_string_buffer(512)
    lib().dnatok_last_error(h, buf, 512)
    return buf.value.decode(errors="replace")


def check(st: int, h=None) -> int:
    if st < 0:
        raise DnatokError(st, last_error(h))
    return st


# ------------------------------------------------------------------ wrappers

def dnatok_create(mode: int, k: int = 1, lut=None, merges=None, fmt: int = RAW, kmer_lut=None,
                  base_ids=None):
    """Returns the handle (an opaque address).  lut: 256 ints or None;
    merges: (M, 2) ints or None; kmer_lut (5^k ints) and base_ids (5 ints):
    KMER_TABLE only."""
    import numpy as np
    t = Tables()
    keep = []
    for name, arr in (("kmer_lut", kmer_lut), ("base_ids", base_ids)):
        if arr is not None:
            a = np.ascontiguousarray(np.asarray(arr, dtype=np.int32).reshape(-1))
            keep.append(a)
            setattr(t, name, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if lut is not None:
        a = np.ascontiguousarray(np.asarray(lut, dtype=np.int32).reshape(256))
        keep.append(a)
        t.ascii_lut256 = a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    if merges is not None:
        m = np.ascontiguousarray(np.asarray(merges, dtype=np.int32).reshape(-1, 2))
        keep.append(m)
        t.merges = m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        t.n_merges = m.shape[0]
    h = _P()
    check(lib().dnatok_create(ctypes.byref(h), mode, k, ctypes.byref(t), fmt), None)
    return h.value


def dnatok_destroy(h) -> None:
    lib().dnatok_destroy(h)


def dnatok_max_tokens(h, n_bytes: int, n_seq: int) -> int:
    c = _I64()
    check(lib().dnatok_max_tokens(h, n_bytes, n_seq, ctypes.byref(c)), h)
    return c.value


def dnatok_reserve(h, max_bytes: int, max_seq: int) -> None:
    check(lib().dnatok_reserve(h, max_bytes, max_seq), h)


def dnatok_encode(h, bytes_d: int, n_bytes: int, seq_offsets_d: int, n_seq: int, ids_out_d: int,
                  ids_capacity: int, id_offsets_d: int, offsets_capacity: int, totals_d: int,
                  stream: int) -> int:
    return check(lib().dnatok_encode(h, bytes_d, n_bytes, seq_offsets_d, n_seq, ids_out_d,
                                     ids_capacity, id_offsets_d, offsets_capacity, totals_d,
                                     stream), h)


def dnatok_encode_host(h, host_bytes: int, n_bytes: int, host_seq_offsets: int, n_seq: int,
                       ids_out_d: int, ids_capacity: int, id_offsets_host: int,
                       offsets_capacity: int, totals_host: int, stream: int) -> int:
    return check(lib().dnatok_encode_host(h, host_bytes, n_bytes, host_seq_offsets, n_seq,
                                          ids_out_d, ids_capacity, id_offsets_host,
                                          offsets_capacity, totals_host, stream), h)


def dnatok_sync(h, stream: int) -> int:
    return check(lib().dnatok_sync(h, stream), h)


def dnatok_last_error(h) -> str:
    return last_error(h)


def dnatok_get_launch(h) -> tuple:
    c = LaunchCfg()
    check(lib().dnatok_get_launch(h, ctypes.byref(c)), h)
    return (c.tile_bytes, c.threads, c.ctas_per_sm, c.chunk_tiles)


def dnatok_set_launch(h, tile_bytes: int, threads: int, ctas_per_sm: int,
                      chunk_tiles: int = 4) -> None:
    c = LaunchCfg(tile_bytes, threads, ctas_per_sm, chunk_tiles)
    check(lib().dnatok_set_launch(h, ctypes.byref(c)), h)


def dnatok_stream_open(h, ids_out_d: int, ids_capacity: int, id_offsets_d: int,
                       offsets_capacity: int, chunk_bytes: int = 0, n_slots: int = 0,
                       overlap: int = 1) -> None:
    c = StreamCfg(chunk_bytes, n_slots, overlap)
    check(lib().dnatok_stream_open(h, ctypes.byref(c), ids_out_d, ids_capacity, id_offsets_d,
                                   offsets_capacity), h)


def dnatok_stream_submit(h, host_bytes: int, n: int, flags: int = 0) -> int:
    r = ctypes.c_uint64()
    check(lib().dnatok_stream_submit(h, host_bytes, n, flags, ctypes.byref(r)), h)
    return r.value


def dnatok_stream_poll(h, req_id: int):
    """None while pending, else (n_ids, n_records, bytes_in)."""
    out = StreamResult()
    st = check(lib().dnatok_stream_poll(h, req_id, ctypes.byref(out)), h)
    if st == 1:
        return None
    return (out.n_ids, out.n_records, out.bytes_in)


def dnatok_stream_wait(h, req_id: int):
    out = StreamResult()
    check(lib().dnatok_stream_wait(h, req_id, ctypes.byref(out)), h)
    return (out.n_ids, out.n_records, out.bytes_in)


def dnatok_stream_close(h) -> None:
    check(lib().dnatok_stream_close(h), h)


def dnatok_set_direct(h, enable: bool) -> None:
    check(lib().dnatok_set_direct(h, int(bool(enable))), h)


def dnatok_direct_ran(h, stream=0) -> int:
    out = ctypes.c_int32(0)
    check(lib().dnatok_direct_ran(h, stream, ctypes.byref(out)), h)
    return out.value


def dnatok_set_kernel_timing(h, enable: bool) -> None:
    check(lib().dnatok_set_kernel_timing(h, int(bool(enable))), h)


def dnatok_kernel_time_ms(h, stream=0) -> float:
    out = ctypes.c_float(0.0)
    check(lib().dnatok_kernel_time_ms(h, stream, ctypes.byref(out)), h)
    return out.value


def dnatok_set_bpe_launch(h, seg_symbols: int, halo: int) -> None:
    check(lib().dnatok_set_bpe_launch(h, seg_symbols, halo), h)


def dnatok_get_bpe_launch(h) -> tuple:
    a, b = ctypes.c_int32(), ctypes.c_int32()
    check(lib().dnatok_get_bpe_launch(h, ctypes.byref(a), ctypes.byref(b)), h)
    return (a.value, b.value)


def dnatok_set_direct_launch(h, slots_per_step: int, ring_steps: int, ctas_per_sm: int = 0) -> None:
    check(lib().dnatok_set_direct_launch(h, slots_per_step, ring_steps, ctas_per_sm), h)


def dnatok_get_direct_launch(h) -> tuple:
    v = (ctypes.c_int32 * 3)()
    check(lib().dnatok_get_direct_launch(h, v), h)
    return (v[0], v[1], v[2])


def dnatok_set_wait_limit(h, polls: int) -> None:
    check(lib().dnatok_set_wait_limit(h, polls), h)


def dnatok_inject_lookback_stall(h, chunk: int) -> None:
    check(lib().dnatok_inject_lookback_stall(h, chunk), h)


def dnatok_bpe_stats(h, stream: int = 0) -> dict:
    v = (_I64 * 3)()
    check(lib().dnatok_bpe_stats(h, v, stream), h)
    return {"symbols": v[0], "segments": v[1], "repaired_segments": v[2]}


def dnatok_graph_begin(h, stream: int) -> None:
    check(lib().dnatok_graph_begin(h, stream), h)


def dnatok_graph_end(h, stream: int) -> int:
    g = _P()
    check(lib().dnatok_graph_end(h, stream, ctypes.byref(g)), h)
    return g.value


def dnatok_graph_launch(g, stream: int) -> None:
    check(lib().dnatok_graph_launch(g, stream))


def dnatok_graph_destroy(g) -> None:
    lib().dnatok_graph_destroy(g)


def dnatok_autotune(h, bytes_d: int, n_bytes: int, seq_offsets_d: int, n_seq: int,
                    ids_out_d: int, ids_capacity: int, id_offsets_d: int, offsets_capacity: int,
                    reps: int = 5, cache_path: str | None = None):
    """Returns ((tile, threads, ctas_per_sm, chunk_tiles) or BPE (seg, halo, 0, 0), ms)."""
    c = LaunchCfg()
    ms = ctypes.c_float()
    check(lib().dnatok_autotune(h, bytes_d, n_bytes, seq_offsets_d, n_seq, ids_out_d,
                                ids_capacity, id_offsets_d, offsets_capacity, reps,
                                cache_path.encode() if cache_path else None, ctypes.byref(c),
                                ctypes.byref(ms)), h)
    return (c.tile_bytes, c.threads, c.ctas_per_sm, c.chunk_tiles), ms.value


def dnatok_server_create(budget_bytes: int = 4 << 30, host_arena_bytes: int = 1 << 30,
                         max_batch_bytes: int = 32 << 20, max_batch_requests: int = 256,
                         n_slots: int = 4, kmer_k: int = 6, merges=None):
    """Returns (server address, keep-alive objects)."""
    import numpy as np
    m = None
    c = ServerCfg(budget_bytes, host_arena_bytes, max_batch_bytes, max_batch_requests, n_slots,
                  kmer_k, 0, None)
    if merges is not None:
        m = np.ascontiguousarray(np.asarray(merges, dtype=np.int32).reshape(-1, 2))
        c.n_merges = m.shape[0]
        c.merges = m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    srv = _P()
    st = lib().dnatok_server_create(ctypes.byref(c), ctypes.byref(srv))
    if st < 0:
        raise DnatokError(st, "dnatok_server_create: " + last_error(None))
    return srv.value


def dnatok_server_submit(srv, mode: int, host_bytes: int, n: int) -> int:
    """Request id, or None when the staging arena is full (retry later)."""
    r = ctypes.c_uint64()
    st = lib().dnatok_server_submit(srv, mode, host_bytes, n, ctypes.byref(r))
    if st == -5:
        return None
    if st < 0:
        raise DnatokError(st, "dnatok_server_submit")
    return r.value


def dnatok_server_poll(srv, req_id: int):
    """None while pending, else (ids device address, n_ids, latency_us)."""
    out = ServerResult()
    st = lib().dnatok_server_poll(srv, req_id, ctypes.byref(out))
    if st == 1:
        return None
    if st < 0:
        raise DnatokError(st, "dnatok_server_poll")
    return (out.ids_d or 0, out.n_ids, out.latency_us)


def dnatok_server_read(srv, req_id: int, n_ids: int):
    """The request's ids as a numpy int32 array (the request must be done)."""
    import numpy as np
    out = np.empty(max(n_ids, 1), dtype=np.int32)
    n = _I64()
    st = lib().dnatok_server_read(srv, req_id, out.ctypes.data, n_ids, ctypes.byref(n))
    if st < 0:
        raise DnatokError(st, "dnatok_server_read")
    return out[:n.value]


def dnatok_server_release(srv, req_id: int) -> None:
    st = lib().dnatok_server_release(srv, req_id)
    if st < 0:
        raise DnatokError(st, "dnatok_server_release")


def dnatok_server_stats(srv) -> dict:
    c = ServerCounters()
    check(lib().dnatok_server_stats(srv, ctypes.byref(c)))
    return {k: getattr(c, k) for k, _ in ServerCounters._fields_}


def dnatok_server_inject(srv, kind: int, count: int = 1) -> None:
    check(lib().dnatok_server_inject(srv, kind, count))


def dnatok_server_destroy(srv) -> None:
    lib().dnatok_server_destroy(srv)


NOALLOC_MAX_BYTES = 1 << 30  # DNATOK_NOALLOC_MAX_BYTES


def dnatok_encode_kmer_noalloc(k: int, bytes_d: int, n_bytes: int, seq_offsets_d: int,
                               n_seq: int, ids_out_d: int, ids_capacity: int, id_offsets_d: int,
                               offsets_capacity: int, totals_d: int, stream: int) -> int:
    """The k-mer encode that allocates nothing (all pointers are device
    addresses the caller owns).  totals read {-1, -1} after a device-side
    error; inputs above NOALLOC_MAX_BYTES raise DnatokError(CAPACITY)."""
    st = lib().dnatok_encode_kmer_noalloc(k, bytes_d, n_bytes, seq_offsets_d, n_seq, ids_out_d,
                                          ids_capacity, id_offsets_d, offsets_capacity, totals_d,
                                          stream)
    if st < 0:
        why = {-1: "bad argument", -3: "n_bytes above %d or an output buffer too small"
               % NOALLOC_MAX_BYTES, -4: "CUDA call failed"}.get(st, "error")
        raise DnatokError(st, "dnatok_encode_kmer_noalloc: " + why)
    return st


def dnatok_max_decoded_bytes(h, n_ids: int, n_seq: int) -> int:
    c = _I64()
    check(lib().dnatok_max_decoded_bytes(h, n_ids, n_seq, ctypes.byref(c)), h)
    return c.value


def dnatok_decode(h, ids_d: int, n_ids: int, id_offsets_d: int, n_seq: int, bytes_out_d: int,
                  bytes_capacity: int, byte_offsets_d: int, totals_d: int, stream: int) -> int:
    return check(lib().dnatok_decode(h, ids_d, n_ids, id_offsets_d, n_seq, bytes_out_d,
                                     bytes_capacity, byte_offsets_d, totals_d, stream), h)


def dnatok_reverse_complement(bytes_d: int, n_bytes: int, seq_offsets_d: int, n_seq: int,
                              out_d: int, stream: int) -> int:
    return check(lib().dnatok_reverse_complement(bytes_d, n_bytes, seq_offsets_d, n_seq, out_d,
                                                 stream))


def dnatok_feed(ids_d: int, id_offsets_d: int, row_begin: int, n_rows: int, token_len: int,
                id_pad: int, out_d: int, out_bytes: int, stream: int) -> int:
    return check(lib().dnatok_feed(ids_d, id_offsets_d, row_begin, n_rows, token_len, id_pad,
                                   out_d, out_bytes, stream))


def dnatok_microbatch_rows(emb_batch_cap: int, tokens_per_call: int, token_len: int) -> int:
    r = _I64()
    check(lib().dnatok_microbatch_rows(emb_batch_cap, tokens_per_call, token_len,
                                       ctypes.byref(r)))
    return r.value


def dnatok_feed_pipeline(ids_d: int, id_offsets_d: int, n_rows: int, token_len: int, id_pad: int,
                         out_bytes: int, rows_per_batch: int, buf0_d: int, buf1_d: int,
                         feed_stream: int, consumer_stream: int, consumer) -> int:
    """consumer(row_begin, n_rows, batch_address, consumer_stream) -> None;
    an exception stops the pipeline (ERR_STATE)."""
    def _cb(user, row_begin, n, batch, stream):
        try:
            consumer(int(row_begin), int(n), int(batch or 0), int(stream or 0))
            return 0
        except Exception:  # reported as ERR_STATE by the library
            return 1
    cb = FEED_CONSUMER(_cb)
    return check(lib().dnatok_feed_pipeline(ids_d, id_offsets_d, n_rows, token_len, id_pad,
                                            out_bytes, rows_per_batch, buf0_d, buf1_d,
                                            feed_stream, consumer_stream, cb, None))


def dnatok_shard_records(seq_offsets, world_size: int):
    """seq_offsets: n_seq + 1 host int64 (numpy-compatible).  Returns the
    world_size + 1 record bounds as a numpy int64 array."""
    import numpy as np
    so = np.ascontiguousarray(seq_offsets, dtype=np.int64)
    out = np.empty(world_size + 1, dtype=np.int64)
    check(lib().dnatok_shard_records(so.ctypes.data, so.size - 1, world_size, out.ctypes.data))
    return out


def dnatok_part_line_map(h, bytes_d: int, n: int, stream=0) -> int:
    out = ctypes.c_int32(0)
    check(lib().dnatok_part_line_map(h, bytes_d, n, ctypes.byref(out), stream), h)
    return out.value


def dnatok_part_encode(h, bytes_d: int, n: int, before, last: bool, ids_out_d: int,
                       ids_capacity: int, id_offsets_d: int, offsets_capacity: int,
                       stream=0) -> PartState:
    """before: a PartState, or None when the part starts the stream."""
    after = PartState()
    check(lib().dnatok_part_encode(h, bytes_d, n, ctypes.byref(before) if before is not None else None,
                                   int(bool(last)), ids_out_d, ids_capacity, id_offsets_d,
                                   offsets_capacity, ctypes.byref(after), stream), h)
    return after


def dnatok_part_combine(k: int, a: PartState, b: PartState) -> PartState:
    out = PartState()
    check(lib().dnatok_part_combine(k, ctypes.byref(a), ctypes.byref(b), ctypes.byref(out)))
    return out
