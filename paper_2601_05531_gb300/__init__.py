"""GB300-native DNA byte -> token-ID library (arXiv 2601.05531's hot path).

``binding`` mirrors the C ABI of ``libdnatok.so`` one function per entry
point.  ``Tokenizer`` below is a convenience wrapper that takes PyTorch CUDA
tensors (PyTorch supplies device memory and streams only; every step of the
tokenization runs in the library's CUDA kernels).
"""
from __future__ import annotations

from . import binding
from .binding import (BPE, CHAR, END_OF_STREAM, FASTA, HOST_PINNED, KMER, KMER_OVERLAP, KMER_TABLE,
                      NEW_RECORD, RAW, DnatokError)

__all__ = ["binding", "Tokenizer", "CHAR", "KMER", "KMER_OVERLAP", "KMER_TABLE", "BPE", "RAW", "FASTA",
           "DnatokError", "END_OF_STREAM", "NEW_RECORD", "HOST_PINNED", "build", "reverse_complement",
           "feed", "microbatch_rows", "feed_pipeline", "shard_records", "global_id_offsets"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def _stream_ptr(stream) -> int:
    """A cudaStream_t value: None -> torch's current stream, an int as it
    is (0: the legacy default stream), else the stream's handle."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Tokenizer:
    """One library handle.  mode: CHAR / KMER / KMER_OVERLAP / KMER_TABLE /
    BPE; fmt: RAW / FASTA."""

    def __init__(self, mode: int, k: int = 1, lut=None, merges=None, fmt: int = RAW,
                 kmer_lut=None, base_ids=None):
        import torch  # noqa: F401  (initializes the CUDA context the library uses)
        torch.cuda.init()
        self.mode, self.k, self.fmt = mode, k, fmt
        self.n_merges = 0 if merges is None else len(merges)
        self.h = binding.dnatok_create(mode, k, lut=lut, merges=merges, fmt=fmt,
                                       kmer_lut=kmer_lut, base_ids=base_ids)

    def close(self):
        if getattr(self, "h", None):
            binding.dnatok_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def max_tokens(self, n_bytes: int, n_seq: int = 1) -> int:
        return binding.dnatok_max_tokens(self.h, n_bytes, n_seq)

    def reserve(self, max_bytes: int, max_seq: int = 1):
        binding.dnatok_reserve(self.h, max_bytes, max_seq)

    def set_launch(self, tile_bytes: int, threads: int, ctas_per_sm: int, chunk_tiles: int = 4):
        binding.dnatok_set_launch(self.h, tile_bytes, threads, ctas_per_sm, chunk_tiles)

    def get_launch(self):
        return binding.dnatok_get_launch(self.h)

    def alloc_outputs(self, n_bytes: int, n_seq: int, offsets_capacity: int | None = None,
                      device=None):
        import torch
        dev = device or torch.device("cuda")
        cap = self.max_tokens(n_bytes, n_seq)
        ids = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        if offsets_capacity is None:
            offsets_capacity = n_seq + 1 if self.fmt == RAW else n_bytes + 2
        offs = torch.empty(max(offsets_capacity, 1), dtype=torch.int64, device=dev)
        totals = torch.zeros(2, dtype=torch.int64, device=dev)
        return ids, offs, totals

    def encode(self, data, seq_offsets=None, ids=None, offsets=None, totals=None, stream=None):
        """Asynchronous encode of a CUDA uint8 tensor.  RAW needs seq_offsets
        (CUDA int64, n_seq + 1).  Returns (ids, offsets, totals) tensors; the
        counts are in totals = [n_ids, n_records] once the stream gets there."""
        n = int(data.numel())
        n_seq = int(seq_offsets.numel()) - 1 if seq_offsets is not None else 0
        if ids is None or offsets is None or totals is None:
            ids, offsets, totals = self.alloc_outputs(n, n_seq, device=data.device)
        binding.dnatok_encode(self.h, data.data_ptr() if n else 0, n,
                              seq_offsets.data_ptr() if seq_offsets is not None else 0, n_seq,
                              ids.data_ptr(), ids.numel(), offsets.data_ptr(), offsets.numel(),
                              totals.data_ptr(), _stream_ptr(stream))
        return ids, offsets, totals

    def sync(self, stream=None):
        binding.dnatok_sync(self.h, _stream_ptr(stream))

    def decode(self, ids, id_offsets, n_ids: int | None = None, out=None, byte_offsets=None,
               totals=None, stream=None):
        """Asynchronous decode of CUDA int32 ids with their record offsets
        (CUDA int64, n_seq + 1).  Returns (bytes, byte_offsets, totals) with
        totals = [bytes written, ids without text] once the stream gets there."""
        import torch
        n_ids = int(ids.numel()) if n_ids is None else n_ids
        n_seq = int(id_offsets.numel()) - 1
        if out is None:
            cap = binding.dnatok_max_decoded_bytes(self.h, n_ids, n_seq)
            out = torch.empty(max(cap, 1), dtype=torch.uint8, device=ids.device)
        if byte_offsets is None:
            byte_offsets = torch.empty(n_seq + 1, dtype=torch.int64, device=ids.device)
        if totals is None:
            totals = torch.zeros(2, dtype=torch.int64, device=ids.device)
        binding.dnatok_decode(self.h, ids.data_ptr() if n_ids else 0, n_ids, id_offsets.data_ptr(),
                              n_seq, out.data_ptr(), out.numel(), byte_offsets.data_ptr(),
                              totals.data_ptr(), _stream_ptr(stream))
        return out, byte_offsets, totals

    # ---------------------------------------------------------------- streams
    def stream_open(self, ids, offsets, chunk_bytes: int = 0, n_slots: int = 0,
                    overlap: bool = True):
        """Open a host-streamed encode writing into the CUDA tensors ids
        (int32) and offsets (int64); keep them alive until stream_close."""
        binding.dnatok_stream_open(self.h, ids.data_ptr(), ids.numel(), offsets.data_ptr(),
                                   offsets.numel(), chunk_bytes, n_slots, int(bool(overlap)))

    def stream_submit(self, data, flags: int = 0) -> int:
        """Queue host bytes (numpy uint8 / pinned CPU tensor).  Pass
        HOST_PINNED only for page-locked memory kept alive until completion."""
        import numpy as np
        if hasattr(data, "data_ptr"):
            ptr, n = data.data_ptr(), int(data.numel())
        else:
            a = np.ascontiguousarray(data, dtype=np.uint8)
            ptr, n = a.ctypes.data, a.size
            if flags & HOST_PINNED:
                raise ValueError("HOST_PINNED needs a page-locked tensor")
        return binding.dnatok_stream_submit(self.h, ptr if n else 0, n, flags)

    def stream_poll(self, req_id: int):
        return binding.dnatok_stream_poll(self.h, req_id)

    def stream_wait(self, req_id: int):
        return binding.dnatok_stream_wait(self.h, req_id)

    def stream_close(self):
        binding.dnatok_stream_close(self.h)

    def encode_host(self, data, seq_offsets=None):
        """Copy host bytes to the device, encode, wait, and return numpy
        (ids, offsets) trimmed to the produced counts (a test helper)."""
        import numpy as np
        import torch
        d = torch.from_numpy(np.ascontiguousarray(data, dtype=np.uint8)).cuda()
        so = None
        if self.fmt == RAW:
            if seq_offsets is None:
                seq_offsets = np.array([0, len(data)], dtype=np.int64)
            so = torch.from_numpy(np.ascontiguousarray(seq_offsets, dtype=np.int64)).cuda()
        ids, offs, tot = self.encode(d, so)
        self.sync()
        n_ids, n_rec = (int(x) for x in tot.cpu().tolist())
        return ids[:n_ids].cpu().numpy(), offs[: n_rec + 1].cpu().numpy()


def reverse_complement(data, seq_offsets, out=None, stream=None):
    """Reverse complement of every record of a CUDA uint8 tensor (records by
    seq_offsets, CUDA int64).  Asynchronous; returns the output tensor."""
    import torch
    n = int(data.numel())
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.uint8, device=data.device)
    binding.dnatok_reverse_complement(data.data_ptr() if n else 0, n, seq_offsets.data_ptr(),
                                      int(seq_offsets.numel()) - 1, out.data_ptr(),
                                      _stream_ptr(stream))
    return out[:n] if n else out[:0]


def feed(ids, id_offsets, token_len: int, id_pad: int, dtype=None, row_begin: int = 0,
         n_rows: int | None = None, out=None, stream=None):
    """Fixed-shape (n_rows, token_len) feed of records row_begin.. of (ids,
    id_offsets): left-padded with id_pad, longer records cut to their first
    token_len ids; dtype torch.int64 (default) or torch.int32."""
    import torch
    dtype = torch.int64 if dtype is None else dtype
    if n_rows is None:
        n_rows = int(id_offsets.numel()) - 1 - row_begin
    if out is None:
        out = torch.empty((n_rows, token_len), dtype=dtype, device=ids.device)
    binding.dnatok_feed(ids.data_ptr(), id_offsets.data_ptr(), row_begin, n_rows, token_len,
                        id_pad, out.data_ptr(), out.element_size(), _stream_ptr(stream))
    return out


def microbatch_rows(emb_batch_cap: int, tokens_per_call: int, token_len: int) -> int:
    return binding.dnatok_microbatch_rows(emb_batch_cap, tokens_per_call, token_len)


def feed_pipeline(ids, id_offsets, token_len: int, id_pad: int, rows_per_batch: int, consumer,
                  dtype=None, feed_stream=None, consumer_stream=None):
    """Micro-batched feed on two streams with two buffers used in turn.  For every
    micro-batch consumer(row_begin, batch, stream) is called with a
    (rows, token_len) tensor view and the torch stream it must enqueue its
    work on (e.g. an embedding lookup); the buffer is reused only after that
    work.  Returns once everything is enqueued."""
    import torch
    dtype = torch.int64 if dtype is None else dtype
    n_rows = int(id_offsets.numel()) - 1
    bufs = [torch.empty((rows_per_batch, token_len), dtype=dtype, device=ids.device)
            for _ in range(2)]
    fs = feed_stream or torch.cuda.Stream(device=ids.device)
    cs = consumer_stream or torch.cuda.current_stream(ids.device)
    # the ids may still be in flight on the caller's stream
    fs.wait_stream(torch.cuda.current_stream(ids.device))
    by_addr = {b.data_ptr(): b for b in bufs}

    def _consume(row_begin, n, addr, _stream):
        consumer(row_begin, by_addr[addr][:n], cs)

    binding.dnatok_feed_pipeline(ids.data_ptr(), id_offsets.data_ptr(), n_rows, token_len, id_pad,
                                 bufs[0].element_size(), rows_per_batch, bufs[0].data_ptr(),
                                 bufs[1].data_ptr(), int(fs.cuda_stream), int(cs.cuda_stream),
                                 _consume)
    return bufs, fs


def shard_records(seq_offsets, world_size: int):
    """Byte-balanced contiguous record bounds (world_size + 1) for one
    process per GPU; rank i encodes records bounds[i] .. bounds[i+1]."""
    return binding.dnatok_shard_records(seq_offsets, world_size)


def global_id_offsets(local_offsets, group=None):
    """Turn a rank's local id offsets (its shard's n + 1 int64 offsets
    starting at 0) into global ones: the exclusive scan of every rank's id
    count, exchanged with one all_gather of one integer per rank (any
    torch.distributed backend).  Returns (global offsets, total ids)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = local_offsets[-1:].to(torch.int64).reshape(1)
    counts = [torch.zeros_like(mine) for _ in range(ws)]
    dist.all_gather(counts, mine, group=group)
    counts = torch.cat(counts).cpu()
    base = int(counts[:rank].sum())
    return local_offsets + base, int(counts.sum())


class StreamPart:
    """One rank's part of a long stream split over processes (one GPU each):
    the protocol of dnatok_part_* in three steps with two exchanges between
    them.  `part` is a CUDA uint8 tensor holding the rank's contiguous bytes
    of the stream; `ids` / `offsets` receive its ids and its records'
    offsets (stream-wide id positions).

        p = StreamPart(tok, part, ids, offsets, rank, world)
        maps = exchange(p.line_map())          # two ints per rank
        states = exchange(p.summary(maps))     # six ints per rank
        n_ids, n_offsets, first_id, first_record = p.finish(states)

    The first rank whose part holds bytes starts the stream (ranks before it
    hold empty parts and write nothing), so the stream start merges with a
    header at its first byte exactly as in one encode.
    """

    def __init__(self, tok, part, ids, offsets, rank: int, world: int, stream=None):
        self.tok, self.part, self.ids, self.offsets = tok, part, ids, offsets
        self.rank, self.world = rank, world
        self.sp = _stream_ptr(stream)
        self.n = int(part.numel())
        self.addr = part.data_ptr() if self.n else 0
        self.line_state = 0
        self.lead = 0
        self.mine = None

    def _encode(self, before, last):
        return binding.dnatok_part_encode(self.tok.h, self.addr, self.n, before, last,
                                          self.ids.data_ptr(), self.ids.numel(),
                                          self.offsets.data_ptr(), self.offsets.numel(), self.sp)

    def line_map(self):
        """Step 1: this part's line-state map and length, to exchange."""
        return [binding.dnatok_part_line_map(self.tok.h, self.addr, self.n, self.sp), self.n]

    def summary(self, maps):
        """Step 2 (maps: every rank's step-1 list): the line state at this
        part's start, and this part's state to exchange (the stream's first
        rank: its real encode; the last rank sends nothing anyone reads)."""
        s = 0
        for r in range(self.rank):
            s = (int(maps[r][0]) >> (2 * s)) & 3
        self.line_state = s
        lead = next((r for r in range(self.world) if int(maps[r][1]) > 0), self.world - 1)
        self.lead = lead
        last = self.rank == self.world - 1
        if self.rank == lead:
            self.mine = self._encode(None, last)
        elif lead < self.rank < self.world - 1:
            self.mine = self._encode(binding.PartState.from_list([0, 0, 0, 0, 0, s]), False)
        else:
            self.mine = binding.PartState()
        return self.mine.as_list()

    def finish(self, states):
        """Step 3 (states: every rank's step-2 list): encode the part from the
        state of the stream before it.  Returns (ids written, offsets
        written, stream index of its first id, of its first record)."""
        if self.rank < self.lead:
            return 0, 0, 0, 0
        if self.rank == self.lead:
            return self.mine.d, self.mine.nb, 0, 0
        k = self.tok.k if self.tok.mode == binding.KMER else 1
        before = binding.PartState.from_list(states[self.lead])
        for r in range(self.lead + 1, self.rank):
            before = binding.dnatok_part_combine(k, before, binding.PartState.from_list(states[r]))
        before.line_state = self.line_state
        after = self._encode(before, self.rank == self.world - 1)
        return after.d - before.d, after.nb - before.nb, before.d, before.nb


def encode_stream_part(tok, part, ids, offsets, group=None, stream=None):
    """StreamPart's three steps with torch.distributed all_gathers (CPU
    tensors for gloo, CUDA tensors for nccl) in the default or given group."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")

    def exchange(vals):
        t = torch.tensor(vals, dtype=torch.int64, device=dev)
        out = [torch.empty_like(t) for _ in range(ws)]
        dist.all_gather(out, t, group=group)
        return [o.cpu().tolist() for o in out]

    p = StreamPart(tok, part, ids, offsets, rank, ws, stream)
    maps = exchange(p.line_map())
    states = exchange(p.summary(maps))
    return p.finish(states)
