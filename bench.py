#!/usr/bin/env python3
"""Benchmark: non-overlapping 6-mer tokenization of 4096 DNA sequences.

Workload (seeded, synthetic): 4096 sequences with lengths log-uniform in
[1 kb, 128 kb] (about 109 MB), order-3 Markov DNA at 40% GC with N runs and
soft-masked lowercase stretches; 6-mer ids (4096 k-mers + UNK), int32.

One step = one dnatok_encode of the whole batch with inputs resident in
HBM, replayed from a CUDA graph captured once (the batched form); the same
call launched directly is reported beside it as `plain_launch`.  Before every
timed step, outside the timed events, L2 is flushed by a 256 MB write followed
by a 256 MB read, so the step starts with none of its data in L2 and with no
dirty lines of the flush left to write back.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  N > 1 runs as torchrun ranks, one GPU each: the global
batch is N copies of the 4096 sequences, split by dnatok_shard_records into
byte-balanced contiguous record ranges (the work per GPU stays fixed: weak
scaling); the only exchange is global_id_offsets' all_gather of one id count
per rank, made once after the timed steps; the timing takes the max over
ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encode tokens/s (device-resident, host-streamed) vs HBM/H2D roofline; p99 ms"
WORKLOAD = "6-mer (k=6) ids of 4096 sequences, lengths log-uniform 1-128 kb (~109 MB), " \
           "order-3 Markov 40% GC, N runs, soft-masked"
KERNEL = "dnatok::direct_kmer_kernel<6> (after direct_plan_kernel; the general " \
         "tile_kernel<MODE_KMER, BSRC_LIST> is launched gated and exits at once)"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for fn in ("direct.cu", "tile_kernel.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2601_05531_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(n_bytes_workload: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (scaled to this workload by bytes)."""
    path = os.path.join(ROOT, "profiles", "direct_kernel_kmer6_4096seq_traffic.txt")
    d = {}
    try:
        with open(path) as f:
            for ln in f:
                key, sep, val = ln.partition(":")
                if sep:
                    d[key.strip()] = val.strip()
    except OSError:
        return None
    if d.get("kernel_source_sha256_16") != _kernel_hash():
        return None
    try:
        return float(d["dram_bytes_per_input_byte"]) * n_bytes_workload
    except (KeyError, ValueError):
        return None


def _workload():
    import synth
    return synth.kmer_batch_4096()


def _h2d_peak(torch, src, dev, chunk: int = 64 << 20, reps: int = 10):
    """Pinned-host -> device copy GB/s: best single 64 MiB chunk of `reps`, and
    the sustained rate of back-to-back chunks over the whole buffer."""
    dst = [torch.empty(chunk, dtype=torch.uint8, device=dev) for _ in range(2)]
    s = torch.cuda.current_stream()
    best = 0.0
    for i in range(reps + 2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        dst[i & 1].copy_(src[:chunk], non_blocking=True)
        b.record(s)
        b.synchronize()
        if i >= 2:
            best = max(best, chunk / (a.elapsed_time(b) / 1e3) / 1e9)
    n_chunks = src.numel() // chunk
    sustained = 0.0
    for _ in range(2):  # the second pass over the buffer is the one reported
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for i in range(n_chunks):
            dst[i & 1].copy_(src[i * chunk:(i + 1) * chunk], non_blocking=True)
        b.record(s)
        b.synchronize()
        sustained = n_chunks * chunk / (a.elapsed_time(b) / 1e3) / 1e9
    return best, sustained


def _streamed(torch, P, dev, n_bytes: int, reps: int = 3):
    """Host-streamed 6-mer encode of a FASTA stream held in pinned host
    memory: 64 MiB chunks, 3 device slots, copy and compute streams.  Wall
    time from the first submit to the completion of the last request."""
    import synth
    host = torch.empty(n_bytes, dtype=torch.uint8, pin_memory=True)
    _, lay = synth.fasta_stream(n_bytes, seed=47, out=host.numpy())
    n_rec = len(lay.rec_off)
    k = 6
    ids = torch.empty(n_bytes // k + 2 * n_rec + 1024, dtype=torch.int32, device=dev)
    offs = torch.empty(n_rec + 2, dtype=torch.int64, device=dev)
    best_h2d, sustained_h2d = _h2d_peak(torch, host, dev)
    out = {"workload": "6-mer ids of a %.2f GiB FASTA stream in pinned host memory "
                       "(records log-uniform 10 kb-10 Mb, headers 20-80 B, lines 60/80)"
                       % (n_bytes / 2**30),
           "chunk_bytes": 64 << 20, "slots": 3, "records": n_rec,
           "h2d_peak_gbs": best_h2d, "h2d_peak": "best of 10 pinned 64 MiB cudaMemcpyAsync",
           "h2d_sustained_gbs": sustained_h2d}
    with P.Tokenizer(P.KMER, k=k, fmt=P.FASTA) as tok:
        for overlap in (True, False):
            times, res = [], None
            for i in range(reps + 1):
                tok.stream_open(ids, offs, chunk_bytes=64 << 20, n_slots=3, overlap=overlap)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = tok.stream_submit(host, P.HOST_PINNED | P.END_OF_STREAM)
                res = tok.stream_wait(r)
                t = time.perf_counter() - t0
                tok.stream_close()
                if i > 0:
                    times.append(t)
            t = statistics.median(times)
            key = "overlap" if overlap else "serial"
            out[key] = {"tokens_per_s": res[0] / t, "ms": 1e3 * t, "h2d_gbs": n_bytes / t / 1e9,
                        "frac_of_h2d_peak": n_bytes / t / 1e9 / best_h2d,
                        "frac_of_h2d_sustained": n_bytes / t / 1e9 / sustained_h2d}
            out["tokens"] = res[0]
    del host
    return out


def _batched(torch, P, dev, data, offs, d_bytes, d_offs, reps: int = 5):
    """The batched form against per-request plain launches: the whole
    4096-sequence batch as one launch (direct and replayed from a CUDA graph)
    versus one dnatok_encode per sequence; and 64 independent 1 MB
    single-nucleotide calls as plain launches versus one graph replay."""
    import numpy as np
    import synth
    B = P.binding
    n, n_seq = len(data), len(offs) - 1
    s = torch.cuda.Stream()
    out = {}
    with P.Tokenizer(P.KMER, k=6) as tok:
        tok.reserve(n, n_seq)
        ids, o, tot = tok.alloc_outputs(n, n_seq, device=dev)
        with torch.cuda.stream(s):
            tok.encode(d_bytes, d_offs, ids, o, tot, stream=s)
        s.synchronize()
        id_off = o[: n_seq + 1].cpu().numpy()
        n_ids = int(tot[0])

        def timed(fn):
            fn()
            s.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            a.record(s)
            for _ in range(reps):
                fn()
            b.record(s)
            b.synchronize()
            return a.elapsed_time(b) / reps, 1e3 * (time.perf_counter() - t0) / reps

        one_ms, one_wall = timed(lambda: B.dnatok_encode(
            tok.h, d_bytes.data_ptr(), n, d_offs.data_ptr(), n_seq, ids.data_ptr(), ids.numel(),
            o.data_ptr(), o.numel(), tot.data_ptr(), s.cuda_stream))
        # per-sequence plain launches, ids written at the same places
        scratch_o = torch.empty(2 * n_seq, dtype=torch.int64, device=dev)
        offs_d = torch.from_numpy(np.stack([np.zeros(n_seq, np.int64),
                                            np.diff(offs)], axis=1).reshape(-1)).to(dev)
        bp, ip = d_bytes.data_ptr(), ids.data_ptr()
        op, sp = offs_d.data_ptr(), scratch_o.data_ptr()

        def per_seq():
            for r in range(n_seq):
                ln = int(offs[r + 1] - offs[r])
                cap = int(id_off[r + 1] - id_off[r])
                B.dnatok_encode(tok.h, bp + int(offs[r]) if ln else 0, ln, op + 16 * r, 1,
                                ip + 4 * int(id_off[r]), max(cap, (ln + 5) // 6 + 1),
                                sp + 16 * r, 2, 0, s.cuda_stream)

        seq_ms, seq_wall = timed(per_seq)
        B.dnatok_graph_begin(tok.h, s.cuda_stream)
        B.dnatok_encode(tok.h, d_bytes.data_ptr(), n, d_offs.data_ptr(), n_seq, ids.data_ptr(),
                        ids.numel(), o.data_ptr(), o.numel(), tot.data_ptr(), s.cuda_stream)
        g = B.dnatok_graph_end(tok.h, s.cuda_stream)
        g_ms, g_wall = timed(lambda: B.dnatok_graph_launch(g, s.cuda_stream))
        B.dnatok_graph_destroy(g)
        tok.sync(s)
        out["kmer6_4096seq"] = {
            "tokens": n_ids,
            "one_launch": {"ms": one_ms, "wall_ms": one_wall, "tokens_per_s": n_ids / one_wall * 1e3},
            "graph_replay": {"ms": g_ms, "wall_ms": g_wall, "tokens_per_s": n_ids / g_wall * 1e3},
            "per_sequence_launches": {"launches": n_seq, "ms": seq_ms, "wall_ms": seq_wall,
                                      "tokens_per_s": n_ids / seq_wall * 1e3},
            "note": "ids may be cut short in the per-sequence arm only where a sequence's "
                    "capacity bound exceeds the batched result; tokens counted from the batch"}
    # 64 independent 1 MB single-nucleotide calls
    one, _ = synth.single_sequence_1mb()
    m1 = len(one)
    calls = 64
    with P.Tokenizer(P.CHAR) as tok:
        tok.reserve(m1, 1)
        ins = [torch.from_numpy(synth.single_sequence_1mb(seed=43 + i)[0]).to(dev)
               for i in range(calls)]
        so = torch.tensor([0, m1], dtype=torch.int64, device=dev)
        outs = [tok.alloc_outputs(m1, 1, device=dev) for _ in range(calls)]

        def plain():
            for i in range(calls):
                ids, o, tot = outs[i]
                B.dnatok_encode(tok.h, ins[i].data_ptr(), m1, so.data_ptr(), 1, ids.data_ptr(),
                                ids.numel(), o.data_ptr(), o.numel(), tot.data_ptr(),
                                s.cuda_stream)

        p_ms, p_wall = timed(plain)
        B.dnatok_graph_begin(tok.h, s.cuda_stream)
        plain()
        g = B.dnatok_graph_end(tok.h, s.cuda_stream)
        g_ms, g_wall = timed(lambda: B.dnatok_graph_launch(g, s.cuda_stream))
        B.dnatok_graph_destroy(g)
        tok.sync(s)
        toks = calls * int(outs[0][2][0])
        out["char_64x1MB"] = {
            "calls": calls,
            "plain_launches": {"us_per_call": 1e3 * p_wall / calls,
                               "tokens_per_s": toks / p_wall * 1e3},
            "graph_replay": {"us_per_call": 1e3 * g_wall / calls,
                             "tokens_per_s": toks / g_wall * 1e3}}
    return out


def _overlap(torch, P, dev, d_bytes, d_offs, n, n_seq, flush_l2, steps: int = 10):
    """The same 4096-sequence batch as overlapping (stride-1) 6-mers: one
    dnatok_encode per step (symbol pass, offsets, emit), L2 flushed between
    steps, CUDA events on the launching stream."""
    s = torch.cuda.current_stream()
    with P.Tokenizer(P.KMER_OVERLAP, k=6) as tok:
        ids, o, tot = tok.alloc_outputs(n, n_seq, device=dev)
        for i in range(3):
            flush_l2(i)
            tok.encode(d_bytes, d_offs, ids, o, tot, stream=s)
        tok.sync()
        n_ids = int(tot[0].item())
        evs = []
        for i in range(steps):
            flush_l2(i)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            tok.encode(d_bytes, d_offs, ids, o, tot, stream=s)
            b.record(s)
            evs.append((a, b))
        torch.cuda.synchronize()
        tok.sync()
    ms = sorted(a.elapsed_time(b) for a, b in evs)
    med = ms[len(ms) // 2]
    alg = n + 4 * n_ids + 16 * (n_seq + 1)
    peak, kind = _peaks()
    return {"workload": "overlapping (stride-1) 6-mers of the same 4096 sequences",
            "tokens": n_ids, "ms": med, "tokens_per_s": n_ids / (med / 1e3),
            "roofline": {"bound": "hbm", "achieved": alg / (med / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": alg / (med / 1e3) / 1e9 / peak,
                         "peak_kind": kind, "algorithmic_bytes_per_step": alg,
                         "duration": "CUDA events around the whole encode (symbol pass, "
                                     "offsets and emit kernels)"}}


def _time_median(torch, fn, flush_l2, steps: int = 10, warm: int = 3):
    """Median CUDA-event time (ms) of fn() on the current stream, L2 flushed
    before each run (outside the events)."""
    s = torch.cuda.current_stream()
    for i in range(warm):
        flush_l2(i)
        fn()
    torch.cuda.synchronize()
    evs = []
    for i in range(steps):
        flush_l2(i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in evs)
    return ms[len(ms) // 2]


def _hbm(alg, ms, what):
    peak, kind = _peaks()
    ach = alg / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": kind, "algorithmic_bytes_per_step": alg, "duration": what}


def _ktab(torch, P, dev, d_bytes, d_offs, n, n_seq, flush_l2):
    """The 4096-sequence batch through a 5^6-entry k-mer table laid out like a
    blocked 6-mer model's vocabulary (windows with N fall back to single
    symbols), straight from the RAW bytes: window plan, count (window
    entries), tile scan and expand, with the general path's five kernels
    launched gated behind them (they exit at once)."""
    import synth
    lut, base = synth.kmer_vocab(6, seed=49)
    s = torch.cuda.current_stream()
    with P.Tokenizer(P.KMER_TABLE, k=6, kmer_lut=lut, base_ids=base) as tok:
        ids, o, tot = tok.alloc_outputs(n, n_seq, device=dev)
        ms = _time_median(torch, lambda: tok.encode(d_bytes, d_offs, ids, o, tot, stream=s), flush_l2)
        tok.sync()
        n_ids = int(tot[0].item())
        direct = P.binding.dnatok_direct_ran(tok.h)
    alg = n + 4 * n_ids + 16 * (n_seq + 1)
    return {"workload": "table-driven 6-mers (5^6 table, single-symbol fallback) of the same "
                        "4096 sequences", "tokens": n_ids, "ms": ms,
            "tokens_per_s": n_ids / (ms / 1e3), "path": "raw bytes" if direct == 1 else "general",
            "roofline": _hbm(alg, ms, "CUDA events around the whole encode (plan, count, scan, "
                                      "expand, and the general path's gated launches)"),
            "gpu_launches_per_step": 9}


def _decode_rc_feed(torch, P, dev, d_bytes, d_offs, n, n_seq, flush_l2):
    """Decode of the batch's 6-mer ids back to text, reverse complement of
    its bytes, and the fixed-shape int64 feed of its ids (rows of 2048, the
    micro-batched two-stream form with an embedding lookup as consumer)."""
    s = torch.cuda.current_stream()
    out = {}
    with P.Tokenizer(P.KMER, k=6) as tok:
        ids, o, tot = tok.alloc_outputs(n, n_seq, device=dev)
        tok.encode(d_bytes, d_offs, ids, o, tot, stream=s)
        tok.sync()
        n_ids = int(tot[0].item())
        ids = ids[:max(n_ids, 1)]
        cap = P.binding.dnatok_max_decoded_bytes(tok.h, n_ids, n_seq)
        text = torch.empty(cap, dtype=torch.uint8, device=dev)
        bo = torch.empty(n_seq + 1, dtype=torch.int64, device=dev)
        dt = torch.zeros(2, dtype=torch.int64, device=dev)
        ms = _time_median(torch, lambda: tok.decode(ids, o, n_ids=n_ids, out=text, byte_offsets=bo,
                                                    totals=dt, stream=s), flush_l2)
        tok.sync()
        n_text = int(dt[0].item())
        alg = 4 * n_ids + n_text + 16 * (n_seq + 1)
        out["decode_kmer6_4096seq"] = {
            "workload": "6-mer ids of the 4096 sequences back to text", "ids": n_ids,
            "bytes_out": n_text, "ms": ms, "ids_per_s": n_ids / (ms / 1e3),
            "roofline": _hbm(alg, ms, "CUDA events around the decode (count, scan, emit)")}

        rc = torch.empty(n, dtype=torch.uint8, device=dev)
        ms = _time_median(torch, lambda: P.reverse_complement(d_bytes, d_offs, out=rc, stream=s),
                          flush_l2)
        alg = 2 * n + 8 * (n_seq + 1)
        out["reverse_complement_4096seq"] = {
            "workload": "reverse complement of every record of the 4096 sequences",
            "bytes": n, "ms": ms, "bytes_per_s": n / (ms / 1e3),
            "roofline": _hbm(alg, ms, "CUDA events around the one launch")}

        T = 2048
        fo = torch.empty((n_seq, T), dtype=torch.int64, device=dev)
        ms = _time_median(torch, lambda: P.feed(ids, o, T, 4097, out=fo, stream=s), flush_l2)
        lens = (o[1:] - o[:-1]).clamp(max=T)
        kept = int(lens.sum().item())
        alg = 4 * kept + 8 * n_seq * T + 16 * (n_seq + 1)
        out["feed_int64_4096x2048"] = {
            "workload": "left-padded int64 feed of the 6-mer ids, 4096 rows of 2048",
            "elements": n_seq * T, "ms": ms, "elements_per_s": n_seq * T / (ms / 1e3),
            "roofline": _hbm(alg, ms, "CUDA events around the one launch")}

        # micro-batched feed into an embedding lookup (d = 256, bf16 table):
        # two streams with two buffers used in turn vs the same work on one stream
        rows = P.microbatch_rows(256, 1 << 18, T)
        emb = torch.randn(4099, 256, device=dev, dtype=torch.bfloat16)
        sink = torch.empty((rows, T, 256), device=dev, dtype=torch.bfloat16)

        def consumer(row_begin, batch, stream):
            with torch.cuda.stream(stream):
                torch.index_select(emb, 0, batch.reshape(-1), out=sink[:batch.shape[0]].view(-1, 256))

        fs, cs = torch.cuda.Stream(), torch.cuda.Stream()
        res = {}
        for name, feed_s in (("pipelined", fs), ("one_stream", cs)):
            for rep in range(2):
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(cs)
                fs.wait_event(a)
                P.feed_pipeline(ids, o, T, 4097, rows, consumer, feed_stream=feed_s,
                                consumer_stream=cs)
                b.record(cs)
                torch.cuda.synchronize()
                res[name] = a.elapsed_time(b)
        out["feed_pipeline_embedding"] = {
            "workload": "4096 rows of 2048 int64 ids in micro-batches of %d rows into an "
                        "embedding lookup (4099 x 256 bf16)" % rows,
            "rows_per_batch": rows, "ms_pipelined": res["pipelined"],
            "ms_one_stream": res["one_stream"]}
    return out


def _served(P, tr, merges, seconds):
    """Replay a request trace in real time through the serving loop.  Latency
    of a request = the time its completion is seen by this host thread minus
    its arrival time in the trace (the time it waits while the loop refuses
    it for lack of memory or slots is included)."""
    import numpy as np
    import torch
    B = P.binding
    n = len(tr.sizes)
    pin = torch.from_numpy(tr.data).pin_memory()
    base = pin.data_ptr()
    srv = B.dnatok_server_create(budget_bytes=4 << 30, host_arena_bytes=1 << 30,
                                 max_batch_bytes=32 << 20, max_batch_requests=256, n_slots=4,
                                 kmer_k=6, merges=merges)
    lat = np.zeros(n)
    toks, refused = 0, 0
    done_t = 0.0
    try:
        pending = []
        t0 = time.perf_counter() + 0.05
        i = 0
        while i < n or pending:
            now = time.perf_counter() - t0
            while i < n and tr.arrival_s[i] <= now:
                r = B.dnatok_server_submit(srv, int(tr.modes[i]), base + int(tr.offsets[i]),
                                           int(tr.sizes[i]))
                if r is None:
                    refused += 1
                    break  # retried on the next pass; its latency keeps running
                pending.append((i, r))
                i += 1
            still = []
            for (k, r) in pending:
                out = B.dnatok_server_poll(srv, r)
                if out is None:
                    still.append((k, r))
                    continue
                done_t = time.perf_counter() - t0
                lat[k] = 1e3 * (done_t - tr.arrival_s[k])
                toks += out[1]
                B.dnatok_server_release(srv, r)
            pending = still
        st = B.dnatok_server_stats(srv)
    finally:
        B.dnatok_server_destroy(srv)
    return {"tokens_per_s": toks / done_t, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "batches": st["batches_launched"],
            "wall_s": done_t, "tokens": int(toks), "refused_submits": refused,
            "offered_bytes_per_s": float(tr.sizes.sum() / seconds)}


def _per_request(torch, P, dev, tr, merges):
    """The same trace through per-request plain launches: each request's
    host copy, encode and wait, one request at a time, in arrival order."""
    import numpy as np
    B = P.binding
    n = len(tr.sizes)
    pin = torch.from_numpy(tr.data).pin_memory()
    base = pin.data_ptr()
    toks_b = {0: P.Tokenizer(P.CHAR), 1: P.Tokenizer(P.KMER, k=6),
              2: P.Tokenizer(P.BPE, merges=merges)}
    mx = int(tr.sizes.max())
    for t in toks_b.values():
        t.reserve(mx, 1)
    ids = torch.empty(mx + 16, dtype=torch.int32, device=dev)
    hso = torch.zeros(2, dtype=torch.int64).pin_memory()
    hoo = torch.zeros(2, dtype=torch.int64).pin_memory()
    hto = torch.zeros(2, dtype=torch.int64).pin_memory()
    s = torch.cuda.Stream()
    lat_b = np.zeros(n)
    toks2 = 0
    t0 = time.perf_counter() + 0.05
    for k in range(n):
        while time.perf_counter() - t0 < tr.arrival_s[k]:
            pass
        ln = int(tr.sizes[k])
        hso[1] = ln
        B.dnatok_encode_host(toks_b[int(tr.modes[k])].h, base + int(tr.offsets[k]), ln,
                             hso.data_ptr(), 1, ids.data_ptr(), ids.numel(), hoo.data_ptr(), 2,
                             hto.data_ptr(), s.cuda_stream)
        now = time.perf_counter() - t0
        lat_b[k] = 1e3 * (now - tr.arrival_s[k])
        toks2 += int(hto[0])
    wall_b = time.perf_counter() - t0
    for t in toks_b.values():
        t.close()
    return {"tokens_per_s": toks2 / wall_b, "p50_ms": float(np.percentile(lat_b, 50)),
            "p99_ms": float(np.percentile(lat_b, 99)), "wall_s": wall_b, "tokens": toks2}


def _serving(torch, P, dev, seconds: float):
    """The serving request trace (Poisson 2000/s, 200 B-1 MB, 30% single-
    nucleotide / 50% 6-mer / 20% BPE with the 4096-merge table) replayed in
    real time through the serving loop, and through per-request plain
    launches (host copy + encode + wait, one request at a time); then both
    at three times the arrival rate (3 s of trace)."""
    import numpy as np
    import synth
    tr = synth.request_trace(duration_s=seconds)
    n = len(tr.sizes)
    m = np.loadtxt(os.path.join(ROOT, "tests", "golden", "bpe_merges_markov45_seed45_4096.txt"),
                   dtype=np.int32)
    res = {"requests": n, "offered_bytes_per_s": float(tr.sizes.sum() / seconds),
           "budget_bytes": 4 << 30,
           "latency": "both arms: completion seen by the submitting host thread minus the "
                      "request's arrival time in the trace (queueing and refused submits "
                      "included)"}
    res["served"] = _served(P, tr, m, seconds)
    res["per_request_launches"] = _per_request(torch, P, dev, tr, m)
    over_s = min(3.0, seconds)
    tr3 = synth.request_trace(rate=6000.0, duration_s=over_s)
    res["served_x3_rate"] = dict(_served(P, tr3, m, over_s), requests=len(tr3.sizes),
                                 rate_per_s=6000.0)
    res["per_request_x3_rate"] = dict(_per_request(torch, P, dev, tr3, m), requests=len(tr3.sizes),
                                      rate_per_s=6000.0)
    return res


def _cpu_baseline(data, offs, budget_s: float = 10.0):
    """The oracle as it stands on this host, on a bounded sample of the same
    workload: single-threaded on a ~25 MB slice of whole records (repeated
    until ~budget_s), and on all cores with the whole batch split into
    byte-balanced record ranges, one per task."""
    import numpy as np

    import oracle
    n_seq = len(offs) - 1
    stop = int(np.searchsorted(offs, 25_000_000))
    stop = max(1, min(stop, n_seq))
    sample = data[: offs[stop]]
    so = offs[: stop + 1].copy()
    toks, secs, reps = 0, 0.0, 0
    while secs < budget_s or reps == 0:
        t0 = time.perf_counter()
        ids, _ = oracle.encode(sample, oracle.KMER, k=6, seq_offsets=so)
        secs += time.perf_counter() - t0
        toks += len(ids)
        reps += 1
    out = {"value": toks / secs, "unit": "tokens/s", "cores": 1, "kind": "oracle",
           "bytes_per_s": reps * int(offs[stop]) / secs,
           "sample": "first %d of %d sequences (%.1f MB), %d pass(es), %.1f s single-threaded"
                     % (stop, n_seq, offs[stop] / 1e6, reps, secs), "cpu_model": _cpu_model()}
    nc = _cores()
    parts = 4 * nc
    cuts = np.searchsorted(offs, np.linspace(0, offs[-1], parts + 1)).clip(0, n_seq)
    cuts[0], cuts[-1] = 0, n_seq
    spans = [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    args = [(data[offs[a]:offs[b]], offs[a:b + 1] - offs[a]) for a, b in spans]
    res, wall = _all_cores(_oracle_kmer_part, args)
    out["all_cores"] = {"value": sum(res) / wall, "unit": "tokens/s", "cores": nc,
                        "bytes_per_s": int(offs[-1]) / wall,
                        "sample": "all %d sequences (%.1f MB) in %d record ranges on %d spawned "
                                  "workers, %.2f s" % (n_seq, offs[-1] / 1e6, len(spans), nc,
                                                       wall)}
    return out


def _extras(line, torch, P, dev, data, offs, d_bytes, d_offs, flush_l2, args):
    """The other configurations and rows, each with its own roofline line."""
    n_bytes, n_seq = len(data), len(offs) - 1
    line["batched"] = _batched(torch, P, dev, data, offs, d_bytes, d_offs)
    line["char_1mb"] = _char_1mb(torch, P, dev, flush_l2)
    line["kmer6_4096seq_uniform"] = _kmer_uniform(torch, P, dev, flush_l2)
    line["bpe_1gib"] = _bpe_1gib(torch, P, dev, flush_l2, with_cpu=not args.no_cpu_baseline)
    line["fasta_chunk_64mib"] = _fasta_chunk(torch, P, dev, 64)
    line["kmer6_overlap_4096seq"] = _overlap(torch, P, dev, d_bytes, d_offs, n_bytes, n_seq,
                                             flush_l2)
    line["kmer6_table_4096seq"] = _ktab(torch, P, dev, d_bytes, d_offs, n_bytes, n_seq, flush_l2)
    line.update(_decode_rc_feed(torch, P, dev, d_bytes, d_offs, n_bytes, n_seq, flush_l2))
    if args.serve_seconds > 0:
        line["serving"] = _serving(torch, P, dev, args.serve_seconds)


def _graph_of(P, tok, stream, fn):
    """fn() captured once on `stream` through the library's graph API."""
    B = P.binding
    B.dnatok_graph_begin(tok.h, stream.cuda_stream)
    fn()
    return B.dnatok_graph_end(tok.h, stream.cuda_stream)


def _char_1mb(torch, P, dev, flush_l2):
    """Single-nucleotide ids of one 1 MB sequence.  One call with
    L2 flushed before it (plain launch and graph replay), and 64 independent
    1 MB calls replayed back to back from one graph (64 MB in, 256 MB out,
    more than L2 holds)."""
    import synth
    B = P.binding
    one, _ = synth.single_sequence_1mb()
    m1 = len(one)
    s = torch.cuda.current_stream()
    out = {"workload": "single-nucleotide ids of one 1 MB sequence (i.i.d. ACGT, 1% N runs, "
                       "5% lowercase)", "input_bytes": m1}
    with P.Tokenizer(P.CHAR) as tok:
        tok.reserve(m1, 1)
        d = torch.from_numpy(one).to(dev)
        so = torch.tensor([0, m1], dtype=torch.int64, device=dev)
        ids, o, tot = tok.alloc_outputs(m1, 1, device=dev)

        def call():
            tok.encode(d, so, ids, o, tot, stream=s)

        plain = _time_median(torch, call, flush_l2, steps=20)
        g = _graph_of(P, tok, s, call)
        rep = _time_median(torch, lambda: B.dnatok_graph_launch(g, s.cuda_stream), flush_l2,
                           steps=20)
        B.dnatok_graph_destroy(g)
        tok.sync()
        n_ids = int(tot[0].item())
        alg = 5 * n_ids + 32
        out.update({"tokens": n_ids, "us_per_call": 1e3 * plain, "us_per_call_graph": 1e3 * rep,
                    "tokens_per_s": n_ids / (rep / 1e3),
                    "roofline": _hbm(alg, rep, "CUDA events around one graph replay of one "
                                               "call (L2 flushed before it)")})
        calls = 64
        ins = [torch.from_numpy(synth.single_sequence_1mb(seed=43 + i)[0]).to(dev)
               for i in range(calls)]
        outs = [tok.alloc_outputs(m1, 1, device=dev) for _ in range(calls)]

        def batch():
            for i in range(calls):
                tok.encode(ins[i], so, *outs[i], stream=s)

        g = _graph_of(P, tok, s, batch)
        ms = _time_median(torch, lambda: B.dnatok_graph_launch(g, s.cuda_stream), flush_l2,
                          steps=10)
        B.dnatok_graph_destroy(g)
        tok.sync()
        toks = sum(int(x[2][0].item()) for x in outs)
        out["x64_graph"] = {"calls": calls, "ms": ms, "us_per_call": 1e3 * ms / calls,
                            "tokens_per_s": toks / (ms / 1e3),
                            "roofline": _hbm(5 * toks + 32 * calls, ms,
                                             "CUDA events around one replay of 64 calls")}
    return out


def _kmer_uniform(torch, P, dev, flush_l2):
    """The same 6-mer encode on 4096 sequences with lengths
    uniform in [1 kb, 128 kb] (about 264 MB), graph replay and plain launch."""
    import synth
    B = P.binding
    data, offs = synth.kmer_batch_4096(uniform=True)
    n, n_seq = len(data), len(offs) - 1
    s = torch.cuda.current_stream()
    with P.Tokenizer(P.KMER, k=6) as tok:
        tok.reserve(n, n_seq)
        d = torch.from_numpy(data).to(dev)
        so = torch.from_numpy(offs).to(dev)
        ids, o, tot = tok.alloc_outputs(n, n_seq, device=dev)

        def call():
            tok.encode(d, so, ids, o, tot, stream=s)

        plain = _time_median(torch, call, flush_l2, steps=10)
        g = _graph_of(P, tok, s, call)
        rep = _time_median(torch, lambda: B.dnatok_graph_launch(g, s.cuda_stream), flush_l2,
                           steps=10)
        B.dnatok_graph_destroy(g)
        tok.sync()
        n_ids = int(tot[0].item())
    alg = n + 4 * n_ids + 16 * (n_seq + 1)
    return {"workload": "6-mer ids of 4096 sequences, lengths uniform 1-128 kb", "input_bytes": n,
            "tokens": n_ids, "ms": rep, "ms_plain": plain, "tokens_per_s": n_ids / (rep / 1e3),
            "roofline": _hbm(alg, rep, "CUDA events around one graph replay"),
            "roofline_plain": _hbm(alg, plain, "CUDA events around one plain call")}


def _bpe_1gib(torch, P, dev, flush_l2, with_cpu: bool = True, steps: int = 5):
    """BPE with the 4096-merge table (trained by the oracle's
    trainer on a 10 MB Markov corpus) on 512 x 2,097,152 fresh bases (1 GiB).
    Device-resident encode (L2 flushed; the input is 8x L2 anyway), the
    repair statistics of the merge pass, the end-to-end call from pinned
    host buffers, and the oracle on a sample of records."""
    import numpy as np
    import synth
    B = P.binding
    data, offs = synth.bpe_apply_corpus()
    merges = np.loadtxt(os.path.join(ROOT, "tests", "golden",
                                     "bpe_merges_markov45_seed45_4096.txt"), dtype=np.int32)
    n, n_seq = len(data), len(offs) - 1
    s = torch.cuda.current_stream()
    out = {"workload": "BPE (4096 merges) of 512 x 2,097,152 uppercase bases (1 GiB), "
                       "order-3 Markov 45% GC", "input_bytes": n}
    with P.Tokenizer(P.BPE, merges=merges) as tok:
        tok.reserve(n, n_seq)
        d = torch.from_numpy(data).to(dev)
        so = torch.from_numpy(offs).to(dev)
        ids, o, tot = tok.alloc_outputs(n, n_seq, device=dev)
        ms = _time_median(torch, lambda: tok.encode(d, so, ids, o, tot, stream=s), flush_l2,
                          steps=steps)
        tok.sync()
        n_ids = int(tot[0].item())
        out["merge_pass"] = B.dnatok_bpe_stats(tok.h, s.cuda_stream)
        out["segment_halo"] = list(B.dnatok_get_bpe_launch(tok.h))
        del d, so
        # end to end from pinned host buffers
        h_bytes = torch.from_numpy(data).pin_memory()
        h_offs = torch.from_numpy(offs).pin_memory()
        h_ooff = torch.empty(n_seq + 1, dtype=torch.int64).pin_memory()
        h_tot = torch.zeros(2, dtype=torch.int64)

        def e2e():
            B.dnatok_encode_host(tok.h, h_bytes.data_ptr(), n, h_offs.data_ptr(), n_seq,
                                 ids.data_ptr(), ids.numel(), h_ooff.data_ptr(), n_seq + 1,
                                 h_tot.data_ptr(), s.cuda_stream)

        e2e()
        t0 = time.perf_counter()
        for _ in range(3):
            e2e()
        e2e_s = (time.perf_counter() - t0) / 3
        assert int(h_tot[0]) == n_ids
    alg = n + 4 * n_ids + 16 * (n_seq + 1)
    out.update({"tokens": n_ids, "bases_per_token": n / n_ids, "ms": ms,
                "tokens_per_s": n_ids / (ms / 1e3), "bytes_per_s": n / (ms / 1e3),
                "roofline": _hbm(alg, ms, "CUDA events around the whole encode (symbol pass, "
                                          "merge pass, maps, scans, emit, offsets)"),
                "e2e": {"value": n_ids / e2e_s, "unit": "tokens/s", "ms_per_step": 1e3 * e2e_s,
                        "h2d_bytes_per_step": n + 8 * (n_seq + 1),
                        "d2h_bytes_per_step": 8 * (n_seq + 1) + 16,
                        "api": "dnatok_encode_host (pinned host buffers)"}})
    if with_cpu:
        out["cpu_baseline"] = _cpu_baseline_bpe(data, offs, merges)
    return out


_FASTA_PATHS = {1: "compacted on the device, then the direct k-mer kernels",
                0: "general tile kernel (the compacted path declined)",
                -1: "general tile kernel"}


def _fasta_chunk(torch, P, dev, mib: int, steps: int = 10):
    """Device-resident 6-mer encode of one FASTA chunk (the first `mib` MiB
    of the seeded 8 GiB stream): the unit of work the host-streamed encode
    hands the general kernel."""
    import numpy as np
    import synth
    n = mib << 20
    host = np.empty(n, dtype=np.uint8)
    synth.fasta_stream(n, seed=47, out=host)
    d = torch.from_numpy(host).to(dev)
    s = torch.cuda.current_stream()
    with P.Tokenizer(P.KMER, k=6, fmt=P.FASTA) as tok:
        ids, o, tot = tok.alloc_outputs(n, 1, device=dev)
        ms = _time_median(torch, lambda: tok.encode(d, None, ids, o, tot, stream=s),
                          lambda i: None, steps=steps)
        tok.sync()
        path = P.binding.dnatok_direct_ran(tok.h)
        n_ids, n_rec = int(tot[0].item()), int(tot[1].item())
    alg = n + 4 * n_ids + 8 * (n_rec + 1)
    return {"workload": "6-mer ids of a %d MiB FASTA chunk (device-resident)" % mib,
            "path": _FASTA_PATHS[path],
            "tokens": n_ids, "records": n_rec, "ms": ms, "gb_per_s": n / (ms / 1e3) / 1e9,
            "roofline": _hbm(alg, ms, "CUDA events around one encode (the chunk is "
                                      "%d MiB; L2 not flushed)" % mib)}


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _oracle_kmer_part(data, offs):
    import oracle
    ids, _ = oracle.encode(data, oracle.KMER, k=6, seq_offsets=offs)
    return len(ids)


def _oracle_bpe_part(r0, r1):
    import numpy as np
    import oracle
    import synth
    d, o = synth.bpe_apply_corpus(records=(r0, r1), threads=1)
    m = np.loadtxt(os.path.join(ROOT, "tests", "golden", "bpe_merges_markov45_seed45_4096.txt"),
                   dtype=np.int32)
    t0 = time.perf_counter()
    ids, _ = oracle.encode(d, oracle.BPE, seq_offsets=o, merges=m)
    return len(ids), time.perf_counter() - t0


def _all_cores(fn, parts):
    """fn(*part) for every part on every core of this process (spawned
    workers, one part each at a time); returns (results, wall seconds of
    the whole map after the workers started)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(_cores(), mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_noop, range(_cores())))  # start every worker first
        t0 = time.perf_counter()
        res = list(ex.map(fn, *zip(*parts)))
        return res, time.perf_counter() - t0


def _noop(_):
    return 0


def _cpu_baseline_bpe(data, offs, merges, budget_s: float = 10.0):
    """The oracle's BPE as it stands on this host: one thread on whole
    records until ~budget_s, and all cores on 4 records per core."""
    import oracle
    n_seq = len(offs) - 1
    toks, secs, recs = 0, 0.0, 0
    while secs < budget_s and recs < n_seq:
        a, b = int(offs[recs]), int(offs[recs + 1])
        t0 = time.perf_counter()
        ids, _ = oracle.encode(data[a:b], oracle.BPE, merges=merges)
        secs += time.perf_counter() - t0
        toks += len(ids)
        recs += 1
    out = {"value": toks / secs, "unit": "tokens/s", "cores": 1, "kind": "oracle",
           "bytes_per_s": int(offs[recs]) / secs,
           "sample": "first %d of %d records (%.1f MB), %.1f s single-threaded"
                     % (recs, n_seq, offs[recs] / 1e6, secs), "cpu_model": _cpu_model()}
    nc = _cores()
    per = 4 * nc
    res, wall = _all_cores(_oracle_bpe_part, [(r, r + 1) for r in range(min(per, n_seq))])
    t_all = sum(r[0] for r in res)
    out["all_cores"] = {"value": t_all / wall, "unit": "tokens/s", "cores": nc,
                        "bytes_per_s": min(per, n_seq) * (offs[1] - offs[0]) / wall,
                        "sample": "%d records (one per task) on %d spawned workers, %.1f s"
                                  % (min(per, n_seq), nc, wall)}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    data, offs = _workload()
    n_seq = len(offs) - 1
    stop = max(1, min(int(np.searchsorted(offs, 12_000_000)), n_seq))
    sample, so = data[: offs[stop]], offs[: stop + 1].copy()
    for _ in range(args.warmup):
        oracle.encode(sample, oracle.KMER, k=6, seq_offsets=so)
    times, toks = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ids, _ = oracle.encode(sample, oracle.KMER, k=6, seq_offsets=so)
        times.append(time.perf_counter() - t0)
        toks = len(ids)
    total = sum(times)
    value = toks * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": "tokens/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "sample_sequences": stop, "sample_mb": offs[stop] / 1e6},
        "cpu_baseline": {"value": value, "unit": "tokens/s", "cores": 1, "kind": "oracle",
                         "sample": "first %d of %d sequences (%.1f MB) per step" %
                                   (stop, n_seq, offs[stop] / 1e6)},
        "e2e": {"value": value, "unit": "tokens/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _shard(data, offs, ws: int, rank: int):
    """This rank's records of the global batch: N copies of the 4096-sequence
    batch back to back (N = world size, so the work per GPU stays fixed),
    split into byte-balanced contiguous record ranges by the library's own
    dnatok_shard_records.  Returns (bytes, offsets rebased to 0, record range)."""
    import numpy as np
    from paper_2601_05531_gb300 import binding
    if ws == 1:
        return data, offs, (0, len(offs) - 1)
    n, n_seq = len(data), len(offs) - 1
    g_offs = np.concatenate([offs[:-1] + i * n for i in range(ws)] + [[ws * n]]).astype(np.int64)
    bounds = binding.dnatok_shard_records(g_offs, ws)
    r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
    b0, b1 = int(g_offs[r0]), int(g_offs[r1])
    reps = np.concatenate([data] * ((b1 - 1) // n - b0 // n + 1)) if b1 > b0 else data[:0]
    mine = reps[b0 - (b0 // n) * n: b0 - (b0 // n) * n + (b1 - b0)]
    return np.ascontiguousarray(mine), g_offs[r0:r1 + 1] - b0, (r0, r1)


def _time_steps(torch, stream, step, flush_l2, steps: int):
    """CUDA-event time (ms) of each of `steps` calls of step() on `stream`,
    L2 flushed before each call, outside the events."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for i in range(steps):
        flush_l2(i)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    from paper_2601_05531_gb300 import binding

    full_data, full_offs = _workload()
    data, offs, (rec0, rec1) = _shard(full_data, full_offs, ws, rank)
    n_bytes, n_seq = len(data), len(offs) - 1
    d_bytes = torch.from_numpy(data).to(dev)
    d_offs = torch.from_numpy(offs).to(dev)
    tok = P.Tokenizer(P.KMER, k=6)
    if args.shape:
        tok.set_launch(*[int(x) for x in args.shape.split(",")])
    tok.reserve(n_bytes, n_seq)
    ids, o_out, totals = tok.alloc_outputs(n_bytes, n_seq, device=dev)
    # the direct kernel's shape (slots per step, ring depth, CTAs per SM),
    # timed on this batch by the library's autotuner and kept in its cache
    import tempfile
    tune_cache = os.path.join(tempfile.gettempdir(), "dnatok_autotune_cache.txt")
    _, tune_ms = binding.dnatok_autotune(tok.h, d_bytes.data_ptr(), n_bytes, d_offs.data_ptr(),
                                         n_seq, ids.data_ptr(), ids.numel(), o_out.data_ptr(),
                                         o_out.numel(), 3, tune_cache)
    dshape = binding.dnatok_get_direct_launch(tok.h)
    # one non-default stream for everything (graph capture needs one)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    flush_rd = torch.ones(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    flush_acc = torch.zeros(1, dtype=torch.int64, device=dev)

    def flush_l2(i):
        # a write larger than L2 evicts the inputs; the read after it leaves L2
        # holding clean lines, so the step pays no write-back of the flush
        flush.fill_(i & 255)
        flush_acc.copy_(flush_rd.sum(dtype=torch.int64).view(1))

    def plain_step():
        tok.encode(d_bytes, d_offs, ids, o_out, totals, stream=stream)

    for _ in range(max(args.warmup, 3)):
        plain_step()
    tok.sync()
    n_ids = int(totals[0].item())
    # the same encode captured once as a CUDA graph (the batched form's launch)
    binding.dnatok_graph_begin(tok.h, stream.cuda_stream)
    plain_step()
    graph = binding.dnatok_graph_end(tok.h, stream.cuda_stream)

    def graph_step():
        binding.dnatok_graph_launch(graph, stream.cuda_stream)

    sampler = ClockSampler(dev.index if ws == 1 else local)
    sampler.start()
    time.sleep(0.3)
    # warm-up steps again right before the timed ones: the GPU has just idled
    # while the clock sampler started
    for i in range(max(args.warmup, 3)):
        flush_l2(i)
        graph_step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = _time_steps(torch, stream, graph_step, flush_l2, args.steps)
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    for i in range(3):
        flush_l2(i)
        plain_step()
    plain_ms = _time_steps(torch, stream, plain_step, flush_l2, args.steps)
    tok.sync()
    assert int(totals[0].item()) == n_ids
    total_ms = sum(step_ms)

    # end to end through the public host-buffer entry point
    h_bytes = torch.from_numpy(data).pin_memory()
    h_offs = torch.from_numpy(offs).pin_memory()
    h_ooff = torch.empty(n_seq + 1, dtype=torch.int64).pin_memory()
    h_tot = torch.zeros(2, dtype=torch.int64)
    e2e_steps = max(3, min(args.steps, 10))

    def e2e_step():
        binding.dnatok_encode_host(tok.h, h_bytes.data_ptr(), n_bytes, h_offs.data_ptr(), n_seq,
                                   ids.data_ptr(), ids.numel(), h_ooff.data_ptr(), n_seq + 1,
                                   h_tot.data_ptr(), stream.cuda_stream)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    assert int(h_tot[0]) == n_ids

    # the dominant kernel's own duration: the same plain step with CUDA events
    # recorded by the library right before and after the direct k-mer kernel
    # (its launch then waits for the record plan instead of starting under it)
    binding.dnatok_set_kernel_timing(tok.h, True)
    kern_ms = []
    for i in range(args.steps + 2):
        flush_l2(i)
        plain_step()
        ms = binding.dnatok_kernel_time_ms(tok.h, stream.cuda_stream)
        if i >= 2:
            kern_ms.append(ms)
    binding.dnatok_set_kernel_timing(tok.h, False)
    tok.sync()

    sharding = None
    if ws > 1:
        # the one exchange of the sharded path: global id offsets
        g_off, g_ids = P.global_id_offsets(o_out[: n_seq + 1])
        sharding = {"records": [rec0, rec1], "global_ids": g_ids}
        t = torch.tensor([total_ms, e2e_s, sum(plain_ms)], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms, e2e_s = float(t[0]), float(t[1])
        all_ids = torch.tensor([n_ids], dtype=torch.int64, device=dev)
        torch.distributed.all_reduce(all_ids)
        job_ids = int(all_ids[0])
    else:
        job_ids = n_ids
    binding.dnatok_graph_destroy(graph)

    if rank == 0:
        peak, peak_kind = _peaks()
        alg_bytes = n_bytes + 4 * n_ids + 16 * (n_seq + 1)
        mean_s = total_ms / 1e3 / args.steps
        achieved = alg_bytes / mean_s / 1e9
        plain_mean = statistics.mean(plain_ms) / 1e3
        traffic = _traffic(n_bytes)
        kern_mean = statistics.mean(kern_ms)
        kern_achieved = alg_bytes / (kern_mean / 1e3) / 1e9
        line = {
            "metric": METRIC,
            "value": job_ids * args.steps / (total_ms / 1e3),
            "unit": "tokens/s",
            "n_gpus": ws, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": total_ms / args.steps,
            "p50_ms": statistics.median(step_ms),
            "max_ms": max(step_ms),
            "p99_ms": float(np.percentile(step_ms, 99)),
            "bytes_per_s": n_bytes * ws * args.steps / (total_ms / 1e3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_sequences": n_seq, "input_bytes": n_bytes,
                       "tokens_per_step": n_ids, "k": 6,
                       "l2": "flushed before every step (256 MB write, then 256 MB read)",
                       "launch_form": "CUDA graph replay of one dnatok_encode (value, "
                                      "roofline); plain_launch below is the same call "
                                      "launched directly",
                       "launch": {"kernel": "direct k-mer", "slots_per_step": dshape[0],
                                  "ring_steps": dshape[1], "ctas_per_sm": dshape[2],
                                  "chosen_by": "dnatok_autotune (cache %s; %s)" % (
                                      tune_cache, "timed now" if tune_ms > 0 else "cache hit")},
                       "parallelism": ("record shards x%d (dnatok_shard_records over %d "
                                       "copies of the batch)" % (ws, ws)) if ws > 1
                       else "one GPU"},
            "roofline": {"bound": "hbm", "achieved": kern_achieved, "peak": peak,
                         "unit": "GB/s", "frac": kern_achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "kernel": KERNEL,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "duration_ms": kern_mean,
                         "duration": "mean over %d steps of CUDA events recorded on the "
                                     "launching stream right before and after the direct "
                                     "k-mer kernel, L2 flushed before each step" % len(kern_ms)},
            "roofline_step": {"bound": "hbm", "achieved": achieved, "peak": peak,
                              "unit": "GB/s", "frac": achieved / peak,
                              "peak_kind": peak_kind,
                              "algorithmic_bytes_per_step": alg_bytes,
                              "duration": "CUDA events around the whole graph replay (every "
                                          "launch of the step: plan, direct kernel, gated "
                                          "general kernel)"},
            "plain_launch": {"ms_per_step": 1e3 * plain_mean,
                             "p50_ms": statistics.median(plain_ms),
                             "tokens_per_s": n_ids / plain_mean,
                             "roofline_frac": alg_bytes / plain_mean / 1e9 / peak},
            "e2e": {"value": job_ids / e2e_s, "unit": "tokens/s",
                    "h2d_bytes_per_step": n_bytes + 8 * (n_seq + 1),
                    "d2h_bytes_per_step": 8 * (n_seq + 1) + 16,
                    "ms_per_step": 1e3 * e2e_s, "api": "dnatok_encode_host (pinned host buffers)"},
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
        }
        if sharding:
            line["sharding"] = sharding
        # the host-streamed measurement runs before the oracle's worker processes
        # start, so that nothing else on the host competes with its pinned copies
        if ws == 1 and args.stream_gib > 0:
            line["host_streamed"] = _streamed(torch, P, dev, int(args.stream_gib * 2**30))
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline(data, offs)
        if ws == 1 and not args.no_extras:
            _extras(line, torch, P, dev, data, offs, d_bytes, d_offs, flush_l2, args)
        print(json.dumps(line), flush=True)
    tok.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_fasta_chunk(args):
    """Device-resident 6-mer encode of one FASTA chunk (the first
    `--fasta-chunk-mib` MiB of the seeded 8 GiB FASTA stream), the unit of work
    the host-streamed encode gives the general kernel: prints one JSON line
    with the per-encode time (CUDA events, median of --steps)."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = int(args.fasta_chunk_mib) << 20
    host = np.empty(n, dtype=np.uint8)
    synth.fasta_stream(n, seed=47, out=host)
    d = torch.from_numpy(host).to(dev)
    with P.Tokenizer(P.KMER, k=6, fmt=P.FASTA) as tok:
        ids, o, tot = tok.alloc_outputs(n, 1, device=dev)
        s = torch.cuda.current_stream()
        for _ in range(max(args.warmup, 3)):
            tok.encode(d, None, ids, o, tot, stream=s)
        tok.sync()
        evs = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            tok.encode(d, None, ids, o, tot, stream=s)
            b.record(s)
            evs.append((a, b))
        torch.cuda.synchronize()
        tok.sync()
        path = P.binding.dnatok_direct_ran(tok.h)
        us = sorted(1e3 * a.elapsed_time(b) for a, b in evs)
        med = us[len(us) // 2]
        print(json.dumps({"workload": "6-mer ids of a %d MiB FASTA chunk (device-resident)"
                                      % args.fasta_chunk_mib, "path": _FASTA_PATHS[path],
                          "median_us": med, "gb_per_s": n / (med * 1e-6) / 1e9,
                          "tokens": int(tot[0])}), flush=True)
    return 0


def run_bpe_only(args):
    """BPE encode (4096 merges) of the first `--bpe-records` records of the
    1 GiB corpus (each 2,097,152 bases), device-resident, inputs larger than L2
    from 32 records up: prints one JSON line with the median CUDA-event time of
    --steps encodes and the merge pass's repair statistics."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    data, offs = synth.bpe_apply_corpus()
    nrec = max(1, min(int(args.bpe_records), len(offs) - 1))
    data, offs = data[: offs[nrec]], offs[: nrec + 1]
    merges = np.loadtxt(os.path.join(ROOT, "tests", "golden",
                                     "bpe_merges_markov45_seed45_4096.txt"), dtype=np.int32)
    d = torch.from_numpy(data).to(dev)
    so = torch.from_numpy(offs).to(dev)
    s = torch.cuda.current_stream()
    with P.Tokenizer(P.BPE, merges=merges) as tok:
        tok.reserve(len(data), nrec)
        ids, o, tot = tok.alloc_outputs(len(data), nrec, device=dev)
        ms = _time_median(torch, lambda: tok.encode(d, so, ids, o, tot, stream=s),
                          lambda i: None, steps=args.steps, warm=max(args.warmup, 3))
        tok.sync()
        n_ids = int(tot[0].item())
        stats = P.binding.dnatok_bpe_stats(tok.h, s.cuda_stream)
    alg = len(data) + 4 * n_ids + 16 * (nrec + 1)
    print(json.dumps({"workload": "BPE (4096 merges) of %d x 2,097,152 bases" % nrec,
                      "tokens": n_ids, "ms": ms, "tokens_per_s": n_ids / (ms / 1e3),
                      "merge_pass": stats,
                      "roofline": _hbm(alg, ms, "CUDA events around one encode")}), flush=True)
    return 0


def run_next_rows(args):
    """The next rows alone on the 4096-sequence batch (overlapping and
    table-driven 6-mers, decode, reverse complement, the int64 feed): one
    JSON line with each row's median time and roofline, L2 flushed before
    every timed call."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_05531_gb300 as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    data, offs = _workload()
    d_bytes = torch.from_numpy(data).to(dev)
    d_offs = torch.from_numpy(offs).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    flush_rd = torch.ones(64 << 20, dtype=torch.int32, device=dev)
    flush_acc = torch.zeros(1, dtype=torch.int64, device=dev)

    def flush_l2(i):
        flush.fill_(i & 255)
        flush_acc.copy_(flush_rd.sum(dtype=torch.int64).view(1))

    n, n_seq = len(data), len(offs) - 1
    line = {"workload": WORKLOAD,
            "kmer6_overlap_4096seq": _overlap(torch, P, dev, d_bytes, d_offs, n, n_seq, flush_l2),
            "kmer6_table_4096seq": _ktab(torch, P, dev, d_bytes, d_offs, n, n_seq, flush_l2)}
    line.update(_decode_rc_feed(torch, P, dev, d_bytes, d_offs, n, n_seq, flush_l2))
    line.pop("feed_pipeline_embedding", None)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--shape", default=None, help="tile_bytes,threads,ctas_per_sm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the served request trace (0 = skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched / serving measurements")
    ap.add_argument("--stream-gib", type=float, default=8.0,
                    help="size of the host-streamed FASTA measurement (0 = skip)")
    ap.add_argument("--fasta-chunk-mib", type=int, default=0,
                    help="time only the device-resident encode of one FASTA chunk of this size")
    ap.add_argument("--bpe-records", type=int, default=0,
                    help="time only the BPE encode of this many records of the 1 GiB corpus")
    ap.add_argument("--next-rows", action="store_true",
                    help="time only the next rows (overlapping and table k-mers, decode, "
                         "reverse complement, feed) on the 4096-sequence batch")
    args = ap.parse_args()
    if args.next_rows:
        return run_next_rows(args)
    if args.bpe_records > 0:
        return run_bpe_only(args)
    if args.fasta_chunk_mib > 0:
        return run_fasta_chunk(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
