#!/usr/bin/env python3
"""Benchmark: non-overlapping 6-mer tokenization of 4096 DNA sequences.

Workload (seeded, synthetic): 4096 sequences with lengths log-uniform in
[1 kb, 128 kb] (about 109 MB), order-3 Markov DNA at 40% GC with N runs and
soft-masked lowercase stretches; 6-mer ids (4096 k-mers + UNK), int32.

One step = one dnatok_encode of the whole batch (one launch of the
single-pass tile kernel) with inputs resident in HBM.  L2 is flushed (a
256 MB write) before every timed step, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  N > 1 runs as torchrun ranks, one GPU each; every
rank encodes its own copy of the batch (independent shards, weak scaling, no
data-path collective); the timing takes the max over ranks.
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
KERNEL = "dnatok::tile_kernel<MODE_KMER, BSRC_LIST>"


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
    for fn in ("tile_kernel.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2601_05531_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(n_bytes_workload: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (scaled to this workload by bytes)."""
    path = os.path.join(ROOT, "profiles", "tile_kernel_kmer6_4096seq_traffic.txt")
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
                        "frac_of_h2d_peak": n_bytes / t / 1e9 / best_h2d}
            out["tokens"] = res[0]
    del host
    return out


def _cpu_baseline(data, offs, budget_s: float = 10.0):
    """The oracle as it stands, single-threaded on this host, on a bounded
    sample of the same workload (whole records, repeated until ~budget_s)."""
    import numpy as np

    import oracle
    n_seq = len(offs) - 1
    # a contiguous slice of records (~25 MB) keeps one pass near a second or two
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
    return {"value": toks / secs, "unit": "tokens/s", "cores": 1, "kind": "oracle",
            "sample": "first %d of %d sequences (%.1f MB), %d pass(es), %.1f s single-threaded"
                      % (stop, n_seq, offs[stop] / 1e6, reps, secs)}


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

    data, offs = _workload()
    n_bytes, n_seq = len(data), len(offs) - 1
    d_bytes = torch.from_numpy(data).to(dev)
    d_offs = torch.from_numpy(offs).to(dev)
    tok = P.Tokenizer(P.KMER, k=6)
    if args.shape:
        tok.set_launch(*[int(x) for x in args.shape.split(",")])
    ids, o_out, totals = tok.alloc_outputs(n_bytes, n_seq, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        tok.encode(d_bytes, d_offs, ids, o_out, totals, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    tok.sync()
    n_ids = int(totals[0].item())

    sampler = ClockSampler(dev.index if ws == 1 else local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 255)  # evict the inputs from L2 (outside the timed events)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    tok.sync()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
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

    if ws > 1:
        t = torch.tensor([total_ms, e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms, e2e_s = float(t[0]), float(t[1])

    if rank == 0:
        peak, peak_kind = _peaks()
        alg_bytes = n_bytes + 4 * n_ids + 16 * (n_seq + 1)
        mean_s = total_ms / 1e3 / args.steps
        achieved = alg_bytes / mean_s / 1e9
        traffic = _traffic(n_bytes)
        line = {
            "metric": METRIC,
            "value": n_ids * ws * args.steps / (total_ms / 1e3),
            "unit": "tokens/s",
            "n_gpus": ws, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": total_ms / args.steps,
            "p50_ms": statistics.median(step_ms),
            "p99_ms": float(np.percentile(step_ms, 99)),
            "bytes_per_s": n_bytes * ws * args.steps / (total_ms / 1e3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_sequences": n_seq, "input_bytes": n_bytes,
                       "tokens_per_step": n_ids, "k": 6, "l2": "flushed before every step",
                       "launch": list(tok.get_launch()), "parallelism": "replicas x%d" % ws},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "kernel": KERNEL,
                         "algorithmic_bytes_per_launch": alg_bytes},
            "e2e": {"value": n_ids * ws / e2e_s, "unit": "tokens/s",
                    "h2d_bytes_per_step": n_bytes + 8 * (n_seq + 1),
                    "d2h_bytes_per_step": 8 * (n_seq + 1) + 16,
                    "ms_per_step": 1e3 * e2e_s, "api": "dnatok_encode_host (pinned host buffers)"},
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline(data, offs)
        if args.stream_gib > 0:
            line["host_streamed"] = _streamed(torch, P, dev, int(args.stream_gib * 2**30))
        print(json.dumps(line), flush=True)
    tok.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--shape", default=None, help="tile_bytes,threads,ctas_per_sm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stream-gib", type=float, default=8.0,
                    help="size of the host-streamed FASTA measurement (0 = skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
