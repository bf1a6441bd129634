"""Host-side checks that need no GPU: the library loads and exports every
entry point its header declares; argument validation on the host."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_05531_gb300 import binding
    return binding.lib()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            names |= set(re.findall(r"DNATOK_API\s+[\w\s\*]+?\b(dnatok_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("dnatok_create", "dnatok_encode", "dnatok_destroy", "dnatok_max_tokens"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2601_05531_gb300 import binding
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", binding.lib_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (dnatok_\w+)", out))
    assert set(declared_functions()) <= exported
    # nothing but the C ABI leaves the library
    assert all(n.startswith("dnatok_") for n in exported)


def test_binding_names_match_abi(lib):
    from paper_2601_05531_gb300 import binding
    for n in declared_functions():
        assert hasattr(binding, n), n


def test_library_is_built_for_sm103a(lib):
    from paper_2601_05531_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_oracle_is_not_linked_into_library(lib):
    from paper_2601_05531_gb300 import binding
    out = subprocess.run(["nm", "-D", binding.lib_path()], capture_output=True, text=True).stdout
    assert "oracle_" not in out


def test_microbatch_rows_rule_on_host(lib):
    # Algorithm 2: b = min(B_emb, max(1, floor(M / T'))); a host-only call
    from paper_2601_05531_gb300 import binding
    cases = [((64, 100_000, 1000), 64), ((64, 10_000, 1000), 10), ((64, 999, 1000), 1),
             ((1, 10 ** 9, 7), 1), ((512, 2 ** 18, 2048), 128)]
    for args, want in cases:
        assert binding.dnatok_microbatch_rows(*args) == want, args
    for bad in ((0, 10, 10), (4, -1, 10), (4, 10, 0)):
        with pytest.raises(binding.DnatokError):
            binding.dnatok_microbatch_rows(*bad)


def test_feed_and_revcomp_reject_bad_arguments_on_host(lib):
    # argument checks happen before any CUDA call
    import ctypes
    from paper_2601_05531_gb300 import binding
    off = (ctypes.c_int64 * 2)(0, 4)
    ids = (ctypes.c_int32 * 4)()
    p_off, p_ids = ctypes.addressof(off), ctypes.addressof(ids)
    ERR_ARG = -1
    L = binding.lib()
    assert L.dnatok_feed(p_ids, p_off, 0, 1, 4, 0, 0, 2, None) == ERR_ARG        # width 2
    assert L.dnatok_feed(p_ids, p_off, 0, 1, 4, 1 << 40, 0, 4, None) == ERR_ARG  # pad > int32
    assert L.dnatok_feed(p_ids, 0, 0, 1, 4, 0, 0, 8, None) == ERR_ARG            # no offsets
    assert L.dnatok_feed(p_ids, p_off, -1, 1, 4, 0, 0, 8, None) == ERR_ARG       # row_begin < 0
    assert L.dnatok_feed(p_ids, p_off, 0, 1, 4, 0, 0, 8, None) == ERR_ARG        # no output
    assert L.dnatok_reverse_complement(0, 10, p_off, 0, 0, None) == ERR_ARG      # bytes, no records
    assert L.dnatok_reverse_complement(0, -1, p_off, 1, 0, None) == ERR_ARG      # negative size
    assert L.dnatok_reverse_complement(0, 0, p_off, 1, 0, None) == 0             # empty: nothing to do
    buf = (ctypes.c_uint8 * 32)()
    b = ctypes.addressof(buf)
    assert L.dnatok_reverse_complement(b, 16, p_off, 1, b + 8, None) == ERR_ARG  # overlapping


def test_shard_records_bounds(lib):
    # contiguous, covering, never splitting a record, and each split at the
    # first record starting at or after i * n_bytes / world
    import numpy as np
    import synth
    from paper_2601_05531_gb300 import binding
    rng = np.random.default_rng(3)
    for trial in range(50):
        n_seq = int(rng.integers(0, 300))
        lens = rng.integers(0, 5000, size=n_seq)
        lens[rng.random(n_seq) < 0.2] = 0
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        for world in (1, 2, 3, 8, 17):
            b = binding.dnatok_shard_records(offs, world)
            assert b[0] == 0 and b[-1] == n_seq and (np.diff(b) >= 0).all()
            n = int(offs[-1])
            for i in range(1, world):
                p = n * i // world
                assert b[i] == int(np.searchsorted(offs[:n_seq + 1], p, side="left")), (trial, world, i)
    # the 4096-sequence batch over 8 ranks: no shard more than one record over its share
    lens = synth.log_uniform_lengths(4096, 1000, 128000, seed=44)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    b = binding.dnatok_shard_records(offs, 8)
    sizes = offs[b[1:]] - offs[b[:-1]]
    assert sizes.max() <= offs[-1] / 8 + lens.max()
    with pytest.raises(binding.DnatokError):
        binding.dnatok_shard_records(np.array([0, 5, 3]), 2)  # decreasing
    with pytest.raises(binding.DnatokError):
        binding.dnatok_shard_records(np.array([1, 5]), 2)     # [0] != 0
