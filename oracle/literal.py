"""Literal pure-Python definitions used to brute-force check the C oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Deliberately naive:
quadratic loops, no data structures, each function a direct restatement of
the definition it names.
"""
from __future__ import annotations

BASES = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3,
         ord("a"): 0, ord("c"): 1, ord("g"): 2, ord("t"): 3}
SEPARATORS = {ord("\n"), ord("\r"), ord(" "), ord("\t")}


def bpe_greedy(word, merges):
    """Greedy BPE (reading C7): while some adjacent pair is in the table,
    merge the lowest-rank pair, leftmost occurrence first.  O(n^2 M)."""
    rank = {(int(a), int(b)): r for r, (a, b) in enumerate(merges)}
    toks = [int(x) for x in word]
    while True:
        best = None
        for i in range(len(toks) - 1):
            r = rank.get((toks[i], toks[i + 1]))
            if r is not None and (best is None or r < best[0]):
                best = (r, i)
        if best is None:
            return toks
        r, i = best
        toks[i:i + 2] = [4 + r]


def bpe_rank_sweep(word, merges):
    """The same result written as a sweep over ranks: for r = 0..M-1 replace
    every occurrence of pair r, left to right without overlap."""
    toks = [int(x) for x in word]
    for r, (a, b) in enumerate(merges):
        out, i = [], 0
        while i < len(toks):
            if i + 1 < len(toks) and toks[i] == a and toks[i + 1] == b:
                out.append(4 + r)
                i += 2
            else:
                out.append(toks[i])
                i += 1
        toks = out
    return toks


def fasta_records(data: bytes):
    """Split FASTA text into records by lines (reading C4), returning the
    list of record bodies (header lines removed, other lines kept with their
    line terminators)."""
    records = []
    lines = data.split(b"\n")
    pieces = [ln + b"\n" for ln in lines[:-1]] + ([lines[-1]] if lines[-1] else [])
    cur = None
    for ln in pieces:
        if ln.startswith(b">"):
            if cur is not None:
                records.append(cur)
            cur = b""
        else:
            if cur is None:
                cur = b""
            cur += ln
    if cur is not None:
        records.append(cur)
    return records


def kept_symbols(body: bytes):
    """Bases and N-class bytes of a record, separators removed (C1-C3):
    base -> 0..3, N-class -> None."""
    out = []
    for b in body:
        if b in SEPARATORS:
            continue
        out.append(BASES.get(b))
    return out


def kmer_ids(symbols, k: int):
    """Non-overlapping k-mers with UNK for N and for the tail (C6)."""
    unk = 4 ** k
    ids = []
    for t in range(0, len(symbols), k):
        chunk = symbols[t:t + k]
        if len(chunk) < k or any(s is None for s in chunk):
            ids.append(unk)
        else:
            ids.append(sum(4 ** (k - 1 - i) * s for i, s in enumerate(chunk)))
    return ids


def bpe_ids(symbols, merges):
    """BPE over words split at N-class symbols (C8)."""
    n_id = 4 + len(merges)
    ids, word = [], []
    for s in symbols + [None]:
        if s is None:
            if word:
                ids.extend(bpe_greedy(word, merges))
                word = []
            ids.append(n_id)
        else:
            word.append(s)
    return ids[:-1]  # drop the sentinel's N_ID


def char_ids(body: bytes, lut):
    return [int(lut[b]) for b in body if int(lut[b]) >= 0]


def kmer_overlap(data: bytes, k: int):
    """Overlapping k-mers of one record, stride 1 (reading C15): drop the
    separators, then for every start j with j + k <= L take bases j..j+k-1;
    the id is their base-4 number, or 4^k when any is not a base letter."""
    kept = [b for b in data if b not in SEPARATORS]
    out = []
    for j in range(len(kept) - k + 1):
        window = kept[j:j + k]
        if all(b in BASES for b in window):
            v = 0
            for b in window:
                v = 4 * v + BASES[b]
            out.append(v)
        else:
            out.append(4 ** k)
    return out


def kmer_table(symbols, k, kmer_lut, base_ids):
    """Reading C16 on one record's kept symbols (0..3, None for N-class):
    whole windows of k go through kmer_lut[sum 5^(k-1-i) d_i] when that entry
    is >= 0, else symbol by symbol through base_ids; a tail goes symbol by
    symbol."""
    digits = [4 if s is None else s for s in symbols]
    out = []
    n_whole = len(digits) // k
    for t in range(n_whole):
        win = digits[t * k:(t + 1) * k]
        index = 0
        for d in win:
            index = 5 * index + d
        if kmer_lut[index] >= 0:
            out.append(int(kmer_lut[index]))
        else:
            out.extend(int(base_ids[d]) for d in win)
    out.extend(int(base_ids[d]) for d in digits[n_whole * k:])
    return out


COMPLEMENT = dict(zip(b"ACGTRYKMBVDHSWNacgtrykmbvdhswn", b"TGCAYRMKVBHDSWNtgcayrmkvbhdswn"))


def reverse_complement(body: bytes) -> bytes:
    """Reading C18 on one record: reversed, each byte complemented (bytes
    outside the IUPAC letters kept)."""
    return bytes(COMPLEMENT.get(b, b) for b in reversed(body))
