"""Readers for the hand-written fixtures under tests/golden/."""
import codecs
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def unescape(s: str) -> bytes:
    return codecs.escape_decode(s.encode())[0]


def rows(name: str):
    """Yield the '|'-separated fields of each non-comment line."""
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if not line.strip() or line.lstrip().startswith("#"):
                continue
            yield [x.strip() for x in line.split("|")]


def keyvals(name: str):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if not line.strip() or line.lstrip().startswith("#"):
                continue
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


def ints(s: str):
    return [int(x) for x in s.split()] if s.strip() else []


def merges(s: str):
    if s.strip() in ("", "-"):
        return []
    return [tuple(int(v) for v in p.split(",")) for p in s.split(";")]
