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
