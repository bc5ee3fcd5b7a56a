"""The C-ABI library builds, loads and exports every symbol include/labs.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(labs_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2409_07222_gb300 import build

    build.build()
    from paper_2409_07222_gb300 import _lib

    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert {"labs_energy_batch", "labs_flip_deltas", "labs_skew_search"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_header(lib):
    from paper_2409_07222_gb300 import _lib

    assert declared_symbols() == set(_lib.SIGNATURES)


def test_status_strings_and_version(lib):
    from paper_2409_07222_gb300 import _lib

    assert lib.labs_abi_version() >= 1
    for code, word in [(0, "ok"), (1, "invalid"), (2, "capacity"), (3, "timed out"), (4, "CUDA"), (5, "memory")]:
        assert word in _lib.status_string(code)


def test_struct_layouts_match_header():
    from paper_2409_07222_gb300 import _lib, CANDIDATE_DTYPE, WALK_STATS_DTYPE

    assert ctypes.sizeof(_lib.WalkCfg) == 104
    assert ctypes.sizeof(_lib.BatchCfg) == 72
    assert ctypes.sizeof(_lib.PqCfg) == 40
    assert CANDIDATE_DTYPE.itemsize == 96 and WALK_STATS_DTYPE.itemsize == 48


def test_null_context_is_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    assert lib.labs_energy_batch(None, None, 13, 0, None, None, None) == 1
    assert lib.labs_flip_deltas(None, None, None, 13, 0, 0, 0, None, None) == 1
