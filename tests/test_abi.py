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
    assert ctypes.sizeof(_lib.PqIndepCfg) == 40
    assert CANDIDATE_DTYPE.itemsize == 96 and WALK_STATS_DTYPE.itemsize == 48


def test_null_context_is_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    assert lib.labs_energy_batch(None, None, 13, 0, None, None, None) == 1
    assert lib.labs_flip_deltas(None, None, None, 13, 0, 0, 0, None, None) == 1


def test_legendre_family_host_enumeration(lib):
    """labs_legendre_family (host code, no device) lists exactly the (prime, rotation) pairs of its
    definition, in increasing order, and reports a short buffer as a capacity error."""
    import ctypes

    import numpy as np

    def family(L, r_lo, r_hi, t_max):
        primes = [p for p in range(2, L + 1) if all(p % d for d in range(2, int(p ** 0.5) + 1))]
        return [(p, o) for p in primes if L - p <= t_max * p for o in range(p) if r_lo <= o / L <= r_hi]

    f = lib.labs_legendre_family
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p]
    for L, r_lo, r_hi, t_max in ((450, 0.20, 0.24, 0.1), (37, 0.0, 1.0, 0.5), (101, 0.2, 0.25, 0.05)):
        want = family(L, r_lo, r_hi, t_max)
        n = ctypes.c_int64()
        assert f(L, r_lo, r_hi, t_max, None, 0, ctypes.byref(n)) == 0 and n.value == len(want)
        out = np.zeros((len(want), 2), dtype=np.int32)
        assert f(L, r_lo, r_hi, t_max, out.ctypes.data, len(want), ctypes.byref(n)) == 0
        assert [tuple(r) for r in out.tolist()] == want
        if len(want) > 1:
            short = np.zeros((1, 2), dtype=np.int32)
            assert f(L, r_lo, r_hi, t_max, short.ctypes.data, 1, ctypes.byref(n)) == 2  # LABS_ERR_CAPACITY


def test_block_split_search_narrows_to_the_first_false():
    """The merge's block-wide split search (every thread tests one of blockDim increasing points, the
    count of true answers narrows the range) returns the first index where a monotone predicate is false,
    the same answer as a binary search -- checked for ranges of every size up to a few blocks."""
    import random
    rng = random.Random(11)
    nt = 256

    def search(lo, hi, first_false):
        steps = 0
        while lo < hi:
            span = hi - lo
            dense = span <= nt
            point = (lambda k: lo + k) if dense else (lambda k: lo + (span * (k + 1)) // (nt + 1))
            np_ = span if dense else nt
            c = sum(1 for t in range(np_) if point(t) < first_false)
            nlo = point(c - 1) + 1 if c > 0 else lo
            hi = point(c) if c < np_ else hi
            lo = nlo
            steps += 1
        return lo, steps

    for _ in range(300):
        lo = rng.randrange(0, 1000)
        hi = lo + rng.choice([0, 1, 2, 255, 256, 257, rng.randrange(0, 5000), rng.randrange(0, 1 << 22)])
        ans = rng.randint(lo, hi)
        got, steps = search(lo, hi, ans)
        assert got == ans
        assert steps <= 4


def _hex_by_definition(s):
    """The paper's coding (Section 4) written out: +1 -> 1, -1 -> 0, left-padded with zeros to a multiple of
    four bits, read as one binary number, printed in hexadecimal with one digit per four bits."""
    bits = "".join("1" if v == 1 else "0" for v in s)
    nd = -(-len(s) // 4)
    return format(int(bits, 2), "0%dX" % nd)


def test_hex_coding_barker13(lib):
    """Barker 13 (+ + + + + - - + + - + - +) is 1F35 in this coding: three zero pads, then 1111100110101."""
    import numpy as np

    import paper_2409_07222_gb300 as lg
    from oracle import pm1_to_words

    s = [1, 1, 1, 1, 1, -1, -1, 1, 1, -1, 1, -1, 1]
    w = pm1_to_words(np.array(s, dtype=np.int8))
    assert lg.labs_seq_to_hex(w, 13) == "1F35"
    assert np.array_equal(lg.labs_hex_to_seq("1f35", 13), w)


@pytest.mark.parametrize("L", [1, 2, 13, 63, 64, 65, 451, 487, 527, 576])
def test_hex_coding_round_trip(lib, L):
    """Every length class (pads of 0..3 bits, one to nine words): the library's digits equal the coding
    written out from its definition, and parsing them returns the same words."""
    import numpy as np

    import paper_2409_07222_gb300 as lg
    from oracle import pm1_to_words

    rng = np.random.default_rng(L)
    for _ in range(4):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=L)
        w = pm1_to_words(s)
        h = lg.labs_seq_to_hex(w, L)
        assert h == _hex_by_definition(s)
        assert np.array_equal(lg.labs_hex_to_seq(h, L), w)


def test_hex_coding_rejects_bad_input(lib):
    import ctypes

    import numpy as np

    w = np.zeros(1, dtype=np.uint64)
    p = w.ctypes.data_as(ctypes.c_void_p)
    assert lib.labs_hex_to_seq(b"1F35", 12, p) == 1      # 12 positions take 3 digits
    assert lib.labs_hex_to_seq(b"3F35", 13, p) == 1      # a pad bit set (13 positions leave three pads)
    assert lib.labs_hex_to_seq(b"1G35", 13, p) == 1      # not a hex digit
    assert lib.labs_hex_to_seq(b"1F35", 0, p) == 1
    buf = ctypes.create_string_buffer(4)
    assert lib.labs_seq_to_hex(p, 13, buf, 4) == 2       # 4 digits need 5 bytes with the NUL
    assert lib.labs_seq_to_hex(p, 13, buf, 5 - 1) == 2
