"""The allocation-free sieve bound (labs_sample_threshold_noalloc) agrees with labs_sample_threshold.

Callers that may not allocate device memory (an application whose allocator owns every device byte,
or one that cannot afford cudaMalloc's synchronisation) use this entry point; it keeps its scratch in a
fixed device array of the library.  This file is collected last so that a failure here leaves every
other test already run; it passes alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import labs_inputs as inp
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_07222_gb300 as lg

    lg.load()
    return lg


def test_noalloc_matches_threshold_on_two_calls(lg):
    cases = [
        (451, True, 24, 2409, 1_000_000, 999),  # the sieve sample of the L=451 walks
        (101, True, 8, 7, 5_000, 4_999),        # a smaller second call: leftovers must not leak in
    ]
    for L, skew, p, seed, n, rank in cases:
        pre = inp.distinct_prefixes(16 if p else 1, p, seed=seed) if p else np.zeros(1, dtype=np.uint64)
        got = lg.labs_sample_threshold_noalloc(L, skew, p, pre, seed, n, rank)
        exp = lg.labs_sample_threshold(L, skew, p, pre, seed, n, rank)
        torch.cuda.synchronize()
        assert int(got.cpu()[0]) == int(exp.cpu()[0]), (L, n, rank)


def test_noalloc_matches_the_oracle(lg):
    """The sieve bound of the fixed-scratch entry point equals the oracle's nearest-rank sample bound
    directly (not only through the allocating entry point), on a sample the oracle finishes in seconds."""
    for L, skew, p, seed, n, rank in [(451, True, 24, 2409, 20_000, 19), (101, True, 8, 7, 5_000, 4_999),
                                      (64, False, 5, 3, 3_001, 1_500)]:
        pre = inp.distinct_prefixes(16, p, seed=seed)
        got = lg.labs_sample_threshold_noalloc(L, skew, p, pre, seed, n, rank)
        torch.cuda.synchronize()
        assert int(got.cpu()[0]) == oracle.threshold(L, skew, p, pre, seed, n, rank), (L, n, rank)


def test_noalloc_rejects_sizes_beyond_its_scratch(lg):
    from paper_2409_07222_gb300 import _lib

    pre = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lg.load().labs_sample_threshold_noalloc(451, 1, 0, ctypes.c_void_p(pre.data_ptr()), 1, 1, (1 << 20) + 1, 0,
                                                 ctypes.c_void_p(out.data_ptr()), st)
    assert rc == _lib.LABS_ERR_CAPACITY
