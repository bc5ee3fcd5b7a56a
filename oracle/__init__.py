"""CPU oracle for the LABS dual-step search (arXiv 2409.07222) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import this package.  The product library never imports, links or runs it, and it
shares no code with the CUDA path.

The arithmetic lives in ``labs_oracle.c`` (plain loops over +-1 arrays, int64 accumulation); this
module only marshals numpy arrays through ctypes.  The learned proposal network's fp64 reference is
in ``oracle/policy.py``.

Packed format (the interface layout): sequence ``q`` of length ``L`` occupies ``W = ceil(L/64)``
uint64 words; bit ``(i-1) % 64`` of word ``(i-1) // 64`` is 1 iff ``s_i = +1``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

INT32_MAX = 2**31 - 1
PURPOSE_WALK = 1
PURPOSE_THRESH = 2
MAX_W = 9

CANDIDATE_DTYPE = np.dtype(
    [("E", "<i4"), ("walk", "<u4"), ("step", "<u4"), ("pad", "<u4"), ("fp", "<u8"), ("seq", "<u8", (MAX_W,))]
)
assert CANDIDATE_DTYPE.itemsize == 96

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        ci = ctypes.c_int
        sig = {
            "oracle_energy_batch": (ci, [P, ci, i64, P, P]),
            "oracle_merit_factor": (f64, [ci, i64]),
            "oracle_skew_fill": (ci, [P, ci, P]),
            "oracle_is_skew": (ci, [P, ci]),
            "oracle_flip_deltas": (ci, [P, ci, i64, ci, ci, P]),
            "oracle_flip_deltas_linear": (ci, [P, ci, i64, ci, ci, P]),
            "oracle_flip_trajectory": (ci, [P, ci, ci, P, ci, P, P]),
            "oracle_sm64_at": (u64, [u64, u64]),
            "oracle_stream_key": (u64, [u64, u64, u64, u64]),
            "oracle_zobrist": (u64, [ci, ci]),
            "oracle_fingerprint_batch": (ci, [P, ci, i64, P]),
            "oracle_make_starts": (ci, [ci, ci, ci, P, ci, ci, u64, u64, i64, i64, u64, P]),
            "oracle_walk_search": (ci, [ci, ci, ci, P, ci, ci, i64, i64, i64, ci, u64, ci, ci, ci, i32, P, P, ci]),
            "oracle_walk_search_biased": (ci, [ci, ci, ci, P, ci, ci, i64, i64, i64, ci, u64, ci, ci, ci, i32, P, ci, ci,
                                               ctypes.c_float, P, P, ci]),
            "oracle_threshold": (ci, [ci, ci, ci, P, ci, ci, u64, i64, i64, P, P]),
            "oracle_skew_exhaustive": (ci, [ci, ci, P, P, P, P, P]),
            "oracle_pq_refine": (ci, [ci, P, ci, i64, ci, i64, i64, ci, P, P, P, P]),
            "oracle_sequence_operators": (ci, [P, ci, i64, P, P, P, P]),
            "oracle_legendre_construct": (ci, [ci, P, i64, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _check(status, what):
    if status != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, status))


def words_per_seq(L):
    return (L + 63) // 64


def _words(seqs, L):
    a = np.ascontiguousarray(seqs, dtype=np.uint64)
    return a.reshape(-1, words_per_seq(L))


# ---------------------------------------------------------------------------------------------
# Format helpers (interface layout, no method arithmetic)
# ---------------------------------------------------------------------------------------------
def pm1_to_words(s):
    """+-1 array(s) of shape [..., L] -> packed uint64 words [..., W]."""
    s = np.asarray(s)
    L = s.shape[-1]
    flat = s.reshape(-1, L)
    W = words_per_seq(L)
    out = np.zeros((flat.shape[0], W), dtype=np.uint64)
    for i in range(L):
        bit = (flat[:, i] == 1).astype(np.uint64) << np.uint64(i % 64)
        out[:, i // 64] |= bit
    return out.reshape(s.shape[:-1] + (W,))


def words_to_pm1(words, L):
    w = np.asarray(words, dtype=np.uint64)
    flat = w.reshape(-1, w.shape[-1])
    out = np.empty((flat.shape[0], L), dtype=np.int8)
    for i in range(L):
        out[:, i] = np.where((flat[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1), 1, -1)
    return out.reshape(w.shape[:-1] + (L,))


# ---------------------------------------------------------------------------------------------
# Section 1 definitions
# ---------------------------------------------------------------------------------------------
def energy_batch(seqs, L, with_C=False):
    w = _words(seqs, L)
    n = w.shape[0]
    E = np.empty(n, dtype=np.int32)
    C = np.empty((n, max(L - 1, 0)), dtype=np.int32) if with_C else None
    _check(lib().oracle_energy_batch(_p(w), L, n, _p(E), _p(C)), "energy_batch")
    return (E, C) if with_C else E


def merit_factor(L, E):
    return lib().oracle_merit_factor(L, int(E))


def skew_fill(head_words, L):
    w = _words(head_words, L)
    out = np.empty_like(w)
    for q in range(w.shape[0]):
        _check(lib().oracle_skew_fill(_p(w[q]), L, _p(out[q])), "skew_fill")
    return out


def is_skew(words, L):
    w = _words(words, L)
    return np.array([bool(lib().oracle_is_skew(_p(w[q]), L)) for q in range(w.shape[0])])


def flip_deltas(seqs, L, skew=False, p=0, linear=False):
    """[n, L] int32: Delta E of each neighbour (position m-1); INT32_MAX outside the free range."""
    w = _words(seqs, L)
    n = w.shape[0]
    dE = np.empty((n, L), dtype=np.int32)
    f = lib().oracle_flip_deltas_linear if linear else lib().oracle_flip_deltas
    _check(f(_p(w), L, n, int(skew), p, _p(dE)), "flip_deltas")
    return dE


def flip_trajectory(seq, L, moves, skew=False):
    w = _words(seq, L)[0].copy()
    mv = np.ascontiguousarray(moves, dtype=np.int32)
    E = np.empty(len(mv), dtype=np.int32)
    out = np.empty_like(w)
    _check(lib().oracle_flip_trajectory(_p(w), L, int(skew), _p(mv), len(mv), _p(E), _p(out)), "flip_trajectory")
    return E, out


# ---------------------------------------------------------------------------------------------
# Counter-based randomness, fingerprints, walk starts
# ---------------------------------------------------------------------------------------------
def sm64_at(key, i):
    return int(lib().oracle_sm64_at(key, i))


def stream_key(seed, purpose, a, b):
    return int(lib().oracle_stream_key(seed, purpose, a, b))


def zobrist(L):
    """[L] uint64: Z_L[i] for i = 1..L (index i-1)."""
    return np.array([lib().oracle_zobrist(L, i) for i in range(1, L + 1)], dtype=np.uint64)


def fingerprints(seqs, L):
    w = _words(seqs, L)
    out = np.empty(w.shape[0], dtype=np.uint64)
    _check(lib().oracle_fingerprint_batch(_p(w), L, w.shape[0], _p(out)), "fingerprints")
    return out


def _prefix_array(prefixes, p):
    pw = max(1, (p + 63) // 64)
    a = np.ascontiguousarray(np.asarray(prefixes, dtype=np.uint64).reshape(-1, pw))
    return a, pw


def make_starts(L, skew, p, prefixes, seed, purpose, first, n, segment=0):
    pre, pw = _prefix_array(prefixes, p)
    out = np.empty((n, words_per_seq(L)), dtype=np.uint64)
    _check(
        lib().oracle_make_starts(L, int(skew), p, _p(pre), pre.shape[0], pw, seed, purpose, first, n, segment,
                                 _p(out)),
        "make_starts",
    )
    return out


# ---------------------------------------------------------------------------------------------
# Algorithm 1 (walks), sieve threshold, exhaustive skew search, Algorithm 2
# ---------------------------------------------------------------------------------------------
def walk_search(L, skew, p, prefixes, n_walks, flip_budget, T_i, seed, R=16, bloom_log2=15, bloom_k=4,
                E_thr=INT32_MAX, walk_begin=0, n_threads=1, logits=None, chunk=64, lam=0.0):
    """Returns (candidates [n_walks, R] structured array, walk_stats [n_walks, 5] int64).

    logits (optional): float32 [n_walks, n_chunks, L] proposal logits, chunk c used for the moves made
    while the walk's flip count is in [c*chunk, (c+1)*chunk); the choice key becomes the FP32 score
    fmaf(-lam, logit, Delta E)."""
    pre, pw = _prefix_array(prefixes, p)
    out = np.zeros((n_walks, R), dtype=CANDIDATE_DTYPE)
    st = np.zeros((n_walks, 5), dtype=np.int64)
    if logits is None:
        _check(
            lib().oracle_walk_search(L, int(skew), p, _p(pre), pre.shape[0], pw, walk_begin, n_walks, flip_budget,
                                     T_i, seed, R, bloom_log2, bloom_k, int(E_thr), _p(out), _p(st), n_threads),
            "walk_search",
        )
    else:
        lg = np.ascontiguousarray(logits, dtype=np.float32)
        assert lg.shape[0] == n_walks and lg.shape[2] == L
        _check(
            lib().oracle_walk_search_biased(L, int(skew), p, _p(pre), pre.shape[0], pw, walk_begin, n_walks,
                                            flip_budget, T_i, seed, R, bloom_log2, bloom_k, int(E_thr), _p(lg),
                                            lg.shape[1], chunk, float(lam), _p(out), _p(st), n_threads),
            "walk_search_biased",
        )
    return out, st


def threshold(L, skew, p, prefixes, seed, n_samples, rank, return_samples=False):
    pre, pw = _prefix_array(prefixes, p)
    thr = np.zeros(1, dtype=np.int32)
    samples = np.empty(n_samples, dtype=np.int32) if return_samples else None
    _check(lib().oracle_threshold(L, int(skew), p, _p(pre), pre.shape[0], pw, seed, n_samples, rank, _p(thr),
                                  _p(samples)), "threshold")
    return (int(thr[0]), samples) if return_samples else int(thr[0])


def skew_exhaustive(L, p=0, prefix=0):
    pre = np.array([prefix], dtype=np.uint64)
    minE = np.zeros(1, dtype=np.int32)
    cnt = np.zeros(1, dtype=np.uint64)
    arg = np.zeros(1, dtype=np.uint64)
    words = np.zeros(words_per_seq(L), dtype=np.uint64)
    _check(lib().oracle_skew_exhaustive(L, p, _p(pre), _p(minE), _p(cnt), _p(arg), _p(words)), "skew_exhaustive")
    return int(minE[0]), int(cnt[0]), int(arg[0]), words


def pq_refine(L, seeds, cap, B, max_expansions, T_u=0, T_r=0):
    """Returns (best_words [W], best_E, best_fp, stats dict).  T_r > 0: every popped pivot also offers its
    2 T_r rotations (1..T_r elements to the left, then to the right) as candidates."""
    w = _words(seeds, L)
    best = np.zeros(words_per_seq(L), dtype=np.uint64)
    bE = np.zeros(1, dtype=np.int32)
    bfp = np.zeros(1, dtype=np.uint64)
    st = np.zeros(8, dtype=np.int64)
    _check(lib().oracle_pq_refine(L, _p(w), w.shape[0], cap, B, max_expansions, T_u, T_r, _p(best), _p(bE), _p(bfp),
                                  _p(st)), "pq_refine")
    names = ["expansions", "rounds", "survivors", "admitted", "evicted", "h_size", "improvements", "stop_reason"]
    return best, int(bE[0]), int(bfp[0]), dict(zip(names, (int(x) for x in st)))


def sequence_operators(seqs, L):
    """End-element operators: (grow [n, 4, W(L+1)], E_grow [n, 4], shrink [n, 2, W(L-1)], E_shrink [n, 2])."""
    w = _words(seqs, L)
    n = w.shape[0]
    grow = np.zeros((n, 4, words_per_seq(L + 1)), dtype=np.uint64)
    Eg = np.zeros((n, 4), dtype=np.int32)
    shrink = np.zeros((n, 2, words_per_seq(L - 1)), dtype=np.uint64)
    Es = np.zeros((n, 2), dtype=np.int32)
    _check(lib().oracle_sequence_operators(_p(w), L, n, _p(grow), _p(Eg), _p(shrink), _p(Es)), "sequence_operators")
    return grow, Eg, shrink, Es


def legendre_construct(L, params):
    """Legendre seeds for (p, off) pairs: (packed words [n, W], energies [n])."""
    pr = np.ascontiguousarray(np.asarray(params, dtype=np.int32).reshape(-1, 2))
    n = pr.shape[0]
    w = np.zeros((n, words_per_seq(L)), dtype=np.uint64)
    E = np.zeros(n, dtype=np.int32)
    _check(lib().oracle_legendre_construct(L, _p(pr), n, _p(w), _p(E)), "legendre_construct")
    return w, E
