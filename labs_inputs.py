"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle's tests.

This module holds no arithmetic of the method (no correlations, energies, skew filling, flips or
fingerprints): it only draws random bits with numpy's PCG64 and lays them out in the packed format
of the library interface -- bit ``(i-1) % 64`` of word ``(i-1) // 64`` is 1 iff ``s_i = +1``, words
are zero above bit ``L-1``.

Workload recipes (the paper runs no public benchmark; these synthetic inputs stand in for its
L = 450..527 experiments):

* ``EXHAUSTIVE_37``   L=37, k=18, p=0: all 2^19 skew assignments.
* ``STEP1_451``       L=451, k=225, p=24, 256 distinct uniform prefixes (seed 2409), 65,536 walks of
                      10^5 flips, T_i = 4(L+1) = 1808, sieve rank 999 of 10^6 samples, R = 16.
* ``STEP2``           L in {451, 487, 527}, 4,096 seeds, heap 2^22, B = 4096, 10^7 expansions.
* ``MIXED``           L = 450..527, walks per length uniform in {1024..16384} (seed 2410),
                      odd L skew with p = 24, even L unrestricted, 10^4 flips per walk.
"""
import numpy as np

EXHAUSTIVE_37 = dict(L=37, p=0)
STEP1_451 = dict(L=451, p=24, n_prefix=256, prefix_seed=2409, n_walks=65536, flip_budget=100000, T_i=1808,
                 seed=2409, R=16, bloom_log2=15, bloom_k=4, n_thresh_samples=1000000, thresh_rank=999)
STEP2 = dict(lengths=(451, 487, 527), n_seeds=4096, cap=1 << 22, B=4096, max_expansions=10**7, T_u=0)
MIXED = dict(L_min=450, L_max=527, p=24, count_seed=2410, count_lo=1024, count_hi=16384, flip_budget=10**4)


def words_per_seq(L):
    return (L + 63) // 64


def _mask_tail(words, L):
    W = words_per_seq(L)
    r = L - 64 * (W - 1)
    if r < 64:
        words[..., W - 1] &= np.uint64((1 << r) - 1)
    return words


def random_words(n, L, seed):
    """n uniform +-1 sequences of length L, packed: uint64 [n, W]."""
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 2**64, size=(n, words_per_seq(L)), dtype=np.uint64)
    return _mask_tail(w, L)


def random_heads(n, L, p, prefixes, seed):
    """Packed words whose positions 1..p hold prefix (q mod n_prefix) and positions p+1..L are uniform.

    Used as the head of a skew-symmetric input: only positions 1..k+1 matter to the skew fill.
    """
    w = random_words(n, L, seed)
    if p > 0:
        pre = np.asarray(prefixes, dtype=np.uint64).reshape(-1)
        keep = np.uint64((1 << p) - 1) if p < 64 else np.uint64(2**64 - 1)
        for q in range(n):
            w[q, 0] = (w[q, 0] & ~keep) | (pre[q % len(pre)] & keep)
    return w


def distinct_prefixes(n_prefix, p, seed):
    """n_prefix distinct uniform p-bit prefixes (bit j <-> s_{j+1}), uint64 [n_prefix] (p <= 64)."""
    if p == 0:
        return np.zeros(n_prefix, dtype=np.uint64)
    if n_prefix > 2**p:
        raise ValueError("cannot draw %d distinct prefixes of %d bits" % (n_prefix, p))
    rng = np.random.default_rng(seed)
    seen, out = set(), []
    while len(out) < n_prefix:
        v = int(rng.integers(0, 2**p, dtype=np.uint64))
        if v not in seen:
            seen.add(v)
            out.append(v)
    return np.array(out, dtype=np.uint64)


def edge_words(L):
    """Edge-case inputs: all +1, all -1, alternating starting +1 / -1, one -1 at each end."""
    rows = []
    for pattern in ("plus", "minus", "alt_plus", "alt_minus", "first_minus", "last_minus"):
        bits = np.ones(L, dtype=bool)
        if pattern == "minus":
            bits[:] = False
        elif pattern == "alt_plus":
            bits[1::2] = False
        elif pattern == "alt_minus":
            bits[0::2] = False
        elif pattern == "first_minus":
            bits[0] = False
        elif pattern == "last_minus":
            bits[-1] = False
        w = np.zeros(words_per_seq(L), dtype=np.uint64)
        for i in np.nonzero(bits)[0]:
            w[i // 64] |= np.uint64(1) << np.uint64(i % 64)
        rows.append(w)
    return np.stack(rows)


def mixed_walk_counts(seed=MIXED["count_seed"], lo=MIXED["count_lo"], hi=MIXED["count_hi"],
                      L_min=MIXED["L_min"], L_max=MIXED["L_max"]):
    """{L: walks} for L = L_min..L_max, uniform in {lo..hi}."""
    rng = np.random.default_rng(seed)
    Ls = list(range(L_min, L_max + 1))
    counts = rng.integers(lo, hi + 1, size=len(Ls))
    return {L: int(c) for L, c in zip(Ls, counts)}
