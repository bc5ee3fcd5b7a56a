"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Every check here compares the oracle with something other than itself: paper-printed values, textbook
sequences, closed forms, a library FFT / correlation, invariances of the definition, brute force on
tiny inputs, or an independently written textbook search.
"""
import heapq
import os

import numpy as np
import pytest

import labs_inputs as inp
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def np_corr(s):
    """C_1..C_{L-1} through numpy.correlate (library routine, independent of the oracle loops)."""
    s = np.asarray(s, dtype=np.int64)
    full = np.correlate(s, s, mode="full")
    return full[len(s):]


def np_energy(s):
    c = np_corr(s)
    return int(np.dot(c, c))


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------------------------
# Energy (Section 1)
# --------------------------------------------------------------------------------------------
def test_barker_sequences():
    for L_str, pattern in read_golden("barker.txt"):
        L = int(L_str)
        s = np.array([1 if ch == "+" else -1 for ch in pattern], dtype=np.int8)
        assert len(s) == L
        E, C = oracle.energy_batch(oracle.pm1_to_words(s[None]), L, with_C=True)
        assert np.all(np.abs(C[0]) <= 1), (L, C[0])
        assert int(E[0]) == L // 2


def test_barker13_is_skew_and_f():
    s = np.array([1 if ch == "+" else -1 for ch in "+++++--++-+-+"], dtype=np.int8)
    w = oracle.pm1_to_words(s[None])
    assert oracle.is_skew(w, 13)[0]
    assert abs(oracle.merit_factor(13, 6) - 14.0833) < 1e-4


@pytest.mark.parametrize("L", [1, 2, 3, 13, 63, 64, 65, 128, 129, 451, 527, 576])
def test_closed_forms(L):
    ones = np.ones(L, dtype=np.int8)
    alt = np.array([(-1) ** i for i in range(L)], dtype=np.int8)
    E, C = oracle.energy_batch(oracle.pm1_to_words(np.stack([ones, alt])), L, with_C=True)
    k = np.arange(1, L)
    assert np.array_equal(C[0], L - k)
    assert np.array_equal(C[1], ((-1) ** k) * (L - k))
    closed = (L - 1) * L * (2 * L - 1) // 6
    assert int(E[0]) == closed and int(E[1]) == closed


@pytest.mark.parametrize("L", [2, 5, 37, 64, 100, 451, 487, 527, 576])
def test_fft_identity_and_library_correlation(L):
    w = inp.random_words(8, L, seed=1000 + L)
    s = oracle.words_to_pm1(w, L).astype(np.int64)
    E, C = oracle.energy_batch(w, L, with_C=True)
    N = 1 << int(np.ceil(np.log2(2 * L)))
    for q in range(len(w)):
        assert np.array_equal(C[q], np_corr(s[q]))
        spec = np.fft.fft(s[q].astype(float), N)
        fourth = float(np.sum(np.abs(spec) ** 4)) / N  # sum over all lags of C_k^2 (Parseval)
        assert round(fourth) == L * L + 2 * int(E[q])
        assert L + 2 * int(C[q].sum()) == int(s[q].sum()) ** 2


@pytest.mark.parametrize("L", [7, 8, 64, 451])
def test_invariances_and_parity(L):
    w = inp.random_words(16, L, seed=77 + L)
    s = oracle.words_to_pm1(w, L)
    alt = np.array([(-1) ** i for i in range(L)], dtype=np.int8)
    E, C = oracle.energy_batch(w, L, with_C=True)
    Er, Cr = oracle.energy_batch(oracle.pm1_to_words(s[:, ::-1]), L, with_C=True)
    En, Cn = oracle.energy_batch(oracle.pm1_to_words(-s), L, with_C=True)
    Ea, Ca = oracle.energy_batch(oracle.pm1_to_words(s * alt), L, with_C=True)
    k = np.arange(1, L)
    assert np.array_equal(E, Er) and np.array_equal(E, En) and np.array_equal(E, Ea)
    assert np.array_equal(C, Cr) and np.array_equal(C, Cn)
    assert np.array_equal(Ca, C * ((-1) ** k))
    assert np.all((C - (L - k)) % 2 == 0)


@pytest.mark.parametrize("L", [3, 4, 5, 8, 11, 13])
def test_brute_force_minimum(L):
    n = 1 << L
    words = np.arange(n, dtype=np.uint64).reshape(n, 1)
    E = oracle.energy_batch(words, L)
    s = oracle.words_to_pm1(words[: min(n, 512)], L)
    assert all(int(E[q]) == np_energy(s[q]) for q in range(len(s)))
    if L in (3, 4, 5, 11, 13):  # Barker lengths: the optimum is the Barker energy floor(L/2)
        assert int(E.min()) == L // 2


def test_paper_printed_merit_factors():
    """Eq. (1) reproduces every merit factor the paper prints with a unique integer energy."""
    for L_str, F_str, *_ in read_golden("merit_factors.txt"):
        L, F = int(L_str), float(F_str)
        hits = [E for E in range(1, L * L) if round(oracle.merit_factor(L, E), 4) == F]
        assert len(hits) == 1, (L, F, hits)
    E455 = [E for E in range(1, 455 * 455) if round(oracle.merit_factor(455, E), 4) == 7.7835]
    E493 = [E for E in range(1, 493 * 493) if round(oracle.merit_factor(493, E), 4) == 7.7791]
    assert E455 == [13299] and E493 == [15622]


# --------------------------------------------------------------------------------------------
# Skew symmetry (Eq. 2) and restriction classes (Eq. 3)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L", [3, 13, 37, 451, 527])
def test_skew_fill_zero_odd_lags(L):
    heads = inp.random_words(12, L, seed=5 + L)
    w = oracle.skew_fill(heads, L)
    assert oracle.is_skew(w, L).all()
    _, C = oracle.energy_batch(w, L, with_C=True)
    k = np.arange(1, L)
    assert np.all(C[:, (k % 2) == 1] == 0)
    # the first k+1 elements are kept, the rest follow Eq. (2) written independently here
    s_head = oracle.words_to_pm1(heads, L)
    s = oracle.words_to_pm1(w, L)
    kk = (L - 1) // 2
    assert np.array_equal(s[:, : kk + 1], s_head[:, : kk + 1])
    for i in range(1, kk + 1):
        assert np.array_equal(s[:, kk + i], ((-1) ** i) * s[:, kk - i])


def test_skew_orbit_count_and_exhaustive_vs_brute():
    for L in (5, 7, 9, 11, 13, 15, 17, 19):
        n = 1 << L
        words = np.arange(n, dtype=np.uint64).reshape(n, 1)
        s = oracle.words_to_pm1(words, L)
        kk = (L - 1) // 2
        skew = np.ones(n, dtype=bool)
        for i in range(1, kk + 1):
            skew &= s[:, kk + i] == ((-1) ** i) * s[:, kk - i]
        E = oracle.energy_batch(words[skew], L)
        minE, count, arg, argw = oracle.skew_exhaustive(L)
        assert minE == int(E.min())
        assert count == int((E == E.min()).sum())
        assert count % 4 == 0  # orbit {s, -s, As, -As}
        assert int(oracle.energy_batch(argw[None], L)[0]) == minE
        # argmin integer: free bit j is 1 iff s_{j+1} = -1; the smallest such integer among argmins
        best_ints = []
        for q in np.nonzero(skew)[0][E == E.min()]:
            best_ints.append(sum(1 << j for j in range(kk + 1) if s[q, j] == -1))
        assert arg == min(best_ints)
    assert oracle.skew_exhaustive(13)[0] == 6  # Barker 13 is skew-symmetric


def test_exhaustive_with_prefix_restricts_space():
    L, p = 15, 3
    for prefix in range(1 << p):
        minE, count, arg, argw = oracle.skew_exhaustive(L, p, prefix)
        s = oracle.words_to_pm1(argw[None], L)[0]
        assert all((s[j] == 1) == bool((prefix >> j) & 1) for j in range(p))
    full = oracle.skew_exhaustive(L)[0]
    assert min(oracle.skew_exhaustive(L, p, x)[0] for x in range(1 << p)) == full


# --------------------------------------------------------------------------------------------
# Neighbour evaluation (Algorithm 1 / 2 flips)
# --------------------------------------------------------------------------------------------
def _np_flip_deltas(s, skew, p):
    L = len(s)
    E0 = np_energy(s)
    out = np.full(L, oracle.INT32_MAX, dtype=np.int64)
    last = (L - 1) // 2 + 1 if skew else L
    for m in range(p + 1, last + 1):
        t = s.astype(np.int64).copy()
        t[m - 1] *= -1
        if skew and L + 1 - m != m:
            t[L - m] *= -1
        out[m - 1] = np_energy(t) - E0
    return out


@pytest.mark.parametrize("L,skew,p", [(2, 0, 0), (13, 0, 0), (13, 1, 0), (13, 1, 3), (64, 0, 5), (65, 1, 8),
                                      (129, 1, 24), (451, 1, 24)])
def test_flip_deltas_definition_and_linear(L, skew, p):
    n = 3 if L > 200 else 6
    w = inp.random_words(n, L, seed=900 + L)
    if skew:
        w = oracle.skew_fill(w, L)
    d_def = oracle.flip_deltas(w, L, skew, p)
    d_lin = oracle.flip_deltas(w, L, skew, p, linear=True)
    assert np.array_equal(d_def, d_lin)
    s = oracle.words_to_pm1(w, L)
    for q in range(min(n, 2)):
        assert np.array_equal(d_def[q].astype(np.int64), _np_flip_deltas(s[q], skew, p))


@pytest.mark.parametrize("L", [13, 37, 451])
def test_flip_deltas_edge_inputs(L):
    w = inp.edge_words(L)
    d = oracle.flip_deltas(w, L, 0, 0, linear=True)
    assert np.array_equal(d, oracle.flip_deltas(w, L, 0, 0))
    ws = oracle.skew_fill(w, L)
    assert np.array_equal(oracle.flip_deltas(ws, L, 1, 0, linear=True), oracle.flip_deltas(ws, L, 1, 0))


@pytest.mark.parametrize("L,skew", [(451, 1), (452, 0)])
def test_flip_trajectory_keeps_table_exact(L, skew):
    rng = np.random.default_rng(3)
    w = inp.random_words(1, L, seed=31)
    if skew:
        w = oracle.skew_fill(w, L)
    last = (L - 1) // 2 + 1 if skew else L
    moves = rng.integers(1, last + 1, size=200)
    E, final = oracle.flip_trajectory(w, L, moves, skew=bool(skew))
    s = oracle.words_to_pm1(w, L)[0].astype(np.int64)
    for t, m in enumerate(moves):
        s[m - 1] *= -1
        if skew and L + 1 - m != m:
            s[L - m] *= -1
        if t % 50 == 49:
            assert int(E[t]) == np_energy(s)
    assert np.array_equal(oracle.words_to_pm1(final[None], L)[0], s)
    if skew:
        assert oracle.is_skew(final[None], L)[0]


# --------------------------------------------------------------------------------------------
# Counter-based generator, fingerprints, starts
# --------------------------------------------------------------------------------------------
def test_splitmix64_published_outputs():
    for idx, hexv in read_golden("splitmix64.txt"):
        assert oracle.sm64_at(0, int(idx)) == int(hexv, 16)


def test_fingerprint_is_xor_of_zobrist():
    L = 451
    Z = oracle.zobrist(L)
    assert len(set(Z.tolist())) == L
    w = inp.random_words(4, L, seed=8)
    s = oracle.words_to_pm1(w, L)
    fp = oracle.fingerprints(w, L)
    for q in range(4):
        acc = np.uint64(0)
        for i in np.nonzero(s[q] == -1)[0]:
            acc ^= Z[i]
        assert int(acc) == int(fp[q])


def test_starts_respect_prefix_and_skew():
    L, p = 451, 24
    pre = inp.distinct_prefixes(256, p, seed=2409)
    assert len(set(pre.tolist())) == 256
    st = oracle.make_starts(L, True, p, pre, seed=2409, purpose=oracle.PURPOSE_WALK, first=0, n=512)
    s = oracle.words_to_pm1(st, L)
    assert oracle.is_skew(st, L).all()
    for q in range(512):
        pv = int(pre[q % 256])
        assert all((s[q, j] == 1) == bool((pv >> j) & 1) for j in range(p))
    # free elements look uniform
    kk = (L - 1) // 2
    frac = (s[:, p: kk + 1] == 1).mean()
    assert 0.47 < frac < 0.53


# --------------------------------------------------------------------------------------------
# Algorithm 1 (walks)
# --------------------------------------------------------------------------------------------
def _replay_walk(L, skew, p, prefix, seed, w, budget, T_i, E_thr, R):
    """Independent set-based replay of one walk (exact visited set instead of a Bloom filter)."""
    last = (L - 1) // 2 + 1 if skew else L
    Z = [0] + [int(z) for z in oracle.zobrist(L)]
    flips, seg = 0, 0
    slots = {}
    while flips < budget:
        start = oracle.make_starts(L, skew, p, np.array([prefix], dtype=np.uint64), seed, oracle.PURPOSE_WALK,
                                   first=w, n=1, segment=seg)
        # make_starts indexes the prefix by id mod n_prefix; with one prefix that is the walk's own
        s = oracle.words_to_pm1(start, L)[0].astype(np.int64)
        seg += 1
        fp = 0
        for i in range(L):
            if s[i] == -1:
                fp ^= Z[i + 1]
        visited = {fp}
        E = np_energy(s)
        it = 0
        while it < T_i and flips < budget:
            it += 1
            best = None
            for m in range(p + 1, last + 1):
                F = [m] if (not skew or L + 1 - m == m) else [m, L + 1 - m]
                nfp = fp
                for f in F:
                    nfp ^= Z[f]
                if nfp in visited:
                    continue
                t = s.copy()
                for f in F:
                    t[f - 1] *= -1
                d = np_energy(t) - E
                if best is None or d < best[0]:
                    best = (d, m, F, nfp)
            if best is None:
                break
            d, m, F, fp = best
            for f in F:
                s[f - 1] *= -1
            visited.add(fp)
            E += d
            flips += 1
            if E <= E_thr and fp not in slots:
                slots[fp] = (E, flips)
    items = sorted((E, fp, st) for fp, (E, st) in slots.items())[:R]
    return items


@pytest.mark.parametrize("L,skew,p", [(13, 1, 0), (15, 1, 2), (12, 0, 0)])
def test_walk_matches_independent_replay(L, skew, p):
    prefix = 0b10 if p else 0
    budget, T_i, R = 40, 9, 6
    E_thr = 10**6
    for w in range(3):
        cands, st = oracle.walk_search(L, skew, p, np.array([prefix], dtype=np.uint64), 1, budget, T_i, seed=99,
                                       R=R, bloom_log2=22, bloom_k=4, E_thr=E_thr, walk_begin=w)
        got = [(int(c["E"]), int(c["fp"]), int(c["step"])) for c in cands[0] if c["E"] != oracle.INT32_MAX]
        exp = _replay_walk(L, skew, p, prefix, 99, w, budget, T_i, E_thr, R)
        # the replay keeps the first visit of each state; the oracle keeps the first visit among its slots
        assert [(E, fp) for E, fp, _ in got] == [(E, fp) for E, fp, _ in exp]
        assert int(st[0, 0]) == budget


def test_walk_invariants_L451():
    L, p = 451, 24
    pre = inp.distinct_prefixes(4, p, seed=11)
    cands, st = oracle.walk_search(L, 1, p, pre, 2, 300, 120, seed=5, R=8, E_thr=oracle.INT32_MAX - 1)
    for w in range(2):
        assert int(st[w, 0]) == 300 and int(st[w, 1]) == 3
        valid = cands[w][cands[w]["E"] != oracle.INT32_MAX]
        assert len(valid) == 8
        assert np.all(np.diff(valid["E"]) >= 0)
        seqs = valid["seq"][:, :8]
        assert oracle.is_skew(seqs, L).all()
        assert np.array_equal(oracle.energy_batch(seqs, L), valid["E"])
        assert np.array_equal(oracle.fingerprints(seqs, L), valid["fp"])
        s = oracle.words_to_pm1(seqs, L)
        pv = int(pre[w % 4])
        assert all((s[:, j] == 1).tolist() == [bool((pv >> j) & 1)] * len(s) for j in range(p))
        assert len(set(valid["fp"].tolist())) == len(valid)
        assert int(st[w, 4]) == int(valid["E"][0])


# --------------------------------------------------------------------------------------------
# Sieve threshold
# --------------------------------------------------------------------------------------------
def test_threshold_is_nearest_rank_of_samples():
    L, p = 101, 8
    pre = inp.distinct_prefixes(16, p, seed=4)
    thr, samples = oracle.threshold(L, True, p, pre, seed=7, n_samples=5000, rank=4, return_samples=True)
    starts = oracle.make_starts(L, True, p, pre, 7, oracle.PURPOSE_THRESH, 0, 5000)
    s = oracle.words_to_pm1(starts, L)
    direct = np.array([np_energy(x) for x in s[:200]])
    assert np.array_equal(samples[:200], direct)
    assert thr == int(np.sort(samples)[4])


# --------------------------------------------------------------------------------------------
# Algorithm 2 (priority queue)
# --------------------------------------------------------------------------------------------
def _textbook_pq(L, seeds_pm1, max_expansions, T_r=0):
    """Algorithm 2 with B = 1: a heapq best-first search with an exact hash set of visited states; with
    T_r > 0 every pivot also offers its rotations by 1..T_r elements left (s[r:] + s[:r]) and right
    (s[-r:] + s[:-r])."""
    Z = [int(z) for z in oracle.zobrist(L)]

    def fp_of(s):
        h = 0
        for i, v in enumerate(s):
            if v == -1:
                h ^= Z[i]
        return h

    heap, H = [], set()
    best = None
    for s in seeds_pm1:
        s = tuple(int(v) for v in s)
        key = (np_energy(s), fp_of(s))
        if key[1] in H:
            continue
        H.add(key[1])
        heapq.heappush(heap, (key, s))
        if best is None or key < best:
            best = key
    exp = 0
    while heap and exp < max_expansions:
        (E, fp), s = heapq.heappop(heap)
        exp += 1
        kids = []
        for i in range(L):
            nfp = fp ^ Z[i]
            if nfp in H:
                continue
            t = list(s)
            t[i] = -t[i]
            kids.append(((np_energy(t), nfp), tuple(t)))
        rots = [s[r:] + s[:r] for r in range(1, T_r + 1)] + [s[-r:] + s[:-r] for r in range(1, T_r + 1)]
        for t in rots:
            rfp = fp_of(t)
            if rfp not in H:
                kids.append(((np_energy(t), rfp), tuple(t)))
        kids.sort()
        for key, t in kids:
            if key[1] in H:
                continue
            H.add(key[1])
            heapq.heappush(heap, (key, t))
        if kids and kids[0][0][0] < best[0]:
            best = kids[0][0]
    return best, exp


@pytest.mark.parametrize("L", [9, 12])
def test_pq_b1_equals_textbook_best_first(L):
    seeds = inp.random_words(3, L, seed=40 + L)
    best_w, best_E, best_fp, st = oracle.pq_refine(L, seeds, cap=1 << 20, B=1, max_expansions=60)
    exp_best, exp_n = _textbook_pq(L, oracle.words_to_pm1(seeds, L), 60)
    assert (best_E, best_fp) == exp_best
    assert st["expansions"] == exp_n
    assert int(oracle.energy_batch(best_w[None], L)[0]) == best_E


@pytest.mark.parametrize("L,T_r", [(9, 1), (12, 3), (15, 7)])
def test_pq_rotations_b1_equal_textbook(L, T_r):
    """MAKE_ROTATIONS: with B = 1 the oracle's search with rotations equals the textbook best-first search
    that also pushes each pivot's 2 T_r rotations."""
    seeds = inp.random_words(2, L, seed=70 + L)
    best_w, best_E, best_fp, st = oracle.pq_refine(L, seeds, cap=1 << 20, B=1, max_expansions=50, T_r=T_r)
    exp_best, exp_n = _textbook_pq(L, oracle.words_to_pm1(seeds, L), 50, T_r=T_r)
    assert (best_E, best_fp) == exp_best
    assert st["expansions"] == exp_n
    assert int(oracle.energy_batch(best_w[None], L)[0]) == best_E
    # rotations add visited states beyond the flips
    _, _, _, st0 = oracle.pq_refine(L, seeds, cap=1 << 20, B=1, max_expansions=50)
    assert st["h_size"] > st0["h_size"]


def test_pq_reaches_global_optimum_l13():
    seeds = inp.random_words(2, 13, seed=1)
    best_w, best_E, _, st = oracle.pq_refine(13, seeds, cap=1 << 14, B=64, max_expansions=1 << 13)
    assert best_E == 6  # Barker-13 energy, the optimum at L = 13
    assert st["h_size"] <= 1 << 13


def test_pq_batch_invariants():
    L = 31
    seeds = inp.random_words(8, L, seed=2)
    _, E_small, _, st_small = oracle.pq_refine(L, seeds, cap=64, B=8, max_expansions=400)
    _, E_big, _, st_big = oracle.pq_refine(L, seeds, cap=1 << 16, B=8, max_expansions=400)
    seedE = oracle.energy_batch(seeds, L)
    assert E_small <= seedE.min() and E_big <= seedE.min()
    assert st_small["expansions"] == 400 and st_big["expansions"] == 400
    assert st_small["evicted"] > 0
    assert st_big["admitted"] + 8 == st_big["h_size"]


_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def _sm64_py(key, i):
    """Output i of SplitMix64 started at `key` (Steele, Lea & Flood 2014), written out in Python."""
    z = (key + (i + 1) * _GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _zobrist_py(L):
    key = _sm64_py(_sm64_py(_sm64_py(0, 0x5A0B), L), 0)
    return [None] + [_sm64_py(key, i - 1) for i in range(1, L + 1)]


def _batch_pq(L, seeds_pm1, cap, B, max_exp, T_u=0, T_r=0):
    """Algorithm 2 in its batch-synchronous reading, restated with Python lists and sets: every round
    pops the b smallest (E, fp) keys, scores every flip child (and, with T_r, every rotation) that is not
    in H from scratch, orders the children by (E, fp, pop, position) keeping the first of each (E, fp),
    improves the best on a strict E decrease, then keeps the cap smallest of (rest of the queue u children)
    and puts exactly the admitted children into H.  Energies by numpy, fingerprints as XOR of Zobrist keys
    computed from the SplitMix64 definition -- nothing shared with the C oracle."""
    Z = _zobrist_py(L)

    def fp_of(s):
        f = 0
        for i, v in enumerate(s, 1):
            if v == -1:
                f ^= Z[i]
        return f

    seen = {}
    for s in seeds_pm1:
        s = tuple(int(v) for v in s)
        seen[(np_energy(list(s)), fp_of(s))] = s
    P = sorted((k[0], k[1], v) for k, v in seen.items())[:cap]
    H = {fp for _, fp, _ in P}
    best = P[0]
    st = dict(expansions=0, rounds=0, survivors=0, admitted=0, evicted=0, improvements=0)
    u, stop = 0, 0
    while True:
        if st["expansions"] >= max_exp:
            stop = 1
            break
        if not P:
            stop = 2
            break
        if T_u > 0 and u >= T_u:
            stop = 3
            break
        b = min(B, len(P), max_exp - st["expansions"])
        popped, rest = P[:b], P[b:]
        children = []
        for pop, (_, _, s) in enumerate(popped):
            kids = [(i, s[:i - 1] + (-s[i - 1],) + s[i:]) for i in range(1, L + 1)]
            kids += [(L + r, s[r:] + s[:r]) for r in range(1, T_r + 1)]               # first r to the end
            kids += [(L + T_r + r, s[-r:] + s[:-r]) for r in range(1, T_r + 1)]       # last r to the start
            for pos, c in kids:
                f = fp_of(c)
                if f not in H:
                    children.append((np_energy(list(c)), f, pop, pos, c))
        children.sort(key=lambda t: t[:4])
        uniq, keys = [], set()
        for t in children:
            if (t[0], t[1]) not in keys:
                keys.add((t[0], t[1]))
                uniq.append(t)
        st["survivors"] += len(uniq)
        if uniq and uniq[0][0] < best[0]:
            best = (uniq[0][0], uniq[0][1], uniq[0][4])
            st["improvements"] += 1
            u = 0
        else:
            u += b
        merged = sorted([(E, f, s, False) for E, f, s in rest] + [(E, f, c, True) for E, f, _, _, c in uniq],
                        key=lambda t: (t[0], t[1]))[:cap]
        new = [t for t in merged if t[3]]
        H |= {t[1] for t in new}
        st["admitted"] += len(new)
        st["evicted"] += len(rest) - (len(merged) - len(new))
        P = [(E, f, s) for E, f, s, _ in merged]
        st["expansions"] += b
        st["rounds"] += 1
    st["h_size"] = len(H)
    st["stop_reason"] = stop
    return best, st


@pytest.mark.parametrize("L,n_seeds,cap,B,max_exp,T_u,T_r", [
    (15, 6, 10, 4, 80, 0, 0),      # a cap that evicts every round
    (21, 9, 25, 7, 140, 30, 0),    # T_u stop
    (13, 5, 9, 5, 100, 0, 2),      # rotations with eviction
    (6, 4, 8, 3, 10_000, 0, 0),    # the queue runs empty (every state of L = 6 visited)
    (17, 12, 4, 16, 90, 0, 1),     # B above the cap, more seeds than the cap
])
def test_pq_batch_path_equals_restatement(L, n_seeds, cap, B, max_exp, T_u, T_r):
    """The oracle's B > 1 / finite-cap path (eviction, survivors, admitted, evicted, H size) equals the
    independent restatement of the batch round: best key and sequence and all eight counters."""
    seeds = inp.random_words(n_seeds, L, seed=500 + L)
    seeds = np.concatenate([seeds, seeds[:1]])  # a duplicate seed is kept once
    best_w, best_E, best_fp, st = oracle.pq_refine(L, seeds, cap=cap, B=B, max_expansions=max_exp, T_u=T_u, T_r=T_r)
    (eE, efp, es), est = _batch_pq(L, oracle.words_to_pm1(seeds, L), cap, B, max_exp, T_u=T_u, T_r=T_r)
    assert (best_E, best_fp) == (eE, efp)
    assert tuple(int(v) for v in oracle.words_to_pm1(best_w[None], L)[0]) == es
    for k in ("expansions", "rounds", "survivors", "admitted", "evicted", "h_size", "improvements", "stop_reason"):
        assert st[k] == est[k], (k, st[k], est[k])
    if cap < 20 and max_exp < 1000:
        assert st["evicted"] > 0


# --------------------------------------------------------------------------------------------
# End-element sequence operators (Fig. 4 loop back into step 2)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L", [3, 13, 64, 65, 127, 128, 451, 575])
def test_sequence_operators_by_slicing(L):
    """The six results equal the operators written with list slicing, and their energies equal the
    energy of those lists computed with numpy."""
    seqs = inp.random_words(5, L, seed=L + 7)
    grow, Eg, shrink, Es = oracle.sequence_operators(seqs, L)
    for q, s in enumerate(oracle.words_to_pm1(seqs, L)):
        s = list(int(v) for v in s)
        want_g = [s + [1], s + [-1], [1] + s, [-1] + s]
        want_s = [s[:-1], s[1:]]
        for v, t in enumerate(want_g):
            assert list(oracle.words_to_pm1(grow[q, v][None], L + 1)[0]) == t
            assert Eg[q, v] == np_energy(t)
        for v, t in enumerate(want_s):
            assert list(oracle.words_to_pm1(shrink[q, v][None], L - 1)[0]) == t
            assert Es[q, v] == np_energy(t)


# --------------------------------------------------------------------------------------------
# Legendre seeds (Section 4, Table 2)
# --------------------------------------------------------------------------------------------
def _primes(n):
    return [p for p in range(2, n + 1) if all(p % d for d in range(2, int(p ** 0.5) + 1))]


def _legendre_family(L, r_lo=0.20, r_hi=0.24, t_max=0.1):
    """Every prime p <= L with L - p <= t_max p, every rotation off < p with r_lo <= off / L <= r_hi."""
    return [(p, off) for p in _primes(L) if L - p <= t_max * p for off in range(p) if r_lo <= off / L <= r_hi]


@pytest.mark.parametrize("p", [7, 11, 19, 23, 43, 431, 443, 467, 491])
def test_legendre_periodic_autocorrelation(p):
    """For a prime p = 3 (mod 4) every non-trivial periodic autocorrelation of the Legendre sequence is -1;
    for p = 1 (mod 4) they lie in {1, -3} (classical two-valued property of quadratic-residue sequences)."""
    w, _ = oracle.legendre_construct(p, [(p, 0)])
    s = oracle.words_to_pm1(w, p)[0].astype(np.int64)
    R = [int(np.dot(s, np.roll(s, -k))) for k in range(1, p)]
    assert set(R) == ({-1} if p % 4 == 3 else {1, -3})


def test_legendre_table2_construction_column():
    """The best seed of the family at each tabulated length has exactly the printed merit factor."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "legendre_table2.txt")) if l.strip() and not l.startswith("#")]
    for L_s, F_s in rows:
        L = int(L_s)
        fam = _legendre_family(L)
        _, E = oracle.legendre_construct(L, fam)
        best = int(E.min())
        assert round(L * L / (2 * best), 4) == float(F_s), (L, best)
