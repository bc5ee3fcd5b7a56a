"""The two-step search of Fig. 4 as one host driver.

Step 1 (Algorithm 1) runs the skew-symmetric walks of an odd length L; every walk keeps the states whose
energy is at most the sieve bound E_l, sampled from random skew sequences of the same prefix classes.
The K best distinct candidates seed step 2 (Algorithm 2) at L.  The end-element operators (Section 3:
append or remove an element at either end) turn step 2's best sequence into four sequences of length
L + 1 and two of length L - 1, which seed step 2 again at those lengths.

Every stage is one call of the C ABI (labs_skew_search, labs_pq_refine, labs_sequence_operators,
labs_seq_to_hex); the host only hands buffers from one stage to the next.  The hand-off between the
steps is record handling on the host (merge.topk_candidates), as in the paper, where step 2 runs on CPU
cores.  With walks sharded over ranks (walk_begin = rank * n_walks, no collective in the walks), the
candidates meet at rank 0 (merge.merge_across_ranks), which alone runs step 2.
"""
import time

import numpy as np
import torch

from . import (LABS_AUTO_THRESHOLD, candidates_numpy, labs_pq_refine, labs_seq_to_hex, labs_sequence_operators,
               labs_skew_search, make_walk_cfg, pq_stats_numpy, stats_numpy, words_per_seq)
from .merge import merge_across_ranks


def default_T_i(L):
    """Walk length per segment: 8 (L + 1) / 2 flips (Section 3)."""
    return 4 * (L + 1)


def merit_factor(L, E):
    """F = L^2 / (2 E) (Eq. 1)."""
    return L * L / (2.0 * E)


def _stage(L, words, E, seconds, stats):
    w = np.ascontiguousarray(words.cpu().numpy()).view(np.uint64)[: words_per_seq(L)]
    return {"L": L, "E": int(E), "F": merit_factor(L, int(E)), "hex": labs_seq_to_hex(w, L), "words": w,
            "seconds": seconds, "stats": stats}


def _refine(L, seeds, B, cap, H_log2, max_expansions, T_u, T_r):
    t0 = time.perf_counter()
    best, bE, st = labs_pq_refine(L, seeds, B=B, cap=cap, H_log2=H_log2, max_expansions=max_expansions, T_u=T_u,
                                  T_r=T_r)
    s = pq_stats_numpy(st)
    E = int(bE.cpu()[0])  # waits for the refinement
    stats = {k: int(s[k]) for k in s.dtype.names}
    if stats["status"] != 0:
        raise RuntimeError("step 2 at L=%d returned status %d" % (L, stats["status"]))
    return best, E, time.perf_counter() - t0, stats


def two_step_search(L, prefixes, p=24, n_walks=65536, flip_budget=10**5, T_i=0, seed=2409, R=16, bloom_log2=15,
                    bloom_k=4, n_thresh_samples=10**6, thresh_rank=999, walk_begin=0, K=4096, B=4096, cap=1 << 22,
                    H_log2=28, max_expansions=10**7, T_u=0, T_r=0, op_max_expansions=None, group=None):
    """Runs Fig. 4 for one odd length L on the current CUDA device.

    prefixes: the restriction-class prefixes of step 1 (uint64 [n, ceil(p/64)], host or device).
    Returns, on rank 0, a dict with "step1" (sieve bound, candidates kept, walk statistics, seconds),
    "seeds" (the K candidates handed to step 2, structured records) and one stage dict per length L,
    L + 1 and L - 1 (best E, merit factor F, hexadecimal coding, packed words, seconds, step-2 statistics);
    on other ranks None after their share of step 1.
    """
    if L % 2 == 0 or L < 5:
        raise ValueError("step 1 searches skew-symmetric sequences: L must be odd and >= 5")
    cfg = make_walk_cfg(L, skew=True, p=p, n_walks=n_walks, flip_budget=flip_budget, T_i=T_i or default_T_i(L),
                        seed=seed, R=R, bloom_log2=bloom_log2, bloom_k=bloom_k, E_thr=LABS_AUTO_THRESHOLD,
                        n_thresh_samples=n_thresh_samples, thresh_rank=thresh_rank, walk_begin=walk_begin)
    t0 = time.perf_counter()
    cand, _, st = labs_skew_search(cfg, prefixes, with_walk_stats=False)
    s1 = stats_numpy(st)  # waits for step 1
    step1 = {k: int(s1[k]) for k in s1.dtype.names}
    step1["seconds"] = time.perf_counter() - t0
    if step1["status"] != 0:
        raise RuntimeError("step 1 returned status %d" % step1["status"])
    seeds = merge_across_ranks(candidates_numpy(cand, n_walks, R), K, group=group)
    if seeds is None:
        return None
    step1["candidates"] = int(len(seeds))
    if len(seeds) == 0:
        raise RuntimeError("the sieve kept no candidate (E_l = %d)" % step1["E_thr"])
    dev = torch.device("cuda", torch.cuda.current_device())
    W = words_per_seq(L)
    seed_words = torch.from_numpy(np.ascontiguousarray(seeds["seq"][:, :W]).view(np.int64)).to(dev)
    out = {"step1": step1, "seeds": seeds}
    best, E, sec, stats = _refine(L, seed_words, B, cap, H_log2, max_expansions, T_u, T_r)
    out[L] = _stage(L, best, E, sec, stats)
    grow, Eg, shrink, Es = labs_sequence_operators(L, best.reshape(1, -1))
    ops = {"E_grow": Eg.cpu().numpy()[0].tolist(), "E_shrink": Es.cpu().numpy()[0].tolist()}
    out["operators"] = ops
    n_op = max_expansions if op_max_expansions is None else op_max_expansions
    for Ln, derived in ((L + 1, grow.reshape(4, -1)), (L - 1, shrink.reshape(2, -1))):
        best_n, E_n, sec_n, stats_n = _refine(Ln, derived, B, cap, H_log2, n_op, T_u, T_r)
        out[Ln] = _stage(Ln, best_n, E_n, sec_n, stats_n)
    return out
