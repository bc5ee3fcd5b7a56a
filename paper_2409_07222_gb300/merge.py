"""Host-side candidate merge of sharded step-1 runs (the only exchange between ranks).

Walks are independent (Section 3), so ranks run disjoint walk ids with no data-path collective; at the
end the sieved candidates of all ranks are reduced to the step-2 seeds: the K smallest distinct (E, fp)
states, the first record of each state in (walk, step) order kept.  Each rank first keeps its own K best,
which is exact: a state among the global K best has fewer than K distinct smaller states anywhere, hence
fewer than K on its own rank, and the first record of it on the rank that holds its first record overall
survives that rank's own reduction.  This module is pure record handling (no arithmetic of the method).
"""
import numpy as np

from ._lib import INT32_MAX


def topk_candidates(cand, K):
    """The K smallest distinct (E, fp) records of a candidate array (structured, the labs_candidate layout),
    ordered by (E, fp); empty slots (E = INT32_MAX) are dropped; of equal (E, fp) the record with the
    smallest (walk, step) is kept."""
    c = np.asarray(cand).reshape(-1)
    c = c[c["E"] != INT32_MAX]
    if len(c) == 0:
        return c.copy()
    c = c[np.lexsort((c["step"], c["walk"], c["fp"], c["E"]))]
    first = np.ones(len(c), dtype=bool)
    first[1:] = (c["E"][1:] != c["E"][:-1]) | (c["fp"][1:] != c["fp"][:-1])
    return c[first][:K].copy()


def merge_across_ranks(local_cand, K, group=None):
    """Reduces every rank's candidates to the global K best (see topk_candidates).  Rank 0 returns them;
    other ranks return None.  Without an initialised process group (or with one rank) it is the local
    reduction.  Works on any backend (gloo on CPUs, NCCL with the current CUDA device set)."""
    import torch.distributed as dist

    local = topk_candidates(local_cand, K)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return local
    rank = dist.get_rank(group)
    parts = [None] * dist.get_world_size(group) if rank == 0 else None
    dist.gather_object(local.tobytes(), parts, dst=0, group=group)
    if rank != 0:
        return None
    merged = np.concatenate([np.frombuffer(b, dtype=local.dtype) for b in parts])
    return topk_candidates(merged, K)
