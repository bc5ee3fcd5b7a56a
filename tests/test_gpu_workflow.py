"""Fig. 4 end to end on the device (workflow.two_step_search) against the oracle's chain of the same
stages: sieve bound -> Algorithm 1 walks -> the K best distinct candidates -> Algorithm 2 -> end-element
operators -> Algorithm 2 at L + 1 and L - 1.  Every stage is compared bit-exactly."""
import numpy as np
import pytest

import labs_inputs as inp
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INT32_MAX = 2**31 - 1


@pytest.fixture(scope="module")
def lg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_07222_gb300 as lg

    lg.load()
    return lg


def k_best_distinct(cand, K):
    """The K smallest distinct (E, fp) sieve records, the first (walk, step) of each, by (E, fp)."""
    recs = sorted((int(r["E"]), int(r["fp"]), int(r["walk"]), int(r["step"]), i)
                  for i, r in enumerate(cand.reshape(-1)) if int(r["E"]) != INT32_MAX)
    out, seen = [], set()
    for E, fp, _, _, i in recs:
        if (E, fp) not in seen:
            seen.add((E, fp))
            out.append(i)
    return cand.reshape(-1)[out[:K]]


@pytest.mark.parametrize("L,p,K,B", [(37, 4, 24, 8), (63, 6, 40, 16)])
def test_two_step_search_equals_oracle_chain(lg, L, p, K, B):
    from paper_2409_07222_gb300 import workflow

    pre = inp.distinct_prefixes(8, p, seed=L)
    n_walks, flips, seed, R = 48, 400, 11 + L, 8
    n_samples, rank = 3000, 600
    cap, H_log2, max_exp, op_exp = 2048, 16, 250, 120
    res = workflow.two_step_search(L, pre, p=p, n_walks=n_walks, flip_budget=flips, seed=seed, R=R,
                                   n_thresh_samples=n_samples, thresh_rank=rank, K=K, B=B, cap=cap, H_log2=H_log2,
                                   max_expansions=max_exp, op_max_expansions=op_exp)

    thr = oracle.threshold(L, True, p, pre, seed, n_samples, rank)
    assert res["step1"]["E_thr"] == thr
    ocand, _ = oracle.walk_search(L, True, p, pre, n_walks, flips, workflow.default_T_i(L), seed, R=R, E_thr=thr)
    oseeds = k_best_distinct(ocand, K)
    seeds = res["seeds"]
    assert len(seeds) == len(oseeds) > 1
    for f in ("E", "fp", "walk", "step", "seq"):
        assert np.array_equal(seeds[f], oseeds[f]), f

    W = oracle.words_per_seq(L)
    ob, oE, _, ost = oracle.pq_refine(L, oseeds["seq"][:, :W], cap, B, max_exp)
    assert res[L]["E"] == oE and np.array_equal(res[L]["words"], ob)
    assert res[L]["stats"]["expansions"] == ost["expansions"]
    assert res[L]["hex"] == lg.labs_seq_to_hex(ob, L)
    assert res[L]["E"] <= int(oseeds["E"][0])

    og, oEg, os_, oEs = oracle.sequence_operators(ob[None], L)
    assert res["operators"]["E_grow"] == oEg[0].tolist() and res["operators"]["E_shrink"] == oEs[0].tolist()
    for Ln, derived in ((L + 1, og.reshape(4, -1)), (L - 1, os_.reshape(2, -1))):
        ob2, oE2, _, ost2 = oracle.pq_refine(Ln, derived, cap, B, op_exp)
        assert res[Ln]["E"] == oE2 and np.array_equal(res[Ln]["words"], ob2), Ln
        assert res[Ln]["stats"]["improvements"] == ost2["improvements"], Ln
        assert abs(res[Ln]["F"] - Ln * Ln / (2 * oE2)) < 1e-12


def test_two_step_search_rejects_even_length(lg):
    from paper_2409_07222_gb300 import workflow

    with pytest.raises(ValueError):
        workflow.two_step_search(36, np.zeros(1, dtype=np.uint64), p=0)
