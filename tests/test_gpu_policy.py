"""The learned proposal network's CUDA kernels against the fp64 oracle (oracle/policy.py).

Weights are BF16 on the device: the oracle is evaluated at the same BF16-rounded weights (biases stay
FP32), so the remaining difference is FP32 accumulation order.  Tolerance: max |GPU - oracle| <= 1e-3 of
the largest |oracle| entry of each tensor (forward logits and every gradient tensor).
"""
import numpy as np
import pytest

import labs_inputs as inp
import oracle
from oracle import policy as opol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ORDER = ["w1", "b1", "w2", "b2", "w3", "b3", "W4", "b4", "W5", "b5"]


@pytest.fixture(scope="module")
def lg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_07222_gb300 as lg

    lg.load()
    return lg


def _params(L, seed):
    p = opol.init_params(L, seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(size=p[k].shape) * 0.05
    flat = np.concatenate([p[k].reshape(-1) for k in ORDER]).astype(np.float32)
    # the values the device computes with: BF16 weights, FP32 biases
    q = {}
    o = 0
    for k in ORDER:
        n = p[k].size
        v = torch.from_numpy(flat[o:o + n].copy())
        if not k.startswith("b"):
            v = v.to(torch.bfloat16)
        q[k] = v.to(torch.float64).numpy().reshape(p[k].shape)
        o += n
    return flat, q


def _batch(L, n, seed):
    w = inp.random_words(n, L, seed=seed)
    s = oracle.words_to_pm1(w, L)
    _, C = oracle.energy_batch(w, L, with_C=True)
    return w, opol.features(s, C)


def _close(got, exp, tol=1e-3):
    scale = max(1e-12, float(np.max(np.abs(exp))))
    return float(np.max(np.abs(got - exp))) <= tol * scale


@pytest.mark.parametrize("L,n", [(13, 5), (64, 3), (200, 130), (451, 2), (576, 3)])
def test_forward_matches_oracle(lg, L, n):
    """The tensor-core inference path against the plain fp64 forward of the network at the same
    BF16-rounded weights, activations unrounded.  The device stores the three convolution outputs as BF16
    (8-bit significand, relative rounding error at most 2^-9 each), so the bound is the BF16-mode
    tolerance, 2e-2 of the largest |logit|.  A second, tighter check evaluates the oracle with those three
    stored activations rounded to BF16 as well: what remains is FP32 summation order, within 2e-3.  Sizes
    span one to five 128-position tiles per sample, a ragged last tile and two 128-sample dense tiles."""
    flat, q = _params(L, 3)
    w, x = _batch(L, n, 7)
    pol = lg.Policy(L)
    pol.set_params(flat)
    got = pol.forward(torch.from_numpy(w.view(np.int64)).cuda()).cpu().numpy()
    exp, _ = opol.forward(q, x)
    assert _close(got, exp, tol=2e-2), float(np.max(np.abs(got - exp)) / np.max(np.abs(exp)))
    exp_stored, _ = opol.forward(q, x, act_bf16=True)
    assert _close(got, exp_stored, tol=2e-3), float(np.max(np.abs(got - exp_stored)) / np.max(np.abs(exp_stored)))


def test_forward_chunks_and_batch_independence(lg):
    """More samples than one inference chunk (8,192): every row equals the same sequence's logits from a
    small batch, bit for bit (no cross-sample state; a summation order that does not depend on the batch)."""
    L, n = 13, 8300
    w = inp.random_words(n, L, seed=31)
    pol = lg.Policy(L, seed=5)
    allw = torch.from_numpy(w.view(np.int64)).cuda()
    full = pol.forward(allw)
    for lo, hi in ((0, 7), (8188, 8198), (8293, 8300)):
        assert torch.equal(full[lo:hi], pol.forward(allw[lo:hi]))


@pytest.mark.parametrize("L,n,lo,hi", [(13, 6, 2, 6), (37, 9, 0, 18), (451, 4, 24, 225)])
def test_gradients_match_oracle(lg, L, n, lo, hi):
    flat, q = _params(L, 5)
    w, x = _batch(L, n, 11)
    rng = np.random.default_rng(2)
    target = rng.integers(lo, hi + 1, size=n).astype(np.int32)
    weight = rng.uniform(0.2, 2.0, size=n).astype(np.float32)
    pol = lg.Policy(L)
    pol.set_params(flat)
    loss, g = pol.train_step(torch.from_numpy(w.view(np.int64)).cuda(), target, weight, lo, hi, lr=0.0, want_grads=True)
    free = np.zeros((n, L), dtype=bool)
    free[:, lo:hi + 1] = True
    eloss, eg, _ = opol.loss_and_grads(q, x, free, target.astype(np.int64), weight.astype(np.float64))
    assert abs(float(loss.cpu()[0]) - eloss) <= 1e-3 * max(1.0, abs(eloss))
    g = g.cpu().numpy()
    o = 0
    for k in ORDER:
        m = eg[k].size
        assert _close(g[o:o + m].reshape(eg[k].shape), eg[k]), k
        o += m
    # lr = 0 leaves the parameters untouched
    assert np.array_equal(pol.get_params().cpu().numpy(), flat)


def test_adam_steps_reduce_the_loss(lg):
    L, n = 37, 32
    w, _ = _batch(L, n, 13)
    target = np.random.default_rng(4).integers(0, 19, size=n).astype(np.int32)
    weight = np.ones(n, dtype=np.float32)
    pol = lg.Policy(L, seed=9)
    seqs = torch.from_numpy(w.view(np.int64)).cuda()
    losses = [float(pol.train_step(seqs, target, weight, 0, 18, lr=1e-3)[0].cpu()[0]) for _ in range(40)]
    assert losses[-1] < 0.5 * losses[0]


def test_adam_matches_restatement_and_refreshes_bf16(lg):
    """Two optimizer steps equal the float32 Adam restatement applied to the GPU's own gradients, and the
    BF16 weight copy the forward uses is refreshed: logits after the steps equal those of a network set
    to the expected parameters."""
    L, n, lr = 29, 16, 3e-3
    w, _ = _batch(L, n, 21)
    target = np.random.default_rng(6).integers(0, 14, size=n).astype(np.int32)
    weight = np.random.default_rng(7).uniform(0.2, 2.0, size=n).astype(np.float32)
    pol = lg.Policy(L, seed=12)
    seqs = torch.from_numpy(w.view(np.int64)).cuda()
    p = pol.get_params().cpu().numpy()
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    for t in (1, 2):
        _, g = pol.train_step(seqs, target, weight, 0, 14, lr=lr, want_grads=True)
        p, m1, m2 = opol.adam_step(p, g.cpu().numpy(), m1, m2, t, lr)
    got = pol.get_params().cpu().numpy()
    assert np.max(np.abs(got - p)) <= 1e-6, np.max(np.abs(got - p))
    ref = lg.Policy(L, seed=0)
    ref.set_params(got)
    assert torch.equal(pol.forward(seqs), ref.forward(seqs))


# ------------------------------------------------------------------------------------------------
# Chunked and learned walks (labs_chunked_search)
# ------------------------------------------------------------------------------------------------
def _walk_cfg(lg, L, p, n, budget, T_i, seed, R):
    return lg.make_walk_cfg(L, skew=L % 2 == 1, p=p, n_walks=n, flip_budget=budget, T_i=T_i, seed=seed, R=R,
                            E_thr=2**31 - 1)


@pytest.mark.parametrize("chunk", [64, 37, 1000])
def test_chunked_without_policy_equals_plain_walks(lg, chunk):
    L, p, n, budget, T_i = 451, 24, 24, 300, 128
    pre = inp.distinct_prefixes(256, p, seed=2409)
    cfg = _walk_cfg(lg, L, p, n, budget, T_i, 2409, 8)
    out, ws, st = lg.labs_skew_search(cfg, pre)
    res = lg.labs_chunked_search(cfg, pre, chunk=chunk)
    torch.cuda.synchronize()
    assert torch.equal(out, res["out"])
    assert torch.equal(ws, res["walk_stats"])
    assert lg.stats_numpy(st)["flips"] == lg.stats_numpy(res["stats"])["flips"] == n * budget


@pytest.mark.parametrize("L,p,lam", [(101, 8, 3.0), (451, 24, 40.0), (100, 0, 5.0)])
def test_learned_walks_replay_in_oracle(lg, L, p, lam):
    """The GPU's logged logits replayed in the oracle give bit-identical moves, energies and statistics."""
    n, budget, T_i, chunk = 12, 260, 100, 64
    pre = inp.distinct_prefixes(64, p, seed=5) if p else np.zeros(1, dtype=np.uint64)
    cfg = _walk_cfg(lg, L, p, n, budget, T_i, 77, 6)
    pol = lg.Policy(L, seed=3)
    res = lg.labs_chunked_search(cfg, pre, policy=pol, lam=lam, chunk=chunk, log_logits=True)
    torch.cuda.synchronize()
    logits = res["logits"].cpu().numpy().transpose(1, 0, 2).copy()  # [n, n_chunks, L]
    assert np.isfinite(logits).all() and logits.std() > 0
    cand = lg.candidates_numpy(res["out"], n, 6)
    oc, ost = oracle.walk_search(L, L % 2 == 1, p, pre, n, budget, T_i, 77, R=6, n_threads=8, logits=logits,
                                 chunk=chunk, lam=lam)
    for f in ("E", "walk", "step", "fp", "seq"):
        assert np.array_equal(cand[f], oc[f]), f
    assert np.array_equal(res["walk_stats"].cpu().numpy()[:, :5], ost)
    # the bias changed the walk: the plain walk differs
    pc, _ = oracle.walk_search(L, L % 2 == 1, p, pre, n, budget, T_i, 77, R=6, n_threads=8)
    assert not np.array_equal(pc["fp"], oc["fp"])


def test_training_is_deterministic(lg):
    """Training sums in a fixed order (no floating-point atomics): two networks trained on the same
    batches from the same initial weights agree bit for bit, losses included."""
    L, n = 41, 40
    w, _ = _batch(L, n, 17)
    target = np.random.default_rng(2).integers(5, 20, size=n).astype(np.int32)
    weight = np.random.default_rng(3).uniform(0.1, 1.0, size=n).astype(np.float32)
    seqs = torch.from_numpy(w.view(np.int64)).cuda()
    runs = []
    for _ in range(2):
        pol = lg.Policy(L, seed=4)
        losses = [pol.train_step(seqs, target, weight, 5, 20, lr=2e-3)[0] for _ in range(3)]
        runs.append((torch.cat(losses).cpu(), pol.get_params().cpu()))
    assert torch.equal(runs[0][0], runs[1][0])
    assert torch.equal(runs[0][1], runs[1][1])
