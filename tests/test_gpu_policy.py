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


@pytest.mark.parametrize("L,n", [(13, 5), (64, 3), (451, 2)])
def test_forward_matches_oracle(lg, L, n):
    flat, q = _params(L, 3)
    w, x = _batch(L, n, 7)
    pol = lg.Policy(L)
    pol.set_params(flat)
    got = pol.forward(torch.from_numpy(w.view(np.int64)).cuda()).cpu().numpy()
    exp, _ = opol.forward(q, x)
    assert _close(got, exp)


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
