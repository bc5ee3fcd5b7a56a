"""Pins of the fp64 network oracle: forward against torch.nn.functional (fp64, CPU), backward against
central finite differences of the oracle's forward, features against their definition."""
import numpy as np
import pytest

import labs_inputs as inp
import oracle
from oracle import policy

torch = pytest.importorskip("torch")


def _batch(L, n, seed):
    w = inp.random_words(n, L, seed=seed)
    s = oracle.words_to_pm1(w, L)
    _, C = oracle.energy_batch(w, L, with_C=True)
    return policy.features(s, C), s, C


def test_features_definition():
    L = 13
    x, s, C = _batch(L, 3, 1)
    assert np.array_equal(x[:, 0, :], s.astype(float))
    assert np.all(x[:, 1, 0] == 0)
    for k in (1, 5, 12):
        assert np.allclose(x[:, 1, k], C[:, k - 1] / np.sqrt(L - k))


def test_forward_matches_torch_fp64():
    import torch.nn.functional as Fn

    L = 17
    p = policy.init_params(L, seed=3)
    for k in p:
        if k.startswith("b"):
            p[k] = np.random.default_rng(7).normal(size=p[k].shape) * 0.1
    x, _, _ = _batch(L, 4, 2)
    logits, _ = policy.forward(p, x)
    t = {k: torch.from_numpy(v) for k, v in p.items()}
    h = torch.from_numpy(x)
    h = torch.relu(Fn.conv1d(h, t["w1"], t["b1"], padding=4))
    h = torch.relu(Fn.conv1d(h, t["w2"], t["b2"], padding=4))
    h = torch.relu(Fn.conv1d(h, t["w3"], t["b3"], padding=4))
    z = torch.relu(Fn.linear(h.reshape(4, -1), t["W4"], t["b4"]))
    ref = Fn.linear(z, t["W5"], t["b5"]).numpy()
    assert np.allclose(logits, ref, rtol=1e-12, atol=1e-12)


def test_backward_matches_finite_differences():
    L = 13
    rng = np.random.default_rng(5)
    p = policy.init_params(L, seed=11)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(size=p[k].shape) * 0.05
    x, _, _ = _batch(L, 3, 4)
    free = np.zeros((3, L), dtype=bool)
    free[:, 2:7] = True
    target = np.array([3, 6, 2])
    weight = np.array([1.0, 0.5, 2.0])
    loss, g, _ = policy.loss_and_grads(p, x, free, target, weight)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(3, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp, _ = policy.loss_and_dlogits(policy.forward(p, x)[0], free, target, weight)
            flat[i] = old - eps
            lm, _ = policy.loss_and_dlogits(policy.forward(p, x)[0], free, target, weight)
            flat[i] = old
            num = (lp - lm) / (2 * eps)
            ana = g[k].reshape(-1)[i]
            assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)), (k, i, num, ana)


def test_loss_is_weighted_cross_entropy_over_free_positions():
    L = 9
    logits = np.random.default_rng(1).normal(size=(2, L))
    free = np.zeros((2, L), dtype=bool)
    free[0, [1, 4, 5]] = True
    free[1, [0, 8]] = True
    target = np.array([4, 8])
    weight = np.array([3.0, 1.0])
    loss, _ = policy.loss_and_dlogits(logits, free, target, weight)
    ce0 = np.log(np.exp(logits[0, [1, 4, 5]]).sum()) - logits[0, 4]
    ce1 = np.log(np.exp(logits[1, [0, 8]]).sum()) - logits[1, 8]
    assert np.isclose(loss, (3 * ce0 + ce1) / 4)


def test_adam_first_step_is_lr_times_sign():
    """Adam's bias correction makes the first step -lr * g / (|g| + eps): -lr sign(g) wherever |g| >> eps,
    and nothing where g = 0; a second identical gradient moves by the same amount again."""
    rng = np.random.default_rng(3)
    p = rng.normal(size=200).astype(np.float32)
    g = rng.normal(size=200).astype(np.float32)
    g[::7] = 0.0
    z = np.zeros_like(p)
    p1, m1, m2 = policy.adam_step(p, g, z, z, 1, 1e-2)
    step = np.where(g == 0, 0.0, -1e-2 * np.sign(g))
    assert np.allclose(p1 - p, step, atol=1e-6)
    p2, _, _ = policy.adam_step(p1, g, m1, m2, 2, 1e-2)
    assert np.allclose(p2 - p1, step, atol=1e-6)


def test_bf16_round_matches_torch():
    """bf16_round against torch's float32 -> bfloat16 conversion (round to nearest even), including ties
    and values that are exact in bfloat16."""
    rng = np.random.default_rng(8)
    v = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-5, 5, size=2000),
                        [0.0, 1.0, -2.5, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 255.0, 257.0]]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(policy.bf16_round(v), ref)
