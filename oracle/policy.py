"""fp64 reference of the learned flip-proposal network -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this network is the library's optional proposal bias for the
self-avoiding walk of Algorithm 1 (the exact energy stays the judge).  Plain numpy in float64, loops
written out so a reader can check each line:

  features  x[0][i] = s_{i+1} (+-1),  x[1][0] = 0,  x[1][k] = C_k / sqrt(L - k)  for k = 1..L-1
  conv_l    y[co][i] = b[co] + sum_{ci, t<9} w[co][ci][t] * h[ci][i + t - 4]   (zero outside 0..L-1)
            three layers 2 -> 64 -> 64 -> 64 channels, each followed by ReLU
  fc1       z[j] = b1[j] + sum_{c, i} W1[j][c * L + i] * h3[c][i],  j < 256, ReLU
  fc2       logits[i] = b2[i] + sum_j W2[i][j] * a[j],  i < L
  loss      per sample n with free positions F_n, taken flip t_n and weight w_n:
            CE_n = logsumexp_{i in F_n} logits[i] - logits[t_n];  loss = sum w_n CE_n / sum w_n

Parity status: forward pinned to torch.nn.functional (fp64, CPU) and the backward to central finite
differences of this forward (tests/test_oracle_policy.py).  Trained weight VALUES are "parity
unpinned": only the arithmetic that maps given weights to logits and gradients is pinned.
"""
import numpy as np

C_HID = 64
KW = 9
PAD = 4
HIDDEN = 256


def param_shapes(L):
    return {
        "w1": (C_HID, 2, KW), "b1": (C_HID,),
        "w2": (C_HID, C_HID, KW), "b2": (C_HID,),
        "w3": (C_HID, C_HID, KW), "b3": (C_HID,),
        "W4": (HIDDEN, C_HID * L), "b4": (HIDDEN,),
        "W5": (L, HIDDEN), "b5": (L,),
    }


def init_params(L, seed):
    """He-uniform initial weights (numpy PCG64), biases zero."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in param_shapes(L).items():
        if k.startswith("b"):
            p[k] = np.zeros(shp)
        else:
            fan_in = int(np.prod(shp[1:]))
            lim = np.sqrt(6.0 / fan_in)
            p[k] = rng.uniform(-lim, lim, size=shp)
    return p


def features(s, C):
    """s: [N, L] +-1; C: [N, L-1] correlations C_1..C_{L-1}.  Returns x [N, 2, L] float64."""
    s = np.asarray(s, dtype=np.float64)
    N, L = s.shape
    x = np.zeros((N, 2, L))
    x[:, 0, :] = s
    for k in range(1, L):
        x[:, 1, k] = np.asarray(C, dtype=np.float64)[:, k - 1] / np.sqrt(L - k)
    return x


def conv_forward(h, w, b):
    N, Cin, L = h.shape
    Cout = w.shape[0]
    y = np.zeros((N, Cout, L))
    for co in range(Cout):
        y[:, co, :] = b[co]
        for ci in range(Cin):
            for t in range(KW):
                sh = t - PAD  # y[i] += w * h[i + sh]
                lo, hi = max(0, -sh), min(L, L - sh)
                y[:, co, lo:hi] += w[co, ci, t] * h[:, ci, lo + sh:hi + sh]
    return y


def conv_backward(h, w, dy):
    """Gradients of y = conv(h, w) + b: (dh, dw, db)."""
    N, Cin, L = h.shape
    Cout = w.shape[0]
    dh = np.zeros_like(h)
    dw = np.zeros_like(w)
    db = dy.sum(axis=(0, 2))
    for co in range(Cout):
        for ci in range(Cin):
            for t in range(KW):
                sh = t - PAD
                lo, hi = max(0, -sh), min(L, L - sh)
                dw[co, ci, t] = np.sum(dy[:, co, lo:hi] * h[:, ci, lo + sh:hi + sh])
                dh[:, ci, lo + sh:hi + sh] += w[co, ci, t] * dy[:, co, lo:hi]
    return dh, dw, db


def bf16_round(a):
    """Rounds to bfloat16 the way the device stores an FP32 value as BF16: first to float32, then to the
    nearest bfloat16 (ties to even) by rounding away the low 16 bits of the float32 encoding."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def forward(p, x, act_bf16=False):
    """Returns (logits [N, L], cache).  act_bf16: the three convolution outputs (after ReLU) are stored
    as bfloat16 before the next layer reads them, as the device's inference path does."""
    r = bf16_round if act_bf16 else (lambda v: v)
    c1 = conv_forward(x, p["w1"], p["b1"])
    h1 = r(np.maximum(c1, 0))
    c2 = conv_forward(h1, p["w2"], p["b2"])
    h2 = r(np.maximum(c2, 0))
    c3 = conv_forward(h2, p["w3"], p["b3"])
    h3 = r(np.maximum(c3, 0))
    N, C, L = h3.shape
    f = h3.reshape(N, C * L)
    z = f @ p["W4"].T + p["b4"]
    a = np.maximum(z, 0)
    logits = a @ p["W5"].T + p["b5"]
    return logits, (x, c1, h1, c2, h2, c3, h3, f, z, a)


def loss_and_dlogits(logits, free_mask, target, weight):
    """Weighted cross-entropy over the free positions; returns (loss, dloss/dlogits)."""
    N, L = logits.shape
    masked = np.where(free_mask, logits, -np.inf)
    mx = masked.max(axis=1, keepdims=True)
    e = np.where(free_mask, np.exp(masked - mx), 0.0)
    Z = e.sum(axis=1, keepdims=True)
    prob = e / Z
    lse = mx[:, 0] + np.log(Z[:, 0])
    ce = lse - logits[np.arange(N), target]
    wsum = weight.sum()
    loss = float(np.sum(weight * ce) / wsum)
    d = prob.copy()
    d[np.arange(N), target] -= 1.0
    d *= (weight / wsum)[:, None]
    return loss, d


def backward(p, cache, dlogits):
    x, c1, h1, c2, h2, c3, h3, f, z, a = cache
    g = {}
    g["W5"] = dlogits.T @ a
    g["b5"] = dlogits.sum(axis=0)
    da = dlogits @ p["W5"]
    dz = da * (z > 0)
    g["W4"] = dz.T @ f
    g["b4"] = dz.sum(axis=0)
    df = dz @ p["W4"]
    dh3 = df.reshape(h3.shape)
    dc3 = dh3 * (c3 > 0)
    dh2, g["w3"], g["b3"] = conv_backward(h2, p["w3"], dc3)
    dc2 = dh2 * (c2 > 0)
    dh1, g["w2"], g["b2"] = conv_backward(h1, p["w2"], dc2)
    dc1 = dh1 * (c1 > 0)
    _, g["w1"], g["b1"] = conv_backward(x, p["w1"], dc1)
    return g


def loss_and_grads(p, x, free_mask, target, weight):
    logits, cache = forward(p, x)
    loss, dl = loss_and_dlogits(logits, free_mask, target, weight)
    return loss, backward(p, cache, dl), logits


def adam_step(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, ICLR 2015, Algorithm 1) in float32, elementwise:
    m1 <- b1 m1 + (1 - b1) g,  m2 <- b2 m2 + (1 - b2) g^2,
    p  <- p - lr (m1 / (1 - b1^t)) / (sqrt(m2 / (1 - b2^t)) + eps).
    Returns (p, m1, m2) as new float32 arrays."""
    f = np.float32
    p, g, m1, m2 = (np.asarray(a, dtype=np.float32) for a in (p, g, m1, m2))
    m1 = f(b1) * m1 + (f(1) - f(b1)) * g
    m2 = f(b2) * m2 + (f(1) - f(b2)) * g * g
    c1 = f(1) - f(b1) ** np.float32(t)
    c2 = f(1) - f(b2) ** np.float32(t)
    p = p - f(lr) * (m1 / c1) / (np.sqrt(m2 / c2) + f(eps))
    return p.astype(np.float32), m1, m2
