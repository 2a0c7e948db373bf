"""Plain FP64 reference of the selector network's arithmetic -- test
infrastructure only.

The network maps 16 features to a logit through three hidden ReLU layers of
32: z1 = W1 x + b1, h1 = max(z1, 0), the same for layers 2 and 3, and
logit = w4 . h3 + b4.  Parameters are packed as in the library
(W1[32][16], b1, W2[32][32], b2, W3[32][32], b3, w4[32], b4; 2689 floats).
Training minimises the weighted binary cross-entropy of the logits,
L = sum_s w_s (softplus(z_s) - y_s z_s) / sum_s w_s, whose gradient is
back-propagated layer by layer below.  This is the definition written out
with numpy products; nothing is blocked or fused.
"""
import numpy as np

NF, H = 16, 32
NPARAM = H * NF + H + 2 * (H * H + H) + H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((H, NF), (H,), (H, H), (H,), (H, H), (H,), (H,), ()):
        size = int(np.prod(shape)) if shape else 1
        out.append(p[o:o + size].reshape(shape) if shape else p[o])
        o += size
    assert o == NPARAM
    return out


def pack(parts):
    return np.concatenate([np.ravel(np.asarray(x, dtype=np.float64)) for x in parts])


def forward(p, X):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3.T + b3
    h3 = np.maximum(z3, 0.0)
    z4 = h3 @ w4 + b4
    return z4, (X, z1, h1, z2, h2, z3, h3)


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def loss(p, X, y, w):
    z4, _ = forward(p, X)
    return float(np.sum(w * (softplus(z4) - y * z4)) / np.sum(w))


def loss_grad(p, X, y, w):
    """(loss, gradient packed like p)"""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p)
    z4, (X, z1, h1, z2, h2, z3, h3) = forward(p, X)
    ws = np.sum(w)
    L = float(np.sum(w * (softplus(z4) - y * z4)) / ws)
    d4 = w * (1.0 / (1.0 + np.exp(-z4)) - y) / ws  # dL/dz4
    gw4 = h3.T @ d4
    gb4 = np.sum(d4)
    dz3 = np.outer(d4, w4) * (z3 > 0)
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3, gw4, gb4])


def init_params(seed):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from numpy's
    seeded generator; float32 like the library."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, shape in ((NF, (H, NF)), (None, (H,)), (H, (H, H)), (None, (H,)), (H, (H, H)), (None, (H,)),
                          (H, (H,)), (None, ())):
        if fan_in is None:
            parts.append(np.zeros(shape))
        else:
            b = np.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-b, b, shape))
    return pack(parts).astype(np.float32)
