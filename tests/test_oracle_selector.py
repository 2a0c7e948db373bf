"""Pins of the selector's reference arithmetic (not GPU).

S1  The network gradient equals central finite differences of the loss.
S2  bfloat16 rounding: round to nearest, ties to even.
S3  The emulated BF16 logit equals the FP64 forward pass exactly when every
    weight, bias and feature and every partial sum is representable (so no
    rounding can occur): pins the parameter layout, the layer order and ReLU.
S4  Features: zero on a constant state; on a linear ramp the ratio and
    mismatch features vanish; at a step the ratio is 1 and the jump feature
    equals jump/(|Q0| + jump).
"""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = mlp.init_params(3).astype(np.float64)
    p[mlp.H * mlp.NF:mlp.H * mlp.NF + mlp.H] = rng.normal(0, 0.1, mlp.H)  # nonzero b1
    X = rng.uniform(0, 1, (40, mlp.NF))
    y = (rng.uniform(size=40) > 0.5).astype(np.float64)
    w = rng.uniform(0.5, 2.0, 40)
    L, g = mlp.loss_grad(p, X, y, w)
    assert L == pytest.approx(mlp.loss(p, X, y, w), rel=1e-14)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        h = 1e-6 * max(1.0, abs(p[i]))
        e[i] = h
        fd = (mlp.loss(p + e, X, y, w) - mlp.loss(p - e, X, y, w)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])), i


def bf16(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def test_bf16_rounding(orc):
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-3], dtype=np.float32)
    exp = np.array([1.0, 1.0, 1.0 + 2 ** -6, -2.5, bf16(np.float32(3.0e-3))], dtype=np.float32)
    assert np.array_equal(bf16(vals), exp)
    # through the oracle: identity weights route a feature to the logit
    p = np.zeros(mlp.NPARAM, dtype=np.float32)
    W1, o = p[:mlp.H * mlp.NF].reshape(mlp.H, mlp.NF), mlp.H * mlp.NF + mlp.H
    W1[0, 0] = 1.0
    W2 = p[o:o + mlp.H * mlp.H].reshape(mlp.H, mlp.H)
    W2[0, 0] = 1.0
    o2 = o + mlp.H * mlp.H + mlp.H
    W3 = p[o2:o2 + mlp.H * mlp.H].reshape(mlp.H, mlp.H)
    W3[0, 0] = 1.0
    o3 = o2 + mlp.H * mlp.H + mlp.H
    p[o3] = 1.0  # w4[0]
    f = np.zeros((len(vals), 16), dtype=np.float32)
    f[:, 0] = np.abs(vals)
    got = orc.selector_logits(p, f)
    assert np.array_equal(got, bf16(np.abs(vals)))


def test_emulated_logit_exact_on_representable_network(orc):
    """Weights in {-1, 0, 1} with at most two nonzeros per row after the first
    layer, biases and features multiples of 1/2: every activation fits in the
    8 significant bits of bfloat16 and every sum is exact in float."""
    rng = np.random.default_rng(11)
    H, NF = mlp.H, mlp.NF
    W1 = rng.choice([-1.0, 0.0, 1.0], (H, NF))
    W1[:, 15] = 0.0

    def sparse():
        W = np.zeros((H, H))
        for o in range(H):
            W[o, rng.choice(H, 2, replace=False)] = rng.choice([-1.0, 1.0], 2)
        return W
    W2, W3 = sparse(), sparse()
    w4 = np.zeros(H)
    w4[rng.choice(H, 4, replace=False)] = rng.choice([-1.0, 1.0], 4)
    b = [rng.choice([-0.5, 0.0, 0.5, 1.0], H) for _ in range(3)]
    p = mlp.pack([W1, b[0], W2, b[1], W3, b[2], w4, 0.5]).astype(np.float32)
    X = rng.choice(np.array([0.0, 0.5, 1.0]), (64, NF)).astype(np.float32)
    X[:, 15] = 0.0
    got = orc.selector_logits(p, X)
    want, (_, z1, _, z2, _, z3, _) = mlp.forward(p.astype(np.float64), X.astype(np.float64))
    for z in (z1, z2, z3):
        assert np.all(bf16(np.maximum(z, 0).astype(np.float32)) == np.maximum(z, 0))
    assert np.array_equal(got.astype(np.float64), want)


def _features(orc, fn, n=(16, 12), bc=(1, 1, 0, 0)):
    o = orc.Oracle(2, n, lo=(0, 0), hi=(1, 1), bc=list(bc))
    o.init(fn)
    return o.selector_features().reshape(n[1], n[0], 16)


def test_features_constant_state(orc):
    f = _features(orc, lambda x, y: [1.2 + 0 * x, 0.3 + 0 * x, -0.2 + 0 * x, 0.8 + 0 * x])
    assert np.all(f == 0.0)


# feature order per class (density 0-4, momentum 5-9, energy 10-14): J, E, R, S, C; G last
def test_features_linear_ramp(orc):
    """Linear data: no second difference (R), no mismatch of the lines with
    the central difference (C), no gradient jump (G); face and corner jumps
    both equal the cell-to-cell increment."""
    f = _features(orc, lambda x, y: [1.0 + 0.1 * x, 0 * x, 0 * x, 1.0 + 0 * x])
    inner = f[:, 1:-1]
    assert np.all(inner[..., 2] < 1e-4) and np.all(inner[..., 4] < 1e-4) and np.all(inner[..., 15] < 1e-5)
    jump = 0.1 / 16 / (1 + 0.1 * ((np.arange(1, 15) + 0.5) / 16))
    for k in (0, 1):
        assert np.all(np.abs(inner[..., k] / (1 - inner[..., k]) - jump) < 1e-5)


def test_features_step(orc):
    """A density step at a face: the cell beside it sees a jump 0.5 on the
    face and on the corners (J = E = 0.5/1.5 after x/(1+x)) and a ratio
    R = 1; cells away from it see nothing."""
    f = _features(orc, lambda x, y: [np.where(x < 0.5, 1.0, 0.5), 0 * x, 0 * x, 1.0 + 0 * x])
    left = f[:, 7]  # the last cell with rho = 1
    assert np.allclose(left[:, 2], 1.0, atol=1e-6)
    assert np.allclose(left[:, 0], 0.5 / 1.5, rtol=1e-6) and np.allclose(left[:, 1], 0.5 / 1.5, rtol=1e-6)
    far = f[:, 2]
    assert np.all(far[:, :3] == 0.0)
