"""Pins of the learned-initialiser oracle (oracle/cnn.py) against library routines,
adjoint identities, closed forms and finite differences."""
import numpy as np
from scipy.signal import correlate2d

from oracle import cnn as O

rng = np.random.default_rng(7)


def test_bf16_round_values():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.0, 3.0e-3])
    y = O.bf16_round(x)
    assert y[0] == 1.0 and y[1] == 1.0 and y[2] == 1 + 2 ** -6 and y[3] == -2.5 and y[4] == 0.0
    assert abs(y[5] - 3.0e-3) <= 3.0e-3 * 2 ** -8


def test_conv3x3_matches_scipy():
    x = rng.normal(size=(2, 3, 9, 7))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = O.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = sum(correlate2d(x[n, c], w[o, c], mode="same", boundary="fill") for c in range(3)) + b[o]
            assert np.abs(y[n, o] - ref).max() < 1e-12


def test_conv_gradients_are_adjoints():
    x = rng.normal(size=(2, 3, 8, 6))
    w = rng.normal(size=(5, 3, 3, 3))
    dy = rng.normal(size=(2, 5, 8, 6))
    y0 = O.conv3x3(x, w, np.zeros(5))
    assert abs(np.sum(y0 * dy) - np.sum(x * O.conv3x3_dgrad(dy, w))) < 1e-9
    dw, db = O.conv3x3_wgrad(dy, x)
    assert abs(np.sum(y0 * dy) - np.sum(w * dw)) < 1e-9
    assert np.allclose(db, dy.sum(axis=(0, 2, 3)))


def test_pool_and_upsample_adjoints():
    x = rng.normal(size=(1, 2, 8, 8))
    y = rng.normal(size=(1, 2, 16, 16))
    assert abs(np.sum(O.up2(x) * y) - np.sum(x * O.up2_bwd(y))) < 1e-12
    big = rng.normal(size=(1, 2, 8, 8))
    pooled, arg = O.maxpool2(big)
    assert np.allclose(pooled, big.reshape(1, 2, 4, 2, 4, 2).max(axis=(3, 5)))
    dy = rng.normal(size=pooled.shape)
    dx = O.maxpool2_bwd(dy, arg, big.shape)
    eps = 1e-6
    for _ in range(5):   # directional derivative of sum(pool(x) * dy)
        d = rng.normal(size=big.shape)
        num = (np.sum(O.maxpool2(big + eps * d)[0] * dy) - np.sum(O.maxpool2(big - eps * d)[0] * dy)) / (2 * eps)
        assert abs(num - np.sum(dx * d)) < 1e-6
    tie = np.zeros((1, 1, 2, 2))
    assert O.maxpool2(tie)[1][0, 0, 0, 0] == 0   # ties go to the first element in row-major order


def test_mse_and_adam_closed_forms():
    a = rng.normal(size=(2, 2, 4, 4))
    loss, g = O.mse(a, a)
    assert loss == 0.0 and np.abs(g).max() == 0.0
    loss, g = O.mse(a, np.zeros_like(a))
    assert abs(loss - np.mean(a * a)) < 1e-15 and np.allclose(g, 2 * a / a.size)
    p = {"w": np.array([1.0, -2.0, 3.0])}
    gr = {"w": np.array([0.5, -4.0, 0.0])}
    m, v = {"w": np.zeros(3)}, {"w": np.zeros(3)}
    O.adam_step(p, gr, m, v, 1, 0.1)
    # first step: m_hat = g, v_hat = g^2 -> w -= lr g / (|g| + eps)
    assert np.allclose(p["w"], [1.0 - 0.1, -2.0 + 0.1, 3.0], atol=1e-7)


def test_unet_gradients_match_finite_differences():
    p = O.init_params(3)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.1, p[k].shape)
    x = rng.normal(size=(1, 2, 16, 16))
    t = rng.normal(size=(1, 2, 16, 16))
    out, cache = O.forward(p, x, bf16=False)
    loss, dout = O.mse(out, t)
    g = O.backward(p, cache, dout, bf16=False)
    eps = 1e-6
    for name in ("e1a.w", "e3b.w", "bb.b", "d3a.w", "d1b.w", "head.w", "head.b"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = O.mse(O.forward(p, x, bf16=False)[0], t)[0]
            flat[idx] = old - eps
            lm = O.mse(O.forward(p, x, bf16=False)[0], t)[0]
            flat[idx] = old
            num = (lp - lm) / (2 * eps)
            ana = g[name].reshape(-1)[idx]
            assert abs(num - ana) <= 1e-5 * max(1.0, abs(num)) + 1e-9, (name, idx, num, ana)
