"""Learned initialiser: the library's tensor-core network against the FP64 oracle.

Same parameters and inputs on both sides; the oracle stores activations and
pre-activation gradients in BF16 like the library (FP64 arithmetic).  Bars:
output field within 2 % of its largest magnitude; each parameter gradient
within 5 % in relative L2 norm; the first Adam step equals its closed form.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1907_05993_gb300 as P
    from paper_1907_05993_gb300 import cnn_params as CP
    from oracle import cnn as OC
    assert torch.cuda.is_available()
    ctx = P.hrebsd_create(0)
    yield torch, P, CP, OC, ctx
    P.hrebsd_destroy(ctx)


def _params(OC, seed):
    p = OC.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.05, p[k].shape)
    return p


def _bf16_tensor(torch, OC, x):
    xr = OC.bf16_round(x)
    return torch.from_numpy(xr.astype(np.float32)).to(torch.bfloat16).cuda(), xr


def test_forward_matches_oracle(env):
    torch, P, CP, OC, ctx = env
    p = _params(OC, 1)
    assert P.hrebsd_cnn_num_params(ctx) == CP.num_params()
    P.hrebsd_cnn_init(ctx, CP.pack(p))
    rng = np.random.default_rng(2)
    xg, xr = _bf16_tensor(torch, OC, rng.normal(size=(3, 2, 64, 64)))
    out = torch.empty((3, 2, 64, 64), device="cuda")
    P.hrebsd_cnn_infer(ctx, xg, 3, out)
    torch.cuda.synchronize()
    exp, _ = OC.forward(CP.unpack(CP.pack(p)), xr, bf16=True)
    got = out.cpu().numpy()
    assert np.abs(got - exp).max() <= 0.02 * np.abs(exp).max()


def test_gradients_match_oracle(env):
    torch, P, CP, OC, ctx = env
    p = _params(OC, 3)
    v = CP.pack(p)
    P.hrebsd_cnn_init(ctx, v)
    rng = np.random.default_rng(4)
    xg, xr = _bf16_tensor(torch, OC, rng.normal(size=(2, 2, 64, 64)))
    target = rng.normal(0, 0.5, (2, 2, 64, 64)).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    P.hrebsd_cnn_train_step(ctx, xg, torch.from_numpy(target).cuda(), 2, 0.0, loss)
    w_after, grads = P.hrebsd_cnn_get_params(ctx)
    assert np.array_equal(w_after, v)   # lr = 0: gradients only
    pu = CP.unpack(v)
    out, cache = OC.forward(pu, xr, bf16=True)
    l_exp, dout = OC.mse(out, target.astype(np.float64))
    assert abs(float(loss) - l_exp) <= 0.02 * l_exp
    g_exp = OC.backward(pu, cache, dout, bf16=True)
    g = CP.unpack(grads)
    for k in g_exp:
        num = np.linalg.norm(g[k] - g_exp[k])
        den = np.linalg.norm(g_exp[k]) + 1e-30
        assert num <= 0.05 * den, (k, num / den)


def test_first_adam_step_closed_form(env):
    torch, P, CP, OC, ctx = env
    p = _params(OC, 5)
    v = CP.pack(p)
    P.hrebsd_cnn_init(ctx, v)
    rng = np.random.default_rng(6)
    xg, _ = _bf16_tensor(torch, OC, rng.normal(size=(2, 2, 64, 64)))
    target = torch.from_numpy(rng.normal(0, 0.5, (2, 2, 64, 64)).astype(np.float32)).cuda()
    lr = 1e-3
    P.hrebsd_cnn_train_step(ctx, xg, target, 2, lr)
    w1, g = P.hrebsd_cnn_get_params(ctx)
    # step 1: m_hat = g, v_hat = g^2 -> w1 = w0 - lr g / (|g| + 1e-8)
    exp = v.astype(np.float64) - lr * g / (np.abs(g) + 1e-8)
    assert np.abs(w1 - exp).max() <= 1e-6


def test_training_reduces_loss(env):
    torch, P, CP, OC, ctx = env
    P.hrebsd_cnn_init(ctx, CP.pack(OC.init_params(7)))
    rng = np.random.default_rng(8)
    x = rng.normal(size=(8, 2, 64, 64))
    yy, xx = np.mgrid[0:64, 0:64] / 64.0
    target = np.stack([np.stack([0.5 * x[b, 0] * 0 + np.sin(3 * xx + b) , np.cos(2 * yy - b)]) for b in range(8)])
    xg, _ = _bf16_tensor(torch, OC, x)
    tg = torch.from_numpy(target.astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    losses = []
    for _ in range(40):
        P.hrebsd_cnn_train_step(ctx, xg, tg, 8, 2e-3, loss)
        losses.append(float(loss))
    assert losses[-1] < 0.5 * losses[0]


def test_tcgen05_convolutions_match_oracle_and_mma_path(env):
    """HREBSD_OPT_CNN_TC on (the default): forward 3x3 convolutions on tcgen05 MMAs into tensor
    memory fed by TMA halo tiles; same bars against the oracle, and close to the mma.sync path."""
    torch, P, CP, OC, ctx0 = env
    P.hrebsd_set_option(ctx0, P.OPT_CNN_TC, 0)
    ctx = P.hrebsd_create(0)
    P.hrebsd_set_option(ctx, P.OPT_CNN_TC, 1)
    try:
        p = _params(OC, 1)
        v = CP.pack(p)
        rng = np.random.default_rng(2)
        xg, xr = _bf16_tensor(torch, OC, rng.normal(size=(3, 2, 64, 64)))
        outs = []
        for c in (ctx, ctx0):
            P.hrebsd_cnn_init(c, v)
            out = torch.empty((3, 2, 64, 64), device="cuda")
            P.hrebsd_cnn_infer(c, xg, 3, out)
            P.hrebsd_device_error(c)
            outs.append(out.cpu().numpy())
        exp, _ = OC.forward(CP.unpack(v), xr, bf16=True)
        scale = np.abs(exp).max()
        assert np.abs(outs[0] - exp).max() <= 0.02 * scale
        assert np.abs(outs[0] - outs[1]).max() <= 0.02 * scale
        # a batch with more tiles than CTAs at every level (persistent loop, both accumulators, ragged
        # last group of 8x8 images): same result as the mma.sync path
        xg2 = torch.from_numpy(rng.normal(size=(523, 2, 64, 64)).astype(np.float32)).cuda().to(torch.bfloat16)
        big = []
        for c in (ctx, ctx0):
            out = torch.empty((523, 2, 64, 64), device="cuda")
            P.hrebsd_cnn_infer(c, xg2, 523, out)
            P.hrebsd_device_error(c)
            big.append(out.cpu().numpy())
        sc2 = np.abs(big[1]).max()
        assert np.isfinite(big[0]).all()
        assert np.abs(big[0] - big[1]).max() <= 0.02 * sc2
        assert np.abs(big[0] - big[1]).mean() <= 1e-3 * sc2
        # gradients
        p3 = _params(OC, 3)
        v3 = CP.pack(p3)
        P.hrebsd_cnn_init(ctx, v3)
        rng = np.random.default_rng(4)
        xg, xr = _bf16_tensor(torch, OC, rng.normal(size=(2, 2, 64, 64)))
        target = rng.normal(0, 0.5, (2, 2, 64, 64)).astype(np.float32)
        loss = torch.zeros(1, device="cuda")
        P.hrebsd_cnn_train_step(ctx, xg, torch.from_numpy(target).cuda(), 2, 0.0, loss)
        P.hrebsd_device_error(ctx)
        _, grads = P.hrebsd_cnn_get_params(ctx)
        pu = CP.unpack(v3)
        o, cache = OC.forward(pu, xr, bf16=True)
        l_exp, dout = OC.mse(o, target.astype(np.float64))
        assert abs(float(loss) - l_exp) <= 0.02 * l_exp
        g_exp = OC.backward(pu, cache, dout, bf16=True)
        g = CP.unpack(grads)
        for k in g_exp:
            num = np.linalg.norm(g[k] - g_exp[k])
            den = np.linalg.norm(g_exp[k]) + 1e-30
            assert num <= 0.05 * den, (k, num / den)
    finally:
        P.hrebsd_set_option(ctx0, P.OPT_CNN_TC, 1)
        P.hrebsd_destroy(ctx)
