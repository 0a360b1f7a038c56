"""Learned initialiser: the library's tensor-core network against the FP64 oracle.

Same parameters and inputs on both sides; the oracle stores activations and
pre-activation gradients in BF16 like the library (FP64 arithmetic), so the
two differ where a different FP32 summation order flips a BF16 rounding (one
unit of 2^-8 relative), and such flips propagate through the 14 convolutions.
Element-wise bars, with u = 2^-8 the BF16 unit roundoff and rms the tensor's
root mean square (the floor for elements near zero):
  output field   |got - exp| <= 8 u (|exp| + rms)
  gradients      |got - exp| <= 16 u (|exp| + rms)   (every weight and bias)
(measured worst cases: 4.0 u for the field, 10.9 u for a weight gradient,
4.0 u for a bias gradient); the loss within 1e-3 relative; the first Adam step
equals its closed form.
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


U_BF16 = 2.0 ** -8


def assert_elementwise(got, exp, k, what=""):
    exp = np.asarray(exp, np.float64)
    rms = float(np.sqrt(np.mean(exp ** 2)))
    r = np.abs(np.asarray(got, np.float64) - exp) / (U_BF16 * (np.abs(exp) + rms))
    assert r.max() <= k, (what, float(r.max()))
    return float(r.max())


def assert_gradients(OC, CP, grads, g_exp):
    g = CP.unpack(grads)
    worst = {k: assert_elementwise(g[k], g_exp[k], 16, k) for k in g_exp}
    print("gradient element-wise worst (units of 2^-8 (|e| + rms)):", max(worst.values()))


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
    assert_elementwise(out.cpu().numpy(), exp, 8, "field")


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
    assert abs(float(loss) - l_exp) <= 1e-3 * l_exp
    g_exp = OC.backward(pu, cache, dout, bf16=True)
    assert_gradients(OC, CP, grads, g_exp)


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
    # 80 Adam steps (gradients are summed with float atomics, so the trajectory varies a little
    # from run to run; 40 steps left the last loss between 0.45 and 0.55 of the first)
    for _ in range(80):
        P.hrebsd_cnn_train_step(ctx, xg, tg, 8, 2e-3, loss)
        losses.append(float(loss))
    assert losses[-1] < 0.5 * losses[0], losses[::10]


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
        assert_elementwise(outs[0], exp, 8, "field (tcgen05)")
        assert_elementwise(outs[1], exp, 8, "field (mma.sync)")
        # a batch with more tiles than CTAs at every level (persistent loop, both accumulators, ragged
        # last group of 8x8 images): same result as the mma.sync path
        xg2 = torch.from_numpy(rng.normal(size=(523, 2, 64, 64)).astype(np.float32)).cuda().to(torch.bfloat16)
        big = []
        for c in (ctx, ctx0):
            out = torch.empty((523, 2, 64, 64), device="cuda")
            P.hrebsd_cnn_infer(c, xg2, 523, out)
            P.hrebsd_device_error(c)
            big.append(out.cpu().numpy())
        assert np.isfinite(big[0]).all()
        assert_elementwise(big[0], big[1], 16, "tcgen05 vs mma.sync, 523 pairs")
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
        assert abs(float(loss) - l_exp) <= 1e-3 * l_exp
        g_exp = OC.backward(pu, cache, dout, bf16=True)
        assert_gradients(OC, CP, grads, g_exp)
        # the input gradients of 11 of the 13 layers run on tcgen05 too (FP32 epilogue): on a batch with
        # more tiles than CTAs, the weight gradients after one backward pass match the mma.sync path
        xb = torch.from_numpy(rng.normal(size=(261, 2, 64, 64)).astype(np.float32)).cuda().to(torch.bfloat16)
        tb = torch.from_numpy(rng.normal(0, 0.5, (261, 2, 64, 64)).astype(np.float32)).cuda()
        gb = []
        for c in (ctx, ctx0):
            P.hrebsd_cnn_init(c, v3)
            P.hrebsd_cnn_train_step(c, xb, tb, 261, 0.0, loss)
            P.hrebsd_device_error(c)
            gb.append(P.hrebsd_cnn_get_params(c)[1])
        g0, g1 = CP.unpack(gb[0]), CP.unpack(gb[1])
        worst = max(assert_elementwise(g0[k], g1[k], 16, f"{k} tcgen05 vs mma.sync") for k in g1)
        print("tcgen05 vs mma.sync gradients, 261 pairs: worst", worst, "units of 2^-8 (|e| + rms)")
    finally:
        P.hrebsd_set_option(ctx0, P.OPT_CNN_TC, 1)
        P.hrebsd_destroy(ctx)
