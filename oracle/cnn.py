"""FP64 numpy oracle of the learned initialiser -- TEST INFRASTRUCTURE.

The paper has no learned component; the initialiser is the project addition
that predicts the coarse (64 x 64) demons field from the downsampled
reference/test pair so that fewer demons iterations are needed.  Network: a
4-level U-Net with 3x3 convolutions of 16-32-64-128 channels.

  enc1 c(2->16) c(16->16) @64, max-pool 2
  enc2 c(16->32) c(32->32) @32, max-pool 2
  enc3 c(32->64) c(64->64) @16, max-pool 2
  bott c(64->128) c(128->128) @8
  dec3 up2, concat [up, enc3] -> c(192->64) c(64->64) @16
  dec2 up2, concat [up, enc2] -> c(96->32) c(32->32) @32
  dec1 up2, concat [up, enc1] -> c(48->16) c(16->16) @64
  head 1x1 c(16->2), no activation -> field (x, y) in 64x64-level pixels

Every 3x3 convolution has zero padding, a bias and a ReLU; up2 is nearest
neighbour; the loss is the mean squared error.  Storage precision: the
trained network keeps activations in BF16 (FP32 accumulation), so the forward
pass here rounds every stored activation to BF16 when ``bf16=True``; the
arithmetic itself is FP64.  Arrays are NCHW numpy float64; weights W[co, ci,
ky, kx], cross-correlation convention y[co] = sum W[co,ci,ky,kx] x[ci, y+ky-1,
x+kx-1].  Only the tests may import this module.
"""
from __future__ import annotations

import numpy as np

# (name, cin, cout) of the 3x3 convolutions, in forward order
CONVS = [("e1a", 2, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32), ("e3a", 32, 64), ("e3b", 64, 64),
         ("ba", 64, 128), ("bb", 128, 128), ("d3a", 192, 64), ("d3b", 64, 64), ("d2a", 96, 32), ("d2b", 32, 32),
         ("d1a", 48, 16), ("d1b", 16, 16)]
HEAD = ("head", 16, 2)


def bf16_round(x):
    """Round float64 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int = 0) -> dict:
    """He-normal weights, zero biases (seeded numpy Generator)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co in CONVS:
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / (ci * 9)), (co, ci, 3, 3))
        p[name + ".b"] = np.zeros(co)
    name, ci, co = HEAD
    p[name + ".w"] = rng.normal(0.0, np.sqrt(1.0 / ci), (co, ci, 1, 1))
    p[name + ".b"] = np.zeros(co)
    return p


# ------------------------------------------------------------------ layers
def conv3x3(x, w, b):
    """x [N, ci, H, W], w [co, ci, 3, 3] -> [N, co, H, W] (zero padding)."""
    N, ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((N, w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + W])
    return y + b[None, :, None, None]


def conv3x3_dgrad(dy, w):
    """Gradient w.r.t. the input of conv3x3."""
    N, co, H, W = dy.shape
    dx = np.zeros((N, w.shape[1], H + 2, W + 2))
    for ky in range(3):
        for kx in range(3):
            dx[:, :, ky:ky + H, kx:kx + W] += np.einsum("oc,nohw->nchw", w[:, :, ky, kx], dy)
    return dx[:, :, 1:-1, 1:-1]


def conv3x3_wgrad(dy, x):
    """Gradients w.r.t. the weights and the bias of conv3x3."""
    N, ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dw = np.zeros((dy.shape[1], ci, 3, 3))
    for ky in range(3):
        for kx in range(3):
            dw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", dy, xp[:, :, ky:ky + H, kx:kx + W])
    return dw, dy.sum(axis=(0, 2, 3))


def conv1x1(x, w, b):
    return np.einsum("oc,nchw->nohw", w[:, :, 0, 0], x) + b[None, :, None, None]


def relu(x):
    return np.maximum(x, 0.0)


def maxpool2(x):
    """2x2 max-pool; the argmax (first maximum in (dy, dx) row-major order) for the backward pass."""
    N, C, H, W = x.shape
    v = x.reshape(N, C, H // 2, 2, W // 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(N, C, H // 2, W // 2, 4)
    return v.max(axis=-1), v.argmax(axis=-1)


def maxpool2_bwd(dy, arg, shape):
    N, C, H, W = shape
    d = np.zeros((N, C, H // 2, W // 2, 4))
    np.put_along_axis(d, arg[..., None], dy[..., None], axis=-1)
    return d.reshape(N, C, H // 2, W // 2, 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(N, C, H, W)


def up2(x):
    return x.repeat(2, axis=2).repeat(2, axis=3)


def up2_bwd(dy):
    N, C, H, W = dy.shape
    return dy.reshape(N, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def mse(pred, target):
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size


# ------------------------------------------------------------------ network
def forward(p, x, bf16=True):
    """x [N, 2, 64, 64] -> (field [N, 2, 64, 64], cache for backward)."""
    q = bf16_round if bf16 else (lambda a: a)
    c = {"x": q(x)}

    def block(name, inp):
        pre = conv3x3(inp, q(p[name + ".w"]), p[name + ".b"])
        out = q(relu(pre))
        c[name + ".in"], c[name + ".out"] = inp, out
        return out
    e1 = block("e1b", block("e1a", c["x"]))
    p1, c["a1"] = maxpool2(e1)
    e2 = block("e2b", block("e2a", p1))
    p2, c["a2"] = maxpool2(e2)
    e3 = block("e3b", block("e3a", p2))
    p3, c["a3"] = maxpool2(e3)
    bt = block("bb", block("ba", p3))
    d3 = block("d3b", block("d3a", np.concatenate([up2(bt), e3], axis=1)))
    d2 = block("d2b", block("d2a", np.concatenate([up2(d3), e2], axis=1)))
    d1 = block("d1b", block("d1a", np.concatenate([up2(d2), e1], axis=1)))
    c["d1"] = d1
    out = conv1x1(d1, q(p["head.w"]), p["head.b"])
    c["shapes"] = (e1.shape, e2.shape, e3.shape)
    return out, c


def backward(p, c, dout, bf16=True):
    """Gradients of every parameter for the output gradient dout.  With bf16=True
    the gradient of each convolution's pre-activation is rounded to BF16 (the
    precision it is stored in as a tensor-core operand); everything else is FP64."""
    q = bf16_round if bf16 else (lambda a: a)
    g = {}
    g["head.w"] = np.einsum("nohw,nchw->oc", dout, c["d1"])[:, :, None, None]
    g["head.b"] = dout.sum(axis=(0, 2, 3))
    dd1 = np.einsum("oc,nohw->nchw", q(p["head.w"])[:, :, 0, 0], dout)

    def block_bwd(name, dout_post):
        dpre = q(dout_post * (c[name + ".out"] > 0))   # stored in BF16 as a tensor-core operand
        g[name + ".w"], g[name + ".b"] = conv3x3_wgrad(dpre, c[name + ".in"])
        return conv3x3_dgrad(dpre, q(p[name + ".w"]))

    s1, s2, s3 = c["shapes"]
    dcat1 = block_bwd("d1a", block_bwd("d1b", dd1))           # [up(d2) 32 | e1 16]
    dd2 = up2_bwd(dcat1[:, :32])
    de1_skip = dcat1[:, 32:]
    dcat2 = block_bwd("d2a", block_bwd("d2b", dd2))           # [up(d3) 64 | e2 32]
    dd3 = up2_bwd(dcat2[:, :64])
    de2_skip = dcat2[:, 64:]
    dcat3 = block_bwd("d3a", block_bwd("d3b", dd3))           # [up(bt) 128 | e3 64]
    dbt = up2_bwd(dcat3[:, :128])
    de3_skip = dcat3[:, 128:]
    dp3 = block_bwd("ba", block_bwd("bb", dbt))
    de3 = maxpool2_bwd(dp3, c["a3"], s3) + de3_skip
    dp2 = block_bwd("e3a", block_bwd("e3b", de3))
    de2 = maxpool2_bwd(dp2, c["a2"], s2) + de2_skip
    dp1 = block_bwd("e2a", block_bwd("e2b", de2))
    de1 = maxpool2_bwd(dp1, c["a1"], s1) + de1_skip
    block_bwd("e1a", block_bwd("e1b", de1))
    return g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of every parameter, in place; t is the 1-based step."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
