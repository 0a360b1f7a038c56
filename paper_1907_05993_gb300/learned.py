"""Training set, training loop and model file of the learned initialiser.

The network (hrebsd_cnn_*) predicts the demons field at the 64x64 pyramid
level from the 64x64 (reference, test) pair.  Its training targets are the
fields this library's demons registration computes at that level on
generated pairs (the registration being parity-checked against the oracle),
i.e. exactly what the plain path would reach there.  Every step calls the
library; this module only schedules the calls and moves tensors.
"""
from __future__ import annotations

import numpy as np

from . import (cnn_params, demons_params, hrebsd_cnn_get_params, hrebsd_cnn_init, hrebsd_cnn_train_step,
               hrebsd_demons_register_batch, hrebsd_downsample_batch, hrebsd_preprocess_batch)

TARGET_CAPS = (100, 100)          # iteration caps of the 64x64 and 32x32 levels
STOP = dict(window=5, tol=1e-4)   # the registration's stop rule


def build_training_set(ctx, spec, chunk: int = 8192, pairs=None):
    """(x [n,2,64,64] bf16, target [n,2,64,64] f32) CUDA tensors for the pairs of `spec`."""
    import torch
    from synth import gpu as SG
    from synth import kikuchi as K
    H = spec.H
    f = H // 64
    pairs = list(range(spec.n_pairs)) if pairs is None else list(pairs)
    n = len(pairs)
    x = torch.empty((n, 2, 64, 64), dtype=torch.bfloat16, device="cuda")
    y = torch.empty((n, 2, 64, 64), dtype=torch.float32, device="cuda")
    prm = demons_params(2, TARGET_CAPS, 1.0, 1.0, 1.0, STOP["tol"], STOP["window"])
    for c0 in range(0, n, chunk):
        ps = pairs[c0:c0 + chunk]
        m = len(ps)
        gs = [K.ref_orientation(spec, K.ref_index(spec, p)) for p in ps]
        rkeys = [int(K.stream_key(spec.seed, 16 * (1_000_000 + K.ref_index(spec, p)) + K.P_NOISE)) for p in ps]
        tkeys = [int(K.stream_key(spec.seed, 16 * p + K.P_NOISE)) for p in ps]
        refs = SG.render_batch(gs, [np.eye(3)] * m, rkeys, H, H, spec.geom, spec.counts)
        tests = SG.render_batch(gs, [K.pair_truth(spec, p) for p in ps], tkeys, H, H, spec.geom, spec.counts)
        hrebsd_preprocess_batch(ctx, refs, m, H, H, 1, refs)
        hrebsd_preprocess_batch(ctx, tests, m, H, H, 1, tests)
        r64 = torch.empty((m, 64, 64), device="cuda")
        t64 = torch.empty((m, 64, 64), device="cuda")
        hrebsd_downsample_batch(ctx, refs, m, H, H, f, r64)
        hrebsd_downsample_batch(ctx, tests, m, H, H, f, t64)
        field = torch.empty((m, 2, 64, 64), device="cuda")
        iters = torch.empty((m, 2), dtype=torch.int32, device="cuda")
        status = torch.empty((m,), dtype=torch.int32, device="cuda")
        ridx = torch.arange(m, dtype=torch.int32, device="cuda")
        hrebsd_demons_register_batch(ctx, r64, t64, ridx, m, m, 64, 64, prm, None, field, iters, status)
        x[c0:c0 + m, 0] = r64.to(torch.bfloat16)
        x[c0:c0 + m, 1] = t64.to(torch.bfloat16)
        y[c0:c0 + m] = field
    torch.cuda.synchronize()
    return x, y


def train(ctx, x, y, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0, params=None):
    """Adam on the MSE over shuffled mini-batches; returns the mean loss of every epoch.
    params: initial parameter vector (None: He-normal from `seed`)."""
    import torch
    hrebsd_cnn_init(ctx, init_params(seed) if params is None else params)
    n = x.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.zeros(1, device="cuda")
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot = torch.zeros(1, device="cuda")
        steps = 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb, yb = x[idx].contiguous(), y[idx].contiguous()
            hrebsd_cnn_train_step(ctx, xb, yb, batch, lr, loss)
            tot += loss
            steps += 1
        hist.append(float(tot) / max(1, steps))
    return hist


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal initial weights (zero biases) in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co in cnn_params.LAYERS:
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / (ci * 9)), (co, ci, 3, 3))
        p[name + ".b"] = np.zeros(co)
    p["head.w"] = rng.normal(0.0, np.sqrt(1.0 / 16), (2, 16, 1, 1))
    p["head.b"] = np.zeros(2)
    return cnn_params.pack(p)


def save(ctx, path: str):
    w, _ = hrebsd_cnn_get_params(ctx)
    np.save(path, w)


def load_model(ctx, path: str):
    hrebsd_cnn_init(ctx, np.load(path))
