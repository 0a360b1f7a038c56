"""Training set, training loop and model file of the learned initialiser.

The network (hrebsd_cnn_*) maps the 64x64 (reference, test) pair to a coarse
64x64 displacement field.  Its training target is the FINAL field of this
library's full multi-resolution registration of the generated pair (the
registration being parity-checked against the oracle), box-averaged to 64x64
in 64x64-pixel units (hrebsd_field_resample).  The registration of a new pair
is then started at a finer level (128x128 by default) from the prediction
resampled to that level, skipping the coarse levels.  Every step calls the
library; this module only schedules the calls and moves tensors.
"""
from __future__ import annotations

import numpy as np

from . import (cnn_params, demons_params, hrebsd_cnn_get_params, hrebsd_cnn_init, hrebsd_cnn_load,
               hrebsd_cnn_save, hrebsd_cnn_train_step,
               hrebsd_demons_register_batch, hrebsd_downsample_batch, hrebsd_field_resample, hrebsd_preprocess_batch)

TARGET_CAP = 100                  # iteration cap of every level of the target registration
STOP = dict(window=5, tol=1e-4)   # the registration's stop rule


def build_training_set(ctx, spec, chunk: int = 8192, pairs=None):
    """(x [n,2,64,64] bf16, target [n,2,64,64] f32) CUDA tensors for the pairs of `spec`.

    Target: the final field of the full registration at spec.H (pyramid down to
    32x32), resampled to 64x64."""
    import math
    import torch
    from synth import gpu as SG
    from synth import kikuchi as K
    H = spec.H
    f = H // 64
    pairs = list(range(spec.n_pairs)) if pairs is None else list(pairs)
    n = len(pairs)
    x = torch.empty((n, 2, 64, 64), dtype=torch.bfloat16, device="cuda")
    y = torch.empty((n, 2, 64, 64), dtype=torch.float32, device="cuda")
    levels = int(round(math.log2(H / 32))) + 1
    prm = demons_params(levels, [TARGET_CAP] * levels, 1.0, 1.0, 1.0, STOP["tol"], STOP["window"])
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
        field = torch.empty((m, 2, H, H), device="cuda")
        iters = torch.empty((m, levels), dtype=torch.int32, device="cuda")
        status = torch.empty((m,), dtype=torch.int32, device="cuda")
        ridx = torch.arange(m, dtype=torch.int32, device="cuda")
        hrebsd_demons_register_batch(ctx, refs, tests, ridx, m, m, H, H, prm, None, field, iters, status)
        hrebsd_field_resample(ctx, field, m, H, H, y[c0:c0 + m], 64, 64)
        x[c0:c0 + m, 0] = r64.to(torch.bfloat16)
        x[c0:c0 + m, 1] = t64.to(torch.bfloat16)
    torch.cuda.synchronize()
    return x, y


def train(ctx, x, y, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0, params=None,
          lr_final: float | None = None):
    """Adam on the MSE over shuffled mini-batches; returns the mean loss of every epoch.
    params: initial parameter vector (None: He-normal from `seed`).  lr_final: if given,
    the step size follows a cosine from lr to lr_final over all steps."""
    import math
    import torch
    hrebsd_cnn_init(ctx, init_params(seed) if params is None else params)
    n = x.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.zeros(1, device="cuda")
    hist = []
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    step = 0
    for _ in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot = torch.zeros(1, device="cuda")
        steps = 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb, yb = x[idx].contiguous(), y[idx].contiguous()
            lr_k = lr if lr_final is None else lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / total))
            hrebsd_cnn_train_step(ctx, xb, yb, batch, lr_k, loss)
            step += 1
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
    """The model file of the library (weights, Adam moments, step): hrebsd_cnn_save."""
    hrebsd_cnn_save(ctx, path)


def load_model(ctx, path: str):
    """Load a model file written by ``save`` or ``save_checkpoint`` (hrebsd_cnn_load)."""
    hrebsd_cnn_load(ctx, path)


def save_checkpoint(ctx, path: str, **extra):
    """Training checkpoint: the network state in the library's model file at ``path``
    (hrebsd_cnn_save, written under a temporary name and renamed), plus any small arrays in
    ``extra`` (e.g. the epoch) in ``path + ".extra.npz"``, written the same way and first, so that a
    model file never pairs with the extras of a later save."""
    import os
    tmp = path + ".extra.tmp.npz"
    np.savez(tmp, **extra)
    os.replace(tmp, path + ".extra.npz")
    hrebsd_cnn_save(ctx, path)


def load_checkpoint(ctx, path: str) -> dict:
    """Restore what save_checkpoint wrote; training continues as if it had not stopped.  Returns the
    extras and the restored parameter vector (key "params")."""
    import os
    hrebsd_cnn_load(ctx, path)
    d = {}
    if os.path.exists(path + ".extra.npz"):
        with np.load(path + ".extra.npz") as z:
            d = {k: z[k] for k in z.files}
    d["params"] = hrebsd_cnn_get_params(ctx)[0]
    return d
