"""The learned initialiser end to end: training data from the registration,
training on the library's kernels, and registration started from its field.

What it must show: training lowers the loss; on held-out pairs the predicted
64x64 field is closer to the plain registration's field at that level than the
zero start is; and the registration started from it is not less accurate
against the ground truth than the plain path (the iterations it saves and the
throughput are measured by the benchmark's learned-initialiser workload)."""
import math

import numpy as np
import pytest

from synth import kikuchi as K

pytestmark = pytest.mark.gpu


def rot_err(Ra, Rb):
    return math.acos(float(np.clip((np.trace(np.asarray(Ra).T @ np.asarray(Rb)) - 1) / 2, -1, 1)))


@pytest.fixture(scope="module")
def trained():
    import torch
    import paper_1907_05993_gb300 as P
    from paper_1907_05993_gb300 import learned as LN
    ctx = P.hrebsd_create(0)
    spec = K.config4(4096)
    x, y = LN.build_training_set(ctx, spec)
    hist = LN.train(ctx, x[:3584], y[:3584], epochs=24, batch=256, lr=2e-3, seed=0)
    yield torch, P, LN, ctx, x, y, hist
    P.hrebsd_destroy(ctx)


def test_training_lowers_loss(trained):
    torch, P, LN, ctx, x, y, hist = trained
    assert hist[-1] < 0.7 * hist[0], hist


def test_prediction_beats_zero_start_on_held_out_pairs(trained):
    torch, P, LN, ctx, x, y, hist = trained
    xv, yv = x[3584:].contiguous(), y[3584:]
    out = torch.empty_like(yv)
    P.hrebsd_cnn_infer(ctx, xv, xv.shape[0], out)
    torch.cuda.synchronize()
    mse_net = float(((out - yv) ** 2).mean())
    mse_zero = float((yv ** 2).mean())
    assert mse_net < 0.8 * mse_zero, (mse_net, mse_zero)


def test_learned_start_reaches_plain_rotation(trained):
    torch, P, LN, ctx, x, y, hist = trained
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    from synth import gpu as SG
    spec = K.config5(400)
    refs, tests, ridx, Ft = SG.make_scan_gpu(spec, range(64))
    roi = K.roi_grid(256, 256, 64, False)
    cfg = PipelineConfig(256, 256, roi, 64, 4, (100, 100, 100, 100), stop_tol=1e-4, stop_window=5)
    pipe = Pipeline(cfg)
    plain = {k: v.clone() for k, v in pipe.run(refs, tests, ridx).items()}
    # the learned start needs the trained network in the pipeline's context
    w, _ = P.hrebsd_cnn_get_params(ctx)
    P.hrebsd_cnn_init(pipe.ctx, w)
    learned = pipe.run(refs, tests, ridx, learned_caps=(100, 100, 100, 0))
    torch.cuda.synchronize()
    Fp = plain["F"].cpu().numpy().reshape(-1, 3, 3)
    Fl = learned["F"].cpu().numpy().reshape(-1, 3, 3)
    d = [rot_err(Fp[b], Fl[b]) for b in range(64)]
    err_p = [rot_err(Fp[b], Ft[b]) for b in range(64)]
    err_l = [rot_err(Fl[b], Ft[b]) for b in range(64)]
    it_p = plain["iters"].cpu().numpy().sum(axis=1)
    it_l = learned["iters"].cpu().numpy().sum(axis=1)
    print("median |R_learned - R_plain| rad", np.median(d), "ground-truth error plain/learned",
          np.median(err_p), np.median(err_l), "iterations plain/learned", it_p.mean(), it_l.mean())
    assert np.median(err_l) <= 1.5 * np.median(err_p) + 1e-4
    pipe.close()
