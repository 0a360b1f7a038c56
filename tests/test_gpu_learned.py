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
    learned = pipe.run(refs, tests, ridx, learned_caps=(100, 100, 25, 0), learned_start_res=64)
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


def test_training_targets_spot_checked_against_oracle(oracle):
    """Training targets (the final field of the full registration, box-averaged to 64x64 in
    64x64-pixel units) from the library path, against the oracle's registration of the same
    numpy-rendered training pairs replayed with the library's per-level iteration counts."""
    import torch
    import paper_1907_05993_gb300 as P
    spec = K.config4(200_000)
    pairs = [3, 70_001, 150_007]
    ctx = P.hrebsd_create(0)
    prm = P.demons_params(3, [100] * 3, 1.0, 1.0, 1.0, 1e-4, 5)
    for p in pairs:
        ref = K.render_ref(spec, K.ref_index(spec, p))
        test = K.render_test(spec, p)
        r_d, t_d = torch.from_numpy(ref[None]).cuda(), torch.from_numpy(test[None]).cuda()
        P.hrebsd_preprocess_batch(ctx, r_d, 1, 128, 128, 1, r_d)
        P.hrebsd_preprocess_batch(ctx, t_d, 1, 128, 128, 1, t_d)
        field = torch.empty((1, 2, 128, 128), device="cuda")
        iters = torch.empty((1, 3), dtype=torch.int32, device="cuda")
        status = torch.empty((1,), dtype=torch.int32, device="cuda")
        P.hrebsd_demons_register_batch(ctx, r_d, t_d, torch.zeros(1, dtype=torch.int32, device="cuda"), 1, 1, 128,
                                       128, prm, None, field, iters, status)
        target = torch.empty((1, 2, 64, 64), device="cuda")
        P.hrebsd_field_resample(ctx, field, 1, 128, 128, target, 64, 64)
        torch.cuda.synchronize()
        it = iters.cpu().numpy()[0]
        pr = oracle.preprocess(ref.astype(np.float64), True)
        pt = oracle.preprocess(test.astype(np.float64), True)
        fo, _ = oracle.demons_register(pr, pt, 3, [100] * 3, 1.0, 1.0, 1.0, 5, 1e-4, replay=it)
        exp = np.stack([oracle.reduce2(fo[c]) / 2 for c in range(2)])
        d = np.abs(target.cpu().numpy()[0] - exp)
        assert np.mean(d <= 1e-3) >= 0.99 and d.max() <= 0.05, (p, d.max(), np.mean(d <= 1e-3))
    P.hrebsd_destroy(ctx)
