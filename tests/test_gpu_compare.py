"""Comparison methods and quality measures (Section 3.1, Fig. 2-3) against the oracle."""
import math

import numpy as np
import pytest

from synth import kikuchi as K

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1907_05993_gb300 as P
    assert torch.cuda.is_available()
    ctx = P.hrebsd_create(0)
    yield torch, P, ctx
    P.hrebsd_destroy(ctx)


def _pair(mis_deg, seed, H=128):
    spec = K.ScanSpec(n_pairs=1, H=H, W=H, n_refs=1, fixed_mis_deg=mis_deg, strain=1e-4, strain_mode="norm",
                      counts=500.0, seed=seed)
    g = K.ref_orientation(spec, 0)
    F = K.pair_truth(spec, 0)
    ref = K.render(g, np.eye(3), H, H, spec.geom, noise=False).astype(np.float32)
    test = K.render(g, F, H, H, spec.geom, noise=False).astype(np.float32)
    return spec, ref, test


def test_polar_batch(env, oracle):
    torch, P, ctx = env
    rng = np.random.default_rng(3)
    Fs = np.stack([K.axis_angle(rng.normal(size=3), rng.uniform(0, 0.3)) @ (np.eye(3) + 0.01 * rng.normal(size=(3, 3)))
                   for _ in range(7)])
    R = torch.empty((7, 9), dtype=torch.float64, device="cuda")
    P.hrebsd_polar_batch(ctx, torch.from_numpy(Fs.reshape(7, 9)).cuda(), 7, R)
    torch.cuda.synchronize()
    for b in range(7):
        assert np.abs(R.cpu().numpy()[b].reshape(3, 3) - oracle.polar(Fs[b])).max() < 1e-12


def test_fit_quality_and_ssim_match_oracle(env, oracle):
    torch, P, ctx = env
    from oracle import compare as CM
    spec, ref, test = _pair(4.0, 5)
    pref, ptest = oracle.preprocess(ref.astype(np.float64)), oracle.preprocess(test.astype(np.float64))
    roi = K.roi_grid(128, 128, 32, True)
    N = len(roi)
    geom = P.hrebsd_geometry(spec.geom.xstar, spec.geom.ystar, spec.geom.zstar)
    Fa, qa, pha = CM.method_a(pref, ptest, roi, 32, spec.geom)
    F1, Rb, field = CM.method_b(pref, ptest, roi, spec.geom, 3, [50] * 3)
    roi_d = torch.from_numpy(np.ascontiguousarray(roi, dtype=np.int32)).cuda()
    mae = torch.empty(1, dtype=torch.float64, device="cuda")
    phm = torch.empty(1, dtype=torch.float64, device="cuda")
    q32 = qa.astype(np.float32)
    P.hrebsd_fit_quality(ctx, torch.from_numpy(Fa.reshape(1, 9)).cuda(), None, torch.from_numpy(q32[None]).cuda(),
                         None, torch.from_numpy(pha.astype(np.float32)[None]).cuda(), 1, 128, 128, roi_d, N, geom, mae,
                         phm)
    torch.cuda.synchronize()
    roi_f = np.asarray(roi, dtype=np.float64)
    exp = CM.mean_angular_error(Fa, roi_f, roi_f + q32.astype(np.float64), spec.geom, 128, 128)
    assert abs(float(mae) - exp) <= 1e-9 * max(exp, 1e-12) + 1e-15
    assert abs(float(phm) - np.mean(pha.astype(np.float32))) < 1e-6
    f32 = field.astype(np.float32)
    P.hrebsd_fit_quality(ctx, torch.from_numpy(F1.reshape(1, 9)).cuda(), None, None,
                         torch.from_numpy(f32[None]).cuda(), None, 1, 128, 128, roi_d, N, geom, mae, None)
    torch.cuda.synchronize()
    r_pts, t_pts = CM.demons_points(f32.astype(np.float64), roi)
    exp_b = CM.mean_angular_error(F1, r_pts, t_pts, spec.geom, 128, 128)
    assert abs(float(mae) - exp_b) <= 1e-6 * exp_b + 1e-9   # field sampled in FP32 on the GPU
    ssim = torch.empty(2, dtype=torch.float64, device="cuda")
    pr32, pt32 = pref.astype(np.float32), ptest.astype(np.float32)
    P.hrebsd_ssim_warped(ctx, torch.from_numpy(pr32[None]).cuda(), None, torch.from_numpy(pt32[None]).cuda(),
                         torch.from_numpy(f32[None]).cuda(), 1, 128, 128, ssim[:1])
    P.hrebsd_ssim_warped(ctx, torch.from_numpy(pr32[None]).cuda(), None, torch.from_numpy(pt32[None]).cuda(), None, 1,
                         128, 128, ssim[1:])
    torch.cuda.synchronize()
    s = ssim.cpu().numpy()
    assert abs(s[0] - CM.ssim_warped(pr32.astype(np.float64), pt32.astype(np.float64), f32.astype(np.float64))) < 1e-4
    assert abs(s[1] - CM.ssim(pr32.astype(np.float64), pt32.astype(np.float64))) < 1e-4


def test_pipeline_compare_matches_oracle_methods(env, oracle):
    torch, P, ctx = env
    from oracle import compare as CM
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    pairs = [_pair(2.0, 11), _pair(6.0, 12)]
    spec = pairs[0][0]
    refs = torch.from_numpy(np.stack([p[1] for p in pairs])).cuda()
    tests = torch.from_numpy(np.stack([p[2] for p in pairs])).cuda()
    ridx = torch.arange(2, dtype=torch.int32, device="cuda")
    roi = K.roi_grid(128, 128, 32, True)
    pipe = Pipeline(PipelineConfig(128, 128, roi, 32, 3, (50, 50, 50)))
    o = pipe.compare(refs, tests, ridx)
    torch.cuda.synchronize()
    for b, (sp, ref, test) in enumerate(pairs):
        pref, ptest = oracle.preprocess(ref.astype(np.float64)), oracle.preprocess(test.astype(np.float64))
        Fa, _, pha = CM.method_a(pref, ptest, roi, 32, sp.geom)
        Fc, Ra, _, phc = CM.method_c(pref, ptest, roi, 32, sp.geom)
        assert np.abs(o["F_a"].cpu().numpy()[b].reshape(3, 3) - Fa).max() <= 1e-6
        assert np.abs(o["R_a"].cpu().numpy()[b].reshape(3, 3) - Ra).max() <= 1e-6
        assert np.abs(o["F_c"].cpu().numpy()[b].reshape(3, 3) - Fc).max() <= 1e-6
        assert abs(float(o["phm_a"][b]) - pha.mean()) < 1e-5 and abs(float(o["phm_c"][b]) - phc.mean()) < 1e-5
    # Fig. 3 orderings on the 6-degree pair: remapping keeps the peak high, the warp raises SSIM
    assert float(o["phm_d"][1]) > float(o["phm_a"][1])
    assert float(o["ssim_b"][1]) > float(o["ssim_none"][1])
    pipe.close()
