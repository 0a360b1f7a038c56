"""Preprocessing for real scans (Section 3.2-3.3) against the oracle."""
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


def _patterns(n=3, H=96, W=80):
    spec = K.ScanSpec(n_pairs=n, H=H, W=W, n_refs=1, mis_lo_deg=0.5, mis_hi_deg=3.0, seed=9)
    return np.stack([K.render_test(spec, p) for p in range(n)]).astype(np.float32)


@pytest.mark.parametrize("lp,hp", [(1.0, 0.0), (0.0, 8.0), (1.5, 12.0), (0.0, 32.0)])
def test_bandpass_parity(env, lp, hp):
    torch, P, ctx = env
    from oracle import filters as FL
    x = _patterns()
    n, H, W = x.shape
    d = torch.from_numpy(x).cuda()
    out = torch.empty_like(d)
    P.hrebsd_bandpass_batch(ctx, d, n, H, W, lp, hp, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for b in range(n):
        exp = FL.bandpass(x[b].astype(np.float64), lp, hp)
        assert np.abs(got[b] - exp).max() <= 2e-5 * np.abs(x[b]).max()
    # in place
    P.hrebsd_bandpass_batch(ctx, d, n, H, W, lp, hp, d)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), got)


def test_background_and_mean_pattern_parity(env):
    torch, P, ctx = env
    from oracle import filters as FL
    x = _patterns(4)
    n, H, W = x.shape
    d = torch.from_numpy(x).cuda()
    bg = torch.empty((H, W), device="cuda")
    P.hrebsd_mean_pattern(ctx, d, n, H, W, bg)
    out = torch.empty_like(d)
    P.hrebsd_background_batch(ctx, d, n, H, W, bg, 10.0, out)
    torch.cuda.synchronize()
    bg_exp = FL.mean_pattern(x.astype(np.float64))
    assert np.abs(bg.cpu().numpy() - bg_exp).max() <= 1e-5 * np.abs(bg_exp).max()
    got = out.cpu().numpy()
    for b in range(n):
        exp = FL.background(x[b].astype(np.float64), static_bg=bg.cpu().numpy().astype(np.float64), sigma_dyn=10.0)
        assert np.abs(got[b] - exp).max() <= 1e-4 * np.abs(exp).max()


def test_shift_zoom_parity(env):
    torch, P, ctx = env
    from oracle import filters as FL
    x = _patterns(2, 40, 36)
    n, H, W = x.shape
    shift = np.array([[1.25, -0.5], [-2.0, 3.75]], dtype=np.float32)
    zoom = np.array([1.03, 0.97], dtype=np.float32)
    geom = P.hrebsd_geometry(0.5, 0.45, 0.6)
    out = torch.empty((n, H, W), device="cuda")
    P.hrebsd_shift_zoom_batch(ctx, torch.from_numpy(x).cuda(), n, H, W, torch.from_numpy(shift).cuda(),
                              torch.from_numpy(zoom).cuda(), geom, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()

    class G:
        xstar, ystar, zstar = 0.5, 0.45, 0.6
    for b in range(n):
        exp = FL.shift_zoom(x[b].astype(np.float64), shift[b].astype(np.float64), float(zoom[b]), G)
        assert np.abs(got[b] - exp).max() <= 1e-4 * np.abs(x[b]).max()
    with pytest.raises(P.HrebsdError):
        P.hrebsd_shift_zoom_batch(ctx, out, n, H, W, None, None, geom, out)
    with pytest.raises(P.HrebsdError):
        P.hrebsd_bandpass_batch(ctx, out, n, H, W, 40.0, 0.0, out)   # radius 120 > 96


def test_pipeline_with_real_scan_preprocessing(env, oracle):
    """Dynamic background correction and band-pass ahead of the method: the filtered patterns
    match the oracle's filters and the rotation is still recovered.  (A static background is the
    mean over a whole scan of many orientations; over a few similar patterns it keeps their bands,
    so this end-to-end check leaves it out; its arithmetic is checked above.)"""
    torch, P, ctx = env
    import math
    from oracle import filters as FL
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    spec = K.ScanSpec(n_pairs=4, H=128, W=128, n_refs=1, fixed_mis_deg=3.0, strain=1e-4, strain_mode="norm",
                      counts=500.0, seed=21)
    refs, tests, ridx, Ft = K.make_scan(spec)
    roi = K.roi_grid(128, 128, 32, True)
    cfg = PipelineConfig(128, 128, roi, 32, 3, (50, 50, 50), dynamic_background=12.0, bandpass=(0.7, 0.0))
    pipe = Pipeline(cfg)
    o = pipe.run(torch.from_numpy(refs).cuda(), torch.from_numpy(tests).cuda(), torch.from_numpy(ridx).cuda())
    torch.cuda.synchronize()
    exp = FL.bandpass(FL.background(tests[1].astype(np.float64), None, 12.0), 0.7, 0.0)
    got = o["test_filtered"].cpu().numpy()[1]
    assert np.abs(got - exp).max() <= 1e-4 * np.abs(exp).max()
    Fg = o["F"].cpu().numpy().reshape(-1, 3, 3)
    for b in range(4):
        e = math.acos(float(np.clip((np.trace(oracle.polar(Fg[b]).T @ oracle.polar(Ft[b])) - 1) / 2, -1, 1)))
        assert e < 0.2 * math.radians(3.0), (b, e)
    pipe.close()
