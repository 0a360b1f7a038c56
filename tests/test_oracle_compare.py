"""Pins of the comparison-method and metric oracle (Section 3.1, Fig. 2-3)."""
import math

import numpy as np

from oracle import compare as CM
from synth import kikuchi as K


class Geom:
    xstar, ystar, zstar = 0.5, 0.5, 0.6


def _project(F, pts, g, H, W):
    r = np.stack([pts[:, 0] - g.xstar * W, pts[:, 1] - g.ystar * H, np.full(len(pts), g.zstar * W)], axis=1)
    p = r @ F.T
    zs = g.zstar * W
    return np.stack([g.xstar * W + zs * p[:, 0] / p[:, 2], g.ystar * H + zs * p[:, 1] / p[:, 2]], axis=1)


def test_mae_zero_on_exact_points_and_brute_force_angle():
    rng = np.random.default_rng(1)
    g, H, W = Geom(), 256, 256
    F = K.axis_angle([0.2, 0.5, 0.8], math.radians(3)) @ (np.eye(3) + np.diag([3e-4, -2e-4, 1e-4]))
    ref = rng.uniform(30, 226, (25, 2))
    test = _project(F, ref, g, H, W)
    assert CM.mean_angular_error(F, ref, test, g, H, W) < 1e-12
    test[7] += [0.8, -0.3]
    # brute force for the moved point: angle between the two 3-D rays by arccos of the normalised dot product
    a = np.array([test[7, 0] - 128, test[7, 1] - 128, 0.6 * 256])
    b = F @ np.array([ref[7, 0] - 128, ref[7, 1] - 128, 0.6 * 256])
    ang = math.acos(np.clip(a @ b / np.linalg.norm(a) / np.linalg.norm(b), -1, 1))
    assert abs(CM.mean_angular_error(F, ref, test, g, H, W) - ang / 25) < 1e-12


def test_ssim_identity_symmetry_and_one_window_brute_force():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(40, 36))
    y = 0.7 * x + rng.normal(scale=0.5, size=x.shape)
    assert abs(CM.ssim(x, x) - 1.0) < 1e-12
    assert abs(CM.ssim(x, y, L=3.0) - CM.ssim(y, x, L=3.0)) < 1e-12
    assert CM.ssim(5 + x, 5 - x) < 0   # positive means, anti-correlated structure
    # an 11 x 11 image has exactly one window: explicit weighted moments
    a, b = x[:11, :11], y[:11, :11]
    w = CM.gauss_window()
    mx, my = (w * a).sum(), (w * b).sum()
    sxx = (w * (a - mx) ** 2).sum()
    syy = (w * (b - my) ** 2).sum()
    sxy = (w * (a - mx) * (b - my)).sum()
    L = b.max() - b.min()
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    exp = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    assert abs(CM.ssim(a, b) - exp) < 1e-12


def _pair(mis_deg, seed=3, H=128):
    spec = K.ScanSpec(n_pairs=1, H=H, W=H, n_refs=1, fixed_mis_deg=mis_deg, strain=1e-4, strain_mode="norm",
                      counts=500.0, seed=seed)
    g = K.ref_orientation(spec, 0)
    F = K.pair_truth(spec, 0)
    ref = K.render(g, np.eye(3), H, H, spec.geom, noise=False).astype(np.float64)
    test = K.render(g, F, H, H, spec.geom, noise=False).astype(np.float64)
    return spec, F, ref, test


def _rot_err(A, B):
    return math.acos(float(np.clip((np.trace(A.T @ B) - 1) / 2, -1, 1)))


def test_methods_recover_a_small_rotation(oracle):
    spec, Ft, ref, test = _pair(1.0)
    pref, ptest = oracle.preprocess(ref), oracle.preprocess(test)
    roi = K.roi_grid(128, 128, 32, True)
    Rt = oracle.polar(Ft)
    Fa, _, _ = CM.method_a(pref, ptest, roi, 32, spec.geom)
    F1, Rb, field = CM.method_b(pref, ptest, roi, spec.geom, 3, [50] * 3)
    Fc, Ra, _, _ = CM.method_c(pref, ptest, roi, 32, spec.geom)
    e0 = _rot_err(np.eye(3), Rt)
    # demons-based (b) recovers most of the rotation; the XCF-based (a) and (c) less (Fig. 2)
    assert _rot_err(oracle.polar(F1), Rt) < 0.2 * e0
    for F in (Fa, Fc):
        assert _rot_err(oracle.polar(F), Rt) < 0.6 * e0
    # the rotation used for the remap in (c) is (a)'s
    assert np.abs(Ra - oracle.polar(Fa)).max() < 1e-12


def test_remapping_raises_peak_height_and_ssim_of_warp(oracle):
    """Fig. 2-3 at 4 degrees: without remapping the correlation peak drops, remapped ROIs keep it
    high (demons remap highest); the demons warp brings the reference much closer to the test
    than no warp; demons-based rotations beat the cross-correlation one."""
    spec, Ft, ref, test = _pair(4.0)
    pref, ptest = oracle.preprocess(ref), oracle.preprocess(test)
    roi = K.roi_grid(128, 128, 32, True)
    _, _, ph_a = CM.method_a(pref, ptest, roi, 32, spec.geom)
    _, _, _, ph_c = CM.method_c(pref, ptest, roi, 32, spec.geom)
    res = oracle.pipeline(ref, test, roi, 32, spec.geom, 3, [50] * 3)
    assert np.mean(res["ph"]) > np.mean(ph_c) > np.mean(ph_a)
    F1, Rb, field = CM.method_b(pref, ptest, roi, spec.geom, 3, [50] * 3)
    assert CM.ssim_warped(pref, ptest, field) > CM.ssim(pref, ptest) + 0.5
    Rt = oracle.polar(Ft)
    Fa0, _, _ = CM.method_a(pref, ptest, roi, 32, spec.geom)
    e_a = _rot_err(oracle.polar(Fa0), Rt)
    assert _rot_err(oracle.polar(F1), Rt) < 0.5 * e_a and _rot_err(oracle.polar(res["F"]), Rt) < 0.5 * e_a
    # MAE of the second pass of (d) is below that of the direct fit (a)
    roi_f = np.asarray(roi, dtype=np.float64)
    Fa, qa, _ = CM.method_a(pref, ptest, roi, 32, spec.geom)
    mae_a = CM.mean_angular_error(Fa, roi_f, roi_f + qa, spec.geom, 128, 128)
    Fm = res["F"] @ res["R_finite"].T
    mae_d = CM.mean_angular_error(Fm, roi_f, roi_f + res["q"], spec.geom, 128, 128)
    assert mae_d < mae_a
