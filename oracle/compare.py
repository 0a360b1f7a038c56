"""FP64 oracle of the comparison methods and quality metrics -- TEST INFRASTRUCTURE.

Section 3.1 compares four ways of measuring the rotation of a pattern pair
(Fig. 2) and two quality measures (Fig. 3):

  (a) cross-correlation: Eq. 3 on the XCF shifts between the un-remapped
      reference and the test -> F (no remapping);
  (b) demons registration: Eq. 3 on the demons field at the ROI centres ->
      F_first (a5);
  (c) first pass (a), remap the reference by polar((a)) (Eq. 4-5), second-pass
      XCF, F = F_inf R (Eq. 12);
  (d) first pass (b), remap, second-pass XCF: the method of the paper
      (``oracle.pipeline``).

Metrics.  MAE, the mean angular error of an Eq. 3 fit: the mean, over the ROI
point pairs (r_i, r'_i) the fit used, of the angle between the measured test
direction (r'_i - PC, Z*) and the direction F_model (r_i - PC, Z*) the fitted
deformation gradient predicts.  PH: the mean normalised XCF peak height over
the ROIs.  SSIM (Wang et al., 2004) between the demons-warped reference
M(x - u(x)) and the test pattern, for method (b), which has no correlation
peak: 11 x 11 Gaussian window of sigma 1.5 (weights normalised over the
window), C1 = (0.01 L)^2, C2 = (0.03 L)^2 with L the test pattern's range
max - min, averaged over the pixels whose window lies inside the image.
The paper names the measures without formulas; these are the readings.
Only the tests may import this module.
"""
from __future__ import annotations

import numpy as np

from . import demons_register, fit_rotation, polar, remap, solve_F, warp, xcf_roi

SSIM_RADIUS = 5
SSIM_SIGMA = 1.5


def method_a(pref, ptest, roi, S, geom):
    """(a) XCF without remapping: returns F, the shifts q and the peak heights."""
    H, W = pref.shape
    q, _, ph, _ = xcf_roi(pref, ptest, roi, S)
    return solve_F(q, roi, H, W, geom, None), q, ph


def method_b(pref, ptest, roi, geom, levels, caps, window=0, tol=0.0):
    """(b) demons only: returns F_first, R_finite and the field."""
    field, _ = demons_register(pref, ptest, levels, caps, 1.0, 1.0, 1.0, window, tol)
    F1, R = fit_rotation(field, roi, geom)
    return F1, R, field


def method_c(pref, ptest, roi, S, geom):
    """(c) remapping with the rotation of (a), then the second pass: returns F, R_a, q2, ph2."""
    H, W = pref.shape
    Fa, _, _ = method_a(pref, ptest, roi, S, geom)
    Ra = polar(Fa)
    rem = remap(pref, Ra, geom)
    q2, _, ph2, _ = xcf_roi(rem, ptest, roi, S)
    return solve_F(q2, roi, H, W, geom, Ra), Ra, q2, ph2


def _lift(pts, geom, H, W):
    p = np.asarray(pts, dtype=np.float64)
    return np.stack([p[:, 0] - geom.xstar * W, p[:, 1] - geom.ystar * H, np.full(len(p), geom.zstar * W)], axis=1)


def mean_angular_error(F_model, ref_pts, test_pts, geom, H, W):
    """Mean angle (rad) between the measured test directions and F_model applied to the reference directions."""
    r = _lift(ref_pts, geom, H, W)
    m = _lift(test_pts, geom, H, W)
    p = r @ np.asarray(F_model, dtype=np.float64).T
    cross = np.linalg.norm(np.cross(p, m), axis=1)
    dot = np.einsum("ij,ij->i", p, m)
    return float(np.mean(np.arctan2(cross, dot)))


def mae_of_shifts(F, R, q, roi):
    """MAE of a second-pass fit: r_i = c_i, r'_i = c_i + q_i, model F_inf = F R^T (Eq. 12)."""
    roi = np.asarray(roi, dtype=np.float64)
    Fm = np.asarray(F) if R is None else np.asarray(F) @ np.asarray(R).T
    return roi, roi + np.asarray(q, dtype=np.float64), Fm


def demons_points(field, roi):
    """The a5 point pairs: r_i = c_i - u(c_i), r'_i = c_i (field sampled at index c - 0.5)."""
    from . import bilinear
    roi = np.asarray(roi, dtype=np.float64)
    u = np.array([[bilinear(field[k], c[0] - 0.5, c[1] - 0.5) for k in range(2)] for c in roi])
    return roi - u, roi


def gauss_window(radius=SSIM_RADIUS, sigma=SSIM_SIGMA):
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-k * k / (2 * sigma * sigma))
    w = np.outer(g, g)
    return w / w.sum()


def ssim(x, y, L=None):
    """Mean SSIM of x against y over the windows inside the image; L defaults to y's range."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if L is None:
        L = float(y.max() - y.min())
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    g = gauss_window()
    k = g.shape[0]
    H, W = x.shape
    # separable weights: the 2-D window is the outer product of one normalised 1-D kernel
    g1 = g.sum(axis=0)

    def blur(a):
        t = sum(g1[j] * a[:, j:W - k + 1 + j] for j in range(k))
        return sum(g1[i] * t[i:H - k + 1 + i, :] for i in range(k))
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    s = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return float(s.mean())


def ssim_warped(ref, test, field):
    """SSIM between the demons-warped reference M(x - u(x)) and the test (method (b))."""
    return ssim(warp(ref, field), test)
