"""FP64 numpy oracle of the pattern preprocessing for real scans -- TEST INFRASTRUCTURE.

Section 3.2-3.3 of the paper name the steps without giving their kernels:
a low-pass and a high-pass filter (remove high-frequency noise and
low-frequency background gradients) before the demons registration, static
and dynamic background correction, and the shift and zoom/shrink correction
of a pattern (an affine transformation about the pattern centre).  Readings:

  * Gaussian filters with radius ceil(3 sigma), weights exp(-k^2 / 2 sigma^2)
    normalised to one, replicated borders, x pass then y pass (the same
    family as the demons smoothing).  Band-pass = low-pass(x) - G_hp * x; a
    sigma of 0 switches that filter off.
  * Static background: the mean pattern of the scan; the correction divides
    by it.  Dynamic background: the pattern's own Gaussian blur of sigma_dyn;
    the correction divides by it.  Divisors of magnitude below 1e-12 give 0.
  * Shift/zoom: out(x) = in(pc + (x - pc - t) / s) in index coordinates
    (pixel centres on integers, pc = (xstar W - 0.5, ystar H - 0.5)), sampled
    with the Keys cubic (a = -0.5) and replicated borders.

Only the tests may import this module.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_taps(sigma):
    if sigma <= 0:
        return np.ones(1)
    r = int(math.ceil(3 * sigma))
    k = np.arange(-r, r + 1, dtype=np.float64)
    t = np.exp(-k * k / (2 * sigma * sigma))
    return t / t.sum()


def blur(img, sigma):
    """Separable Gaussian, replicated borders (x pass, then y pass)."""
    a = np.asarray(img, dtype=np.float64)
    t = gauss_taps(sigma)
    r = len(t) // 2
    if r == 0:
        return a.copy()
    H, W = a.shape
    p = np.pad(a, ((0, 0), (r, r)), mode="edge")
    x = sum(t[j] * p[:, j:j + W] for j in range(len(t)))
    p = np.pad(x, ((r, r), (0, 0)), mode="edge")
    return sum(t[i] * p[i:i + H, :] for i in range(len(t)))


def bandpass(img, sigma_lp, sigma_hp):
    a = np.asarray(img, dtype=np.float64)
    lp = blur(a, sigma_lp) if sigma_lp > 0 else a
    return lp - blur(a, sigma_hp) if sigma_hp > 0 else lp


def mean_pattern(imgs):
    return np.mean(np.asarray(imgs, dtype=np.float64), axis=0)


def _safe_div(a, d):
    out = np.zeros_like(a)
    ok = np.abs(d) >= 1e-12
    out[ok] = a[ok] / d[ok]
    return out


def background(img, static_bg=None, sigma_dyn=0.0):
    """Static correction (divide by the scan's mean pattern), then dynamic (divide by the own blur)."""
    a = np.asarray(img, dtype=np.float64)
    if static_bg is not None:
        a = _safe_div(a, np.asarray(static_bg, dtype=np.float64))
    if sigma_dyn > 0:
        a = _safe_div(a, blur(a, sigma_dyn))
    return a


def _keys(t):
    """Keys cubic convolution weights (a = -0.5) for the 4 taps at offsets -1, 0, 1, 2 of fraction t."""
    a = -0.5

    def w(x):
        x = abs(x)
        if x <= 1:
            return (a + 2) * x ** 3 - (a + 3) * x ** 2 + 1
        if x < 2:
            return a * x ** 3 - 5 * a * x ** 2 + 8 * a * x - 4 * a
        return 0.0
    return [w(t + 1), w(t), w(1 - t), w(2 - t)]


def cubic_sample(img, x, y):
    H, W = img.shape
    x0, y0 = math.floor(x), math.floor(y)
    wx, wy = _keys(x - x0), _keys(y - y0)
    s = 0.0
    for j in range(4):
        yy = min(max(y0 - 1 + j, 0), H - 1)
        for i in range(4):
            xx = min(max(x0 - 1 + i, 0), W - 1)
            s += wy[j] * wx[i] * img[yy, xx]
    return s


def shift_zoom(img, shift, zoom, geom):
    """out(x) = in(pc + (x - pc - t) / s); pure-Python loop, small images only."""
    a = np.asarray(img, dtype=np.float64)
    H, W = a.shape
    pcx, pcy = geom.xstar * W - 0.5, geom.ystar * H - 0.5
    out = np.empty_like(a)
    for yy in range(H):
        for xx in range(W):
            sx = pcx + (xx - pcx - shift[0]) / zoom
            sy = pcy + (yy - pcy - shift[1]) / zoom
            out[yy, xx] = cubic_sample(a, sx, sy)
    return out
