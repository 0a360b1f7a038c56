"""Pins of the preprocessing oracle for real scans (Section 3.2-3.3)."""
import math

import numpy as np

from oracle import filters as FL


class Geom:
    xstar, ystar, zstar = 0.5, 0.5, 0.6


def test_gaussian_filters_constant_ramp_and_sinusoid():
    c = np.full((40, 50), 3.25)
    assert np.abs(FL.bandpass(c, 1.5, 0.0) - 3.25).max() < 1e-12
    assert np.abs(FL.bandpass(c, 0.0, 6.0)).max() < 1e-12
    yy, xx = np.mgrid[0:40, 0:50].astype(np.float64)
    ramp = 0.3 * xx - 0.7 * yy + 2
    r = int(math.ceil(3 * 6.0))
    hp = FL.bandpass(ramp, 0.0, 6.0)
    assert np.abs(hp[r:-r, r:-r]).max() < 1e-10   # a symmetric kernel passes linear functions unchanged
    # a sinusoid along x is scaled by the discrete transfer function sum_k t_k cos(2 pi f k)
    f = 0.09
    s = np.sin(2 * np.pi * f * xx + 0.4)
    t = FL.gauss_taps(2.0)
    k = np.arange(len(t)) - len(t) // 2
    Hf = float(np.sum(t * np.cos(2 * np.pi * f * k)))
    out = FL.blur(s, 2.0)
    r = len(t) // 2
    # the y pass sees a constant along y: rows stay scaled copies
    assert np.abs(out[:, r:-r] - Hf * s[:, r:-r]).max() < 1e-12


def test_background_corrections():
    rng = np.random.default_rng(4)
    bg = 1.0 + 0.2 * rng.random((30, 30))
    sig = 1.0 + 0.1 * rng.normal(size=(30, 30))
    assert np.abs(FL.background(bg * sig, static_bg=bg) - sig).max() < 1e-12
    pats = [bg * 2.0, bg * 4.0]
    assert np.abs(FL.mean_pattern(pats) - 3.0 * bg).max() < 1e-12
    # the dynamic correction is invariant to the pattern's scale, and maps a constant to ones
    x = 5.0 + rng.random((30, 30))
    assert np.abs(FL.background(7.0 * x, sigma_dyn=4.0) - FL.background(x, sigma_dyn=4.0)).max() < 1e-12
    assert np.abs(FL.background(np.full((20, 20), 2.5), sigma_dyn=3.0) - 1.0).max() < 1e-12


def test_shift_zoom_identity_integer_shift_and_linear():
    rng = np.random.default_rng(5)
    img = rng.normal(size=(24, 20))
    g = Geom()
    assert np.abs(FL.shift_zoom(img, (0.0, 0.0), 1.0, g) - img).max() < 1e-12
    out = FL.shift_zoom(img, (3.0, -2.0), 1.0, g)   # out(x) = in(x - t)
    assert np.abs(out[2:20, 3:20] - img[4:22, 0:17]).max() < 1e-12
    # Keys' cubic reproduces linear functions, so a zoom about pc maps a ramp to the zoomed ramp
    yy, xx = np.mgrid[0:24, 0:20].astype(np.float64)
    ramp = 0.5 * xx + 0.25 * yy
    s, t = 1.1, (0.7, -0.4)
    pcx, pcy = 0.5 * 20 - 0.5, 0.5 * 24 - 0.5
    exp = 0.5 * (pcx + (xx - pcx - t[0]) / s) + 0.25 * (pcy + (yy - pcy - t[1]) / s)
    out = FL.shift_zoom(ramp, t, s, g)
    assert np.abs(out[3:-3, 3:-3] - exp[3:-3, 3:-3]).max() < 1e-12
