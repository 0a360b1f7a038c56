"""Pins of the oracle's demons update and XCF tie flag against independent library restatements
(scipy / numpy), covering the configurations the other pins leave at their defaults, and of the
conditioning helper that the GPU field bar uses.

- One demons iteration (Eq. 1 with the workloads' regularisation) is, step by step:
  d = M(x - u) - F, du = d grad F / (|grad F|^2 + alpha^2 d^2), u <- G_f * (u + G_u * du).  Here the
  warp is scipy's linear map_coordinates (edge mode: the clamped bilinear sample), the gradient
  numpy's (central inside, one-sided at the borders), and the Gaussians scipy's correlate1d with
  replicated edges.  Distinct sigma_update and sigma_field and alpha != 1 make a swapped role, a
  wrong smoothing order or alpha instead of alpha^2 fail.
- The XCF near-tie flag: a surface with two equal maxima is flagged, one with a clear maximum is not.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

from synth import kikuchi as K


def gauss(sigma):
    r = math.ceil(3 * sigma)
    k = np.arange(-r, r + 1)
    w = np.exp(-k * k / (2 * sigma * sigma))
    return w / w.sum()


def smooth(img, sigma):
    if sigma <= 0:
        return img.copy()
    w = gauss(sigma)
    return ndimage.correlate1d(ndimage.correlate1d(img, w, axis=1, mode="nearest"), w, axis=0, mode="nearest")


def force(F, M, u, alpha):
    H, W = F.shape
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    mw = ndimage.map_coordinates(M, [Y - u[1], X - u[0]], order=1, mode="nearest")
    gy, gx = np.gradient(F)
    d = mw - F
    den = gx * gx + gy * gy + alpha * alpha * d * d
    t = np.where(den > 1e-9, d / np.where(den > 1e-9, den, 1.0), 0.0)
    return np.stack([t * gx, t * gy]), float(np.sum(d * d))


def pair(H=40, W=48, seed=3):
    spec = K.ScanSpec(n_pairs=1, H=H, W=W, n_refs=1, mis_lo_deg=1.0, mis_hi_deg=3.0, seed=seed)
    import oracle
    M = oracle.preprocess(K.render_ref(spec, 0).astype(np.float64))
    F = oracle.preprocess(K.render_test(spec, 0).astype(np.float64))
    rng = np.random.default_rng(seed)
    u = np.stack([smooth(rng.normal(0, 1.5, (H, W)), 2.0) for _ in range(2)])
    return F, M, u


@pytest.mark.parametrize("alpha", [0.5, 2.0])
def test_force_matches_library_composition(oracle, alpha):
    F, M, u = pair()
    du, ssd = oracle.demons_force(F, M, u, alpha)
    e_du, e_ssd = force(F, M, u, alpha)
    assert np.abs(du - e_du).max() < 1e-12 and abs(ssd - e_ssd) < 1e-9 * e_ssd
    # alpha (not alpha^2) in the denominator would differ
    wrong, _ = force(F, M, u, math.sqrt(alpha))
    assert np.abs(du - wrong).max() > 1e-3


@pytest.mark.parametrize("sigma_up,sigma_f,alpha", [(0.0, 1.0, 1.0), (1.6, 1.0, 0.5), (0.7, 2.0, 2.0)])
def test_one_update_is_smoothed_sum(oracle, sigma_up, sigma_f, alpha):
    F, M, u = pair()
    got, k, trace = oracle.demons_level(F, M, u, alpha, sigma_up, sigma_f, 1, 0, 0.0, 1)
    assert k == 1
    du, ssd = force(F, M, u, alpha)
    exp = np.stack([smooth(u[c] + smooth(du[c], sigma_up), sigma_f) for c in range(2)])
    assert np.abs(got - exp).max() < 1e-12
    assert abs(trace[0] - ssd) < 1e-9 * ssd
    # the other readings are measurably different: swapped roles, smoothing before the sum
    swapped = np.stack([smooth(u[c] + smooth(du[c], sigma_f), sigma_up) for c in range(2)])
    other_order = np.stack([smooth(u[c], sigma_f) + smooth(du[c], sigma_up) for c in range(2)])
    assert np.abs(got - swapped).max() > 1e-4
    assert np.abs(got - other_order).max() > 1e-4


def test_two_updates_chain(oracle):
    F, M, u = pair(seed=8)
    got, k, _ = oracle.demons_level(F, M, u, 2.0, 1.6, 1.0, 2, 0, 0.0, 2)
    exp = u
    for _ in range(2):
        du, _ = force(F, M, exp, 2.0)
        exp = np.stack([smooth(exp[c] + smooth(du[c], 1.6), 1.0) for c in range(2)])
    assert k == 2 and np.abs(got - exp).max() < 1e-12


def periodic_pair(S, a, b, wb, seed=0):
    """ref = one period R0 of size S tiled over 2S x 2S; test = R0 shifted by a plus wb x R0 shifted by b
    (circular, the same tiling), so that inside an S x S ROI aligned with the period the circular
    cross-correlation (window off) has the values c(a) and c(b) of a two-peak surface."""
    rng = np.random.default_rng(seed)
    R0 = ndimage.gaussian_filter(rng.normal(size=(S, S)), 1.0, mode="wrap")
    T0 = np.roll(R0, a, axis=(0, 1)) + wb * np.roll(R0, b, axis=(0, 1))
    return np.tile(R0, (2, 2)), np.tile(T0, (2, 2))


def test_near_tie_flag(oracle):
    S = 32
    roi = np.array([[S // 2 + S // 2, S // 2 + S // 2]], np.int32)   # ROI = rows/cols [S/2, 3S/2): one period
    # equal weights: c(a) = c(b) up to rounding (the autocorrelation is symmetric) -> near tie
    ref, test = periodic_pair(S, (3, -5), (-6, 4), 1.0)
    q, peak, ph, tie = oracle.xcf_roi(ref, test, roi, S, window=False)
    assert tie[0]
    # the peak is one of the two maxima
    assert tuple(peak[0]) in {(-5, 3), (4, -6)}
    # a clearly weaker second copy: a unique maximum at shift a, no tie
    ref, test = periodic_pair(S, (3, -5), (-6, 4), 0.8)
    q, peak, ph, tie = oracle.xcf_roi(ref, test, roi, S, window=False)
    assert not tie[0] and tuple(peak[0]) == (-5, 3)
    # brute-force surface: the two equal-weight maxima are equal to 1e-12 relative
    ref, test = periodic_pair(S, (3, -5), (-6, 4), 1.0)
    c, _, _ = oracle.xcf_surface(ref, test, S // 2, S // 2, S, window=False)
    assert abs(c[3 % S, -5 % S] - c[-6 % S, 4 % S]) < 1e-12 * abs(c).max()


def test_perturbed_register_helper(oracle):
    """The conditioning helper of the field bar (tests/fp32_sensitivity.py) runs the oracle's own
    registration: unperturbed it equals oracle.demons_register replaying the same counts bit for bit;
    its FP32-storage members (seeded stochastic rounding) stay within FP32-sized distances of it and
    differ from one another; the stochastic rounding is unbiased and lands on FP32 values."""
    import fp32_sensitivity as FS
    spec = K.ScanSpec(n_pairs=1, H=64, W=64, n_refs=1, mis_lo_deg=1.0, mis_hi_deg=2.0, seed=12)
    M = oracle.preprocess(K.render_ref(spec, 0).astype(np.float64))
    F = oracle.preprocess(K.render_test(spec, 0).astype(np.float64))
    it = np.array([7, 5, 4], np.int32)
    exp, _ = oracle.demons_register(M, F, 3, [10] * 3, 1.0, 1.0, 1.0, 0, 0.0, -1, None, it)
    got = FS.perturbed_register(oracle, M, F, 3, it, seed=-1)
    assert np.array_equal(got, exp)
    init = np.full((2, 32, 32), 0.25)
    exp2, _ = oracle.demons_register(M, F, 3, [10] * 3, 2.0, 0.0, 1.6, 0, 0.0, 1, init, it)
    got2 = FS.perturbed_register(oracle, M, F, 3, it, 2.0, 0.0, 1.6, seed=-1, init=init, start_level=1)
    assert np.array_equal(got2, exp2)
    m = FS.perturbed_fields(oracle, M, F, 3, it, members=2)
    s = FS.sensitivity(exp, m)
    assert 0 < np.median(s) < 1e-5 and s.max() < 1e-2 and not np.array_equal(m[0], m[1])
    m2 = FS.perturbed_fields(oracle, M, F, 3, it, members=1, alpha=2.0, sigma_up=0.0, sigma_f=1.6,
                             init=init, start_level=1)
    assert np.abs(m2[0] - exp2).max() < 1e-3
    r = np.random.default_rng(0)
    a = r.normal(size=200_000)
    b = FS.round32(a, r)
    assert np.array_equal(b, b.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(b - a) <= np.spacing(np.abs(a).astype(np.float32)))
    assert abs(np.mean(b - a)) < 1e-3 * np.mean(np.spacing(np.abs(a).astype(np.float32)))


def test_arithmetic_register_helper(oracle):
    """The FP32-arithmetic executions of the helper (every elementary operation of the iteration
    rounded) restate the oracle's registration: without rounding they agree with
    oracle.demons_register replaying the same counts to FP64 rounding (the sums are grouped as an FP32
    code groups them), and their members stay within FP32-sized distances of it and differ from one
    another."""
    import fp32_sensitivity as FS
    spec = K.ScanSpec(n_pairs=1, H=64, W=64, n_refs=1, mis_lo_deg=1.0, mis_hi_deg=2.0, seed=12)
    M = oracle.preprocess(K.render_ref(spec, 0).astype(np.float64))
    F = oracle.preprocess(K.render_test(spec, 0).astype(np.float64))
    it = np.array([7, 5, 4], np.int32)
    exp, _ = oracle.demons_register(M, F, 3, [10] * 3, 1.0, 1.0, 1.0, 0, 0.0, -1, None, it)
    assert np.abs(FS.arithmetic_register(oracle, M, F, 3, it, seed=-1) - exp).max() < 1e-10
    exp2, _ = oracle.demons_register(M, F, 3, [10] * 3, 2.0, 0.0, 1.6, 0, 0.0, -1, None, it)
    got2 = FS.arithmetic_register(oracle, M, F, 3, it, 2.0, 0.0, 1.6, seed=-1)
    assert np.abs(got2 - exp2).max() < 1e-10
    m = FS.arithmetic_fields(oracle, M, F, 3, it, members=2)
    s = FS.sensitivity(exp, m)
    assert 0 < np.median(s) < 1e-5 and s.max() < 1e-2 and not np.array_equal(m[0], m[1])


def test_pyramid_for_sizes_that_do_not_halve(oracle):
    """Reading for the paper's 1244 x 1024 patterns: a level is floor(H/2) x floor(W/2) (an odd last row
    or column takes no part in the 2 x 2 box mean) and the prolongation fills the stored finer size, its
    extra last row/column taking the clamped edge value."""
    x = np.random.default_rng(3).normal(size=(13, 19))
    assert np.allclose(oracle.reduce2(x), x[:12, :18].reshape(6, 2, 9, 2).mean(axis=(1, 3)), atol=1e-14)
    Yc, Xc = np.mgrid[0:6, 0:9].astype(float)
    uc = np.stack([0.3 * Xc + 0.2, -0.1 * Yc + 0.4])
    uf = oracle.prolong(uc, 13, 19)
    assert uf.shape == (2, 13, 19)
    assert np.array_equal(uf[:, :12, :18], oracle.prolong(uc))
    Yf, Xf = np.mgrid[0:13, 0:19].astype(float)
    # interior of a linear field: 2 a ((x_f + 0.5)/2 - 0.5) + 2 b
    assert np.allclose(uf[0][:, 1:17], 0.3 * (Xf[:, 1:17] - 0.5) + 0.4, atol=1e-13)
    # the last column (x_c = 8.75 beyond the coarse edge 8) and the one before it (x_c = 8.25) clamp to 8
    assert np.allclose(uf[0][:, 17], 2 * (0.3 * 8 + 0.2)) and np.allclose(uf[0][:, 18], 2 * (0.3 * 8 + 0.2))
    assert np.allclose(uf[1][12], 2 * (-0.1 * 5 + 0.4))
    # a registration on 100 x 92 patterns (levels 100x92, 50x46, 25x23) recovers a sub-pixel shift
    H, W, t = 100, 92, (0.6, -0.35)
    Y, X = np.mgrid[0:H, 0:W].astype(float)

    def img(dx, dy):
        return (np.sin(0.31 * (X - dx) + 0.2 * (Y - dy)) + np.cos(0.17 * (X - dx) - 0.27 * (Y - dy))
                + 0.5 * np.sin(0.05 * ((X - dx) ** 2 + (Y - dy) ** 2) / 10))
    ref, test = oracle.normalize(img(0, 0)), oracle.normalize(img(*t))
    field, iters = oracle.demons_register(ref, test, 3, [60] * 3, 1.0, 1.0, 1.0)
    assert field.shape == (2, H, W)
    inner = (slice(None), slice(15, -15), slice(15, -15))
    assert abs(field[inner][0].mean() - t[0]) < 0.02 and abs(field[inner][1].mean() - t[1]) < 0.02
