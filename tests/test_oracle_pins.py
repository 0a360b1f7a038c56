"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms, invariants, brute force on tiny inputs, library routines for special
cases, or values the paper prints.  None of these touch the CUDA library.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.signal import convolve2d

from synth import kikuchi as K

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


def rot_err(Ra, Rb):
    c = np.clip((np.trace(Ra.T @ Rb) - 1) / 2, -1, 1)
    return math.acos(c)


# ------------------------------------------------------------------ a1
def test_normalize_moments(oracle):
    x = rng.normal(3.0, 7.0, (17, 23))
    y = oracle.normalize(x)
    assert abs(y.mean()) < 1e-12 and abs(y.std() - 1.0) < 1e-12
    # affine invariance: a*x + b normalises to the same image
    assert np.allclose(oracle.normalize(5.0 * x - 2.0), y, atol=1e-12)


def test_preprocess_removes_quadric_background(oracle):
    H, W = 24, 32
    x = (np.arange(W) + 0.5) / W * 2 - 1
    y = (np.arange(H) + 0.5) / H * 2 - 1
    X, Y = np.meshgrid(x, y)
    bg = 3.0 + 0.4 * X - 0.3 * Y - 0.5 * X * X + 0.2 * X * Y - 0.6 * Y * Y
    # a pure quadric divides to a constant -> zero after normalisation
    assert np.abs(oracle.preprocess(bg, True)).max() < 1e-9
    # a texture on top of a quadric: the background is largely removed
    tex = 1.0 + 0.05 * np.sin(1.3 * X * 7) * np.cos(2.1 * Y * 5)
    out = oracle.preprocess(bg * tex, True)
    ref = oracle.normalize(tex)
    assert np.corrcoef(out.ravel(), ref.ravel())[0, 1] > 0.99
    # flat=False is plain normalisation
    assert np.allclose(oracle.preprocess(bg, False), oracle.normalize(bg), atol=1e-12)


def test_reduce2_is_box_mean(oracle):
    x = rng.normal(size=(12, 20))
    assert np.allclose(oracle.reduce2(x), x.reshape(6, 2, 10, 2).mean(axis=(1, 3)), atol=1e-14)


# ------------------------------------------------------------------ a2
def test_gauss_taps(oracle):
    t = oracle.gauss_taps(1.0)
    assert len(t) == 7 and abs(t.sum() - 1) < 1e-15 and np.allclose(t, t[::-1])
    assert abs(t[4] / t[3] - math.exp(-0.5)) < 1e-14 and abs(t[5] / t[3] - math.exp(-2.0)) < 1e-14
    assert len(oracle.gauss_taps(1.5)) == 11
    assert np.array_equal(oracle.gauss_taps(0.0), [1.0])


def test_smooth_equals_direct_2d_convolution(oracle):
    x = rng.normal(size=(19, 26))
    for sigma in (0.7, 1.0, 2.0):
        t = oracle.gauss_taps(sigma)
        r = len(t) // 2
        direct = convolve2d(np.pad(x, r, mode="edge"), np.outer(t, t)[::-1, ::-1], mode="valid")
        assert np.abs(oracle.smooth(x, sigma) - direct).max() < 1e-12
    assert np.abs(oracle.smooth(np.full((9, 9), 2.5), 1.0) - 2.5).max() < 1e-14
    imp = np.zeros((15, 15))
    imp[7, 7] = 1.0
    t = oracle.gauss_taps(1.0)
    assert np.abs(oracle.smooth(imp, 1.0)[4:11, 4:11] - np.outer(t, t)).max() < 1e-16
    assert np.array_equal(oracle.smooth(x, 0.0), x)


def test_gradient_of_polynomials(oracle):
    H, W = 9, 11
    Y, X = np.mgrid[0:H, 0:W].astype(float)
    gx, gy = oracle.gradient(2.0 * X - 3.0 * Y + 1.0)
    assert np.allclose(gx, 2.0, atol=1e-14) and np.allclose(gy, -3.0, atol=1e-14)
    gx, gy = oracle.gradient(X * X + Y * Y * Y)
    assert np.allclose(gx[:, 1:-1], 2 * X[:, 1:-1], atol=1e-12)          # central diff exact for x^2
    assert np.allclose(gy[1:-1, :], 3 * Y[1:-1, :] ** 2 + 1, atol=1e-12)  # (y+1)^3-(y-1)^3 = 6y^2 + 2
    assert np.allclose(gx[:, 0], 1.0) and np.allclose(gx[:, -1], (W - 1) ** 2 - (W - 2) ** 2)


def test_bilinear_nodes_linear_and_clamp(oracle):
    img = rng.normal(size=(6, 7))
    for (i, j) in [(0, 0), (2, 3), (5, 6), (5, 0)]:
        assert oracle.bilinear(img, j, i) == img[i, j]
    Y, X = np.mgrid[0:6, 0:7].astype(float)
    lin = 0.3 * X - 1.7 * Y + 2
    for x, y in [(0.25, 0.5), (3.7, 4.2), (5.99, 4.999)]:
        assert abs(oracle.bilinear(lin, x, y) - (0.3 * x - 1.7 * y + 2)) < 1e-13
    assert oracle.bilinear(img, -3.0, -1.0) == img[0, 0]
    assert oracle.bilinear(img, 50.0, 2.0) == img[2, 6]


def test_warp_zero_and_integer_shift(oracle):
    M = rng.normal(size=(10, 12))
    u = np.zeros((2, 10, 12))
    assert np.array_equal(oracle.warp(M, u), M)
    u[0], u[1] = 2.0, -1.0            # Mw(x) = M(x - u)
    w = oracle.warp(M, u)
    assert np.array_equal(w[0:8, 2:12], M[1:9, 0:10])


def test_demons_force_closed_form(oracle):
    # F = M = linear ramp a x; constant field t: Mw = a (x - t), d = -a t, grad = (a, 0)
    # du_x = d a / (a^2 + alpha^2 d^2) = -t / (1 + alpha^2 t^2)
    H, W, a, t = 8, 16, 0.7, 0.4
    X = np.tile(np.arange(W, dtype=float), (H, 1))
    img = a * X
    u = np.zeros((2, H, W))
    u[0] = t
    for alpha in (1.0, 2.0):
        du, ssd = oracle.demons_force(img, img, u, alpha)
        assert np.allclose(du[0][:, 2:-2], -t / (1 + alpha ** 2 * t ** 2), atol=1e-14)
        assert np.abs(du[1]).max() == 0.0
    # identical pair at zero field: no force, zero SSD
    P = rng.normal(size=(12, 12))
    du, ssd = oracle.demons_force(P, P, np.zeros((2, 12, 12)), 1.0)
    assert ssd == 0.0 and np.abs(du).max() == 0.0


def _pattern(H, W, pc_shift=(0.0, 0.0), F=None, seed=7, noise=False, background=False):
    g = K.random_rotation(seed, 0)
    return K.render(g, np.eye(3) if F is None else F, H, W, K.Geometry(), noise=noise, background=background,
                    pc_shift=pc_shift, seed=seed, stream=1).astype(np.float64)


def test_identical_pair_gives_zero_field(oracle):
    P = oracle.preprocess(_pattern(32, 32, noise=True), True)
    field, iters = oracle.demons_register(P, P, 2, [20, 20], 1.0, 1.0, 1.0)
    assert np.abs(field).max() == 0.0 and list(iters) == [20, 20]


def test_ssd_decreases(oracle):
    ref = oracle.preprocess(_pattern(48, 48))
    test = oracle.preprocess(_pattern(48, 48, F=K.axis_angle([0.2, 0.5, 1.0], math.radians(1.5))))
    u, k, trace = oracle.demons_level(test, ref, np.zeros((2, 48, 48)), 1.0, 1.0, 1.0, 40)
    # large steady decrease while the images are misregistered; afterwards the
    # field smoothing trades a little SSD for smoothness, so only a bound holds
    assert np.all(np.diff(trace[:6]) < 0)
    assert trace[-1] < 0.2 * trace[0] and trace[-1] < 1.1 * trace.min()


def test_stop_rule_and_replay(oracle):
    ref = oracle.preprocess(_pattern(32, 32))
    test = oracle.preprocess(_pattern(32, 32, pc_shift=(0.6, -0.3)))
    u0 = np.zeros((2, 32, 32))
    u, k, tr = oracle.demons_level(test, ref, u0, 1.0, 1.0, 1.0, 200, window=5, tol=1e-3)
    assert 5 <= k < 200
    assert (tr[k - 5] - tr[k]) < 1e-3 * tr[k - 5]                                # stop condition met at k
    assert all((tr[j - 5] - tr[j]) >= 1e-3 * tr[j - 5] for j in range(5, k))    # and not before
    u2, k2, _ = oracle.demons_level(test, ref, u0, 1.0, 1.0, 1.0, 200, replay=k)
    assert k2 == k and np.array_equal(u, u2)


def test_subpixel_translation_recovered(oracle):
    t = (0.37, -0.21)
    ref = oracle.preprocess(_pattern(64, 64), False)
    test = oracle.preprocess(_pattern(64, 64, pc_shift=t), False)
    field, _ = oracle.demons_register(ref, test, 3, [100, 100, 100], 1.0, 1.0, 1.0)
    inner = field[:, 12:-12, 12:-12]
    for c in range(2):
        assert abs(inner[c].mean() - t[c]) < 0.02
        assert np.median(np.abs(inner[c] - t[c])) < 0.1


# ------------------------------------------------------------------ a4
def test_prolong_constant_and_linear(oracle):
    uc = np.zeros((2, 5, 6))
    uc[0], uc[1] = 0.75, -1.25
    uf = oracle.prolong(uc)
    assert uf.shape == (2, 10, 12) and np.allclose(uf[0], 1.5) and np.allclose(uf[1], -2.5)
    Yc, Xc = np.mgrid[0:5, 0:6].astype(float)
    uc[0], uc[1] = 0.3 * Xc, 0.1 * Yc
    uf = oracle.prolong(uc)
    Yf, Xf = np.mgrid[0:10, 0:12].astype(float)
    # interior: 2 * a * ((x_f + 0.5)/2 - 0.5) = a (x_f - 0.5)
    assert np.allclose(uf[0][:, 1:-1], 0.3 * (Xf[:, 1:-1] - 0.5), atol=1e-13)
    assert np.allclose(uf[1][1:-1, :], 0.1 * (Yf[1:-1, :] - 0.5), atol=1e-13)


# ------------------------------------------------------------------ a5, a8 (Eq. 2-5)
def _project(F, pts, xpc, ypc, zs):
    r = np.c_[pts[:, 0] - xpc, pts[:, 1] - ypc, np.full(len(pts), zs)]
    v = (F @ r.T).T
    return zs * v[:, :2] / v[:, 2:3] + [xpc, ypc]


def test_fit_F_recovers_known_deformation(oracle):
    xpc, ypc, zs = 64.0, 64.0, 76.8
    roi = K.roi_grid(128, 128, 32, True).astype(float)
    for trial in range(5):
        eps = rng.normal(0, 1e-3, (3, 3))
        F = K.axis_angle(rng.normal(size=3), math.radians(rng.uniform(0.5, 12))) @ (np.eye(3) + (eps + eps.T) / 2)
        Fh = oracle.fit_F(roi, _project(F, roi, xpc, ypc, zs), xpc, ypc, zs)
        assert np.abs(Fh - F / np.cbrt(np.linalg.det(F))).max() < 1e-11
        assert abs(np.linalg.det(Fh) - 1) < 1e-13


def test_fit_F_is_least_squares_optimum(oracle):
    xpc, ypc, zs = 128.0, 128.0, 153.6
    roi = K.roi_grid(256, 256, 64, False).astype(float)
    F = K.axis_angle([1, 2, 3], math.radians(4))
    obs = _project(F, roi, xpc, ypc, zs) + rng.normal(0, 0.3, roi.shape)
    Fh = oracle.fit_F(roi, obs, xpc, ypc, zs)

    def cost(G):
        return 0.5 * np.sum((_project(G, roi, xpc, ypc, zs) - obs) ** 2)

    c0 = cost(Fh)
    for _ in range(20):   # any perturbation raises the Eq. 3 objective
        assert cost(Fh + rng.normal(0, 1e-5, (3, 3))) >= c0 - 1e-12


def test_polar_rotation(oracle):
    for _ in range(5):
        R = K.axis_angle(rng.normal(size=3), rng.uniform(0, 3))
        A = rng.normal(size=(3, 3))
        U = np.eye(3) + 0.05 * (A @ A.T)
        assert np.abs(oracle.polar(R @ U) - R).max() < 1e-13
        assert np.abs(oracle.polar(R) - R).max() < 1e-14


def test_fit_rotation_reads_field_at_roi_centres(oracle):
    # field of a pure rotation built on the pixel grid: u(x) = x - proj(F^-1 x)
    H = W = 128
    geom = K.Geometry()
    xpc, ypc, zs = 64.0, 64.0, 76.8
    F = K.axis_angle([0.3, -0.2, 0.9], math.radians(3))
    Y, X = np.mgrid[0:H, 0:W].astype(float)
    pts = np.c_[X.ravel() + 0.5, Y.ravel() + 0.5]
    src = _project(np.linalg.inv(F), pts, xpc, ypc, zs)
    field = (pts - src).T.reshape(2, H, W)
    roi = K.roi_grid(H, W, 32, True).astype(float)
    F1, R = oracle.fit_rotation(field, roi, geom)
    assert rot_err(R, F) < 2e-5


# ------------------------------------------------------------------ a6
def test_remap_identity_and_inverse(oracle):
    geom = K.Geometry()
    img = _pattern(64, 64)
    assert np.abs(oracle.remap(img, np.eye(3), geom) - img).max() < 1e-9 * np.abs(img).max()
    R = K.axis_angle([0.1, 0.7, 0.3], math.radians(2))
    back = oracle.remap(oracle.remap(img, R, geom), R.T, geom)
    assert np.abs(back - img)[16:-16, 16:-16].max() < 0.02 * np.abs(img).max()


def test_remap_matches_rendered_rotation(oracle):
    # the remapped reference must look like a pattern rendered with the rotation (Eq. 2 direction)
    geom = K.Geometry()
    R = K.axis_angle([0.2, 0.4, 1.0], math.radians(2))
    ref, test = _pattern(128, 128), _pattern(128, 128, F=R)
    good = np.abs(oracle.remap(ref, R, geom) - test)[16:-16, 16:-16].max()
    bad = np.abs(oracle.remap(ref, R.T, geom) - test)[16:-16, 16:-16].max()
    assert good < 0.01 * np.abs(test).max() and bad > 20 * good


# ------------------------------------------------------------------ a7
def test_fft_matches_library(oracle):
    for n in (8, 32, 64):
        x = rng.normal(size=n) + 1j * rng.normal(size=n)
        r, i = oracle.fft(x.real, x.imag)
        assert np.abs((r + 1j * i) - np.fft.fft(x)).max() < 1e-12 * n
        r, i = oracle.fft(x.real, x.imag, inverse=True)
        assert np.abs((r + 1j * i) - np.fft.ifft(x)).max() < 1e-13
    x = rng.normal(size=(16, 16))
    r, i = oracle.fft2(x, np.zeros_like(x))
    assert np.abs((r + 1j * i) - np.fft.fft2(x)).max() < 1e-11


def test_xcf_surface_equals_direct_correlation(oracle):
    S = 16
    a, b = rng.normal(size=(40, 40)), rng.normal(size=(40, 40))
    x0, y0 = 7, 11
    for window in (False, True):
        c, nr, nt = oracle.xcf_surface(a, b, x0, y0, S, window)
        n = np.arange(S)
        w = 0.5 * (1 - np.cos(2 * np.pi * n / (S - 1))) if window else np.ones(S)
        A = a[y0:y0 + S, x0:x0 + S]
        B = b[y0:y0 + S, x0:x0 + S]
        A = (A - A.mean()) * np.outer(w, w)
        B = (B - B.mean()) * np.outer(w, w)
        direct = np.zeros((S, S))
        for sy in range(S):
            for sx in range(S):   # c(s) = sum_x test(x + s) ref(x), circular
                direct[sy, sx] = np.sum(np.roll(B, (-sy, -sx), axis=(0, 1)) * A)
        assert np.abs(c - direct).max() < 1e-10 * np.abs(direct).max()
        assert abs(nr - np.linalg.norm(A)) < 1e-12 and abs(nt - np.linalg.norm(B)) < 1e-12


def test_xcf_integer_circular_shift_exact(oracle):
    S = 32
    base = rng.normal(size=(S, S))
    for (dx, dy) in [(3, -2), (0, 5), (-7, -7), (15, 1)]:
        shifted = np.roll(base, (dy, dx), axis=(0, 1))     # test(x) = ref(x - q), q = (dx, dy)
        q, peak, ph, tie = oracle.xcf_roi(base, shifted, np.array([[S // 2, S // 2]]), S, window=False)
        assert tuple(peak[0]) == (dx, dy)
        assert np.abs(q[0] - [dx, dy]).max() < 1e-9
        assert abs(ph[0] - 1.0) < 1e-12 and not tie[0]


def test_xcf_identical_rois(oracle):
    img = _pattern(128, 128)
    roi = K.roi_grid(128, 128, 32, True)
    q, peak, ph, tie = oracle.xcf_roi(img, img, roi, 32)
    assert np.all(peak == 0) and np.abs(q).max() < 1e-9 and np.allclose(ph, 1.0, atol=1e-12)


def test_xcf_subpixel_sign_and_size(oracle):
    # periodic band-limited ROI content, shifted exactly by a Fourier phase ramp
    S = 32
    k = np.fft.fftfreq(S) * S
    KX, KY = np.meshgrid(k, k)
    spec = np.fft.fft2(rng.normal(size=(S, S))) * np.exp(-(KX ** 2 + KY ** 2) / (2 * 3.0 ** 2))
    ref = np.real(np.fft.ifft2(spec))
    for t in [(0.3, -0.4), (-0.2, 0.15), (1.25, 0.45)]:
        test = np.real(np.fft.ifft2(spec * np.exp(-2j * np.pi * (KX * t[0] + KY * t[1]) / S)))
        q, peak, ph, tie = oracle.xcf_roi(ref, test, np.array([[S // 2, S // 2]]), S, window=False)
        assert tuple(peak[0]) == (int(round(t[0])), int(round(t[1])))
        assert np.all(np.sign(q[0] - peak[0]) == np.sign(np.array(t) - peak[0]))
        assert np.abs(q[0] - t).max() < 0.1


def test_solve_F_composes_with_R_finite(oracle):
    H = W = 256
    geom = K.Geometry()
    xpc, ypc, zs = 128.0, 128.0, 153.6
    roi = K.roi_grid(H, W, 64, False)
    Finf = K.axis_angle([1, 0, 1], math.radians(0.05)) @ (np.eye(3) + np.diag([3e-4, -2e-4, 1e-4]))
    Rf = K.axis_angle([0, 1, 2], math.radians(6))
    q = _project(Finf, roi.astype(float), xpc, ypc, zs) - roi
    F = oracle.solve_F(q, roi, H, W, geom, Rf)
    Fi = Finf / np.cbrt(np.linalg.det(Finf))
    assert np.abs(F - Fi @ Rf).max() < 1e-11          # Eq. 12: F = F_inf R_finite
    assert np.abs(F - Rf @ Fi).max() > 1e-5            # (and not the other order)
    assert np.abs(oracle.solve_F(q, roi, H, W, geom) - Fi).max() < 1e-11


# ------------------------------------------------------------------ a12 + paper's printed values
def _bunge(phi1, Phi, phi2):
    def rz(a):
        return np.array([[math.cos(a), math.sin(a), 0], [-math.sin(a), math.cos(a), 0], [0, 0, 1]])

    def rx(a):
        return np.array([[1, 0, 0], [0, math.cos(a), math.sin(a)], [0, -math.sin(a), math.cos(a)]])
    return rz(phi2) @ rx(Phi) @ rz(phi1)


def test_axis_angle_and_paper_orientations(oracle):
    gold = json.load(open(os.path.join(GOLDEN, "paper_orientations.json")))
    s1 = gold["test_set_1"]
    assert abs(math.radians(s1["tests_deg"][0][0]) - s1["first_rad"][0]) < 5e-5
    assert abs(math.radians(s1["tests_deg"][-1][0]) - s1["last_rad"][0]) < 5e-5
    for e in s1["tests_deg"]:
        g = _bunge(*np.radians(e))
        m, th, om = oracle.axis_angle(g.T @ _bunge(0, 0, 0))
        # rotation about the screen normal only: a single in-plane component omega_12
        assert abs(th - math.radians(e[0])) < 1e-12
        assert abs(abs(om[1, 0]) - math.radians(e[0])) < 1e-12 and abs(om[2, 1]) < 1e-15 and abs(om[0, 2]) < 1e-15
        assert np.allclose(om, -om.T)
    s2 = gold["test_set_2"]
    assert np.allclose(np.radians(s2["reference_deg"]), s2["reference_rad"], atol=5e-5)
    assert np.allclose(np.radians(s2["test_deg"]), s2["test_rad"], atol=5e-5)
    ga, gb = _bunge(*np.radians(s2["reference_deg"])), _bunge(*np.radians(s2["test_deg"]))
    m, th, om = oracle.axis_angle(gb @ ga.T)
    assert abs(math.degrees(th) - s2["misorientation_deg_approx"]) < 0.5
    assert abs(np.linalg.norm(m) - 1) < 1e-12
    R = K.axis_angle([0.3, 0.4, 0.5], 0.01)
    m, th, om = oracle.axis_angle(R)
    assert abs(th - 0.01) < 1e-12 and np.allclose(om, (R - R.T) / 2, atol=1e-6)


# ------------------------------------------------------------------ end to end (sanity band)
def test_end_to_end_recovers_known_rotation(oracle):
    spec = K.config1()
    g = K.ref_orientation(spec, 0)
    F = K.pair_truth(spec, 0)
    ref = K.render(g, np.eye(3), 128, 128, spec.geom, noise=False).astype(np.float64)
    test = K.render(g, F, 128, 128, spec.geom, noise=False).astype(np.float64)
    roi = K.roi_grid(128, 128, 32, True)
    res = oracle.pipeline(ref, test, roi, 32, spec.geom, 3, [50, 50, 50])
    Rt = oracle.polar(F)
    e_final = rot_err(oracle.polar(res["F"]), Rt)
    e_none = rot_err(np.eye(3), Rt)
    # measured 7.1e-4 rad; the floor is the XCF's parabolic sub-pixel estimate (test below)
    assert e_final < 0.05 * e_none and e_final < 1.5e-3
    assert rot_err(res["R_finite"], Rt) < 0.25 * e_none


def test_end_to_end_error_budget(oracle):
    """Where the rotation error of a noise-free pair comes from (the config-1 pair: 2 deg, 128x128,
    3 levels x 50 iterations, 21 ROIs of 32x32), stage by stage:
    - the shift-to-F convention (Eq. 2-3, Eq. 12): the exact projective shifts of the residual
      deformation at the ROI centres give back the rotation to rounding;
    - the remap interpolation (bicubic, Eq. 12): the reference rendered at the remap rotation instead
      of interpolated changes the final error by little;
    - the XCF shifts: their error (0.04 px rms here) is the floor, and it is the parabolic sub-pixel
      fit's: on the reference pattern shifted by exact Fourier phase ramps the estimate is pulled toward
      the integer (0.3 px is read as 0.23 px on average, 0.07 px at worst); at ROIs where one band
      dominates, the correlation peak is a ridge along the band, and its y reading under a pure x shift
      wanders by up to 0.35 px (the aperture problem of a one-dimensional feature), which the
      least-squares fit over 21 ROIs averages."""
    spec = K.config1()
    H = W = 128
    geom = spec.geom
    g = K.ref_orientation(spec, 0)
    F = K.pair_truth(spec, 0)
    Rt = oracle.polar(F)
    ref = K.render(g, np.eye(3), H, W, geom, noise=False).astype(np.float64)
    test = K.render(g, F, H, W, geom, noise=False).astype(np.float64)
    roi = K.roi_grid(H, W, 32, True)
    res = oracle.pipeline(ref, test, roi, 32, geom, 3, [50, 50, 50])
    R = res["R_finite"]
    e_final = rot_err(oracle.polar(res["F"]), Rt)
    # exact shifts of the deformation left after the remap, F R^T, at the ROI centres
    q_exact = _project(F @ R.T, roi.astype(float), geom.xstar * W, geom.ystar * H, geom.zstar * W) - roi
    assert np.abs(oracle.polar(oracle.solve_F(q_exact, roi, H, W, geom, R)) - Rt).max() < 1e-12
    # remap by rendering instead of interpolating
    pref_exact = oracle.preprocess(K.render(g, R, H, W, geom, noise=False).astype(np.float64), True)
    q2, _, _, _ = oracle.xcf_roi(pref_exact, res["ptest"], roi, 32)
    e_exact_remap = rot_err(oracle.polar(oracle.solve_F(q2, roi, H, W, geom, R)), Rt)
    assert abs(e_exact_remap - e_final) < 0.25 * e_final + 1e-4
    # the XCF shift error against the exact shifts
    rms = float(np.sqrt(np.mean((res["q"] - q_exact) ** 2)))
    assert 0.01 < rms < 0.15
    # the parabolic fit's bias on exact sub-pixel shifts of the reference
    pref = res["pref"]
    P = np.fft.fft2(pref)
    fx = np.fft.fftfreq(W)[None, :]
    shifted = np.real(np.fft.ifft2(P * np.exp(-2j * np.pi * fx * 0.3)))   # features move by +0.3 px in x
    q3, _, _, _ = oracle.xcf_roi(pref, shifted, roi, 32)
    bias = q3[:, 0] - 0.3
    assert -0.15 < bias.mean() < -0.02 and np.all(bias < 0)
