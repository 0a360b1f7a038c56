"""How far the FP64 oracle's own demons field moves under FP32-sized perturbations -- TEST HELPER.

The demons iteration (Eq. 1) amplifies small differences at a few pixels: where both the
test-image gradient and the residual d are near zero the force d grad F / (|grad F|^2 + alpha^2 d^2)
turns fast, and at the finest level a perturbation of 1e-6 px entering the level can grow to
1e-2 px over a hundred iterations.  An FP32 implementation carries perturbations of that size (its
field differs from the FP64 one by ~1e-6 px at the start of a level), so beyond ~10 iterations per
level the field cannot agree with the FP64 oracle to 1e-3 px at every pixel; which pixels diverge
depends on the direction of the perturbation, so it cannot be certified pixel by pixel either.

``perturbed_fields`` runs the oracle's registration (its gradient, warp, smoothing, box pyramid and
prolongation, in the oracle's order and with the force of Eq. 1 written out in numpy) with every
stored intermediate rounded to FP32 by seeded stochastic rounding (up or down with the probabilities
that make the rounding unbiased): the preprocessed images, the pyramid, the test-image gradient,
the warped moving image, d, the force denominator and quotient, du, each smoothing pass, the field
after each update and after prolongation.  Each seed is one FP32 execution of the method; the
members' spread is how far FP32 storage alone moves the FP64 result.  Where the field under test
came from FP32-preprocessed patterns (end-to-end tests), the members' images also carry uniform
noise of +-`input_ulps` FP32 units, the size of the FP32 preprocessing error (``preprocess_ulps``
measures it on the patterns at hand; test_preprocess_parity holds it within 32 units).  ``assert_field_parity`` then holds the deviation d(x) = |got - oracle| to the distribution
of the members' own deviations from the oracle: at the quantiles 99 %, 99.9 %, 99.99 % and the
maximum, d is at most max(1e-3 px, 3 x the largest member's value of that quantile), and the
fraction of pixels with d > 1e-3 px is at most 3 x the largest member's fraction plus the larger of 1e-4 and
four pixels (the tail
of a chaotic response is heavy: the members' own maxima differ by up to 10x).  In words: the FP32
field is no further from the FP64 oracle than the FP64 oracle is from itself under FP32-sized
perturbations, at every level of the distribution up to the worst pixel.  ``strict`` holds every
pixel to 1e-3 px instead (the bar for runs short enough not to reach the unstable regime).

``arithmetic_fields`` is the stronger model: every elementary operation of the iteration (each
product and sum of the smoothing passes, of the bilinear warp, of d, of the force denominator, of the
quotient and of the update) rounded to FP32 by the same seeded stochastic rounding, as an FP32
implementation rounds each operation.  Storage rounding keeps the arithmetic in FP64 between
stores, and at a pixel where the iteration has two nearby fixed points (the force of Eq. 1 is not
monotone in d) it can miss the branch that FP32 arithmetic reaches: one training pair (178925 of the
training set) has such a pixel, where 64 storage-rounding executions stay within 3.3e-3 px of the
FP64 field while 9 of 16 arithmetic-rounding executions settle 3.5e-2 px away, on the other branch.

Test infrastructure: imports the oracle; only tests use it."""
from __future__ import annotations

import numpy as np

FIELD_TOL = 1e-3


def round32(a, rng):
    """Stochastic rounding of an FP64 array to the FP32 grid: to the neighbour above with probability
    (a - below) / (above - below), so that the rounding is unbiased."""
    a = np.asarray(a, np.float64)
    f = a.astype(np.float32)
    lo = np.where(f.astype(np.float64) > a, np.nextafter(f, np.float32(-np.inf)), f)
    hi = np.nextafter(lo, np.float32(np.inf))
    lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
    span = hi64 - lo64
    p = np.where(span > 0, (a - lo64) / np.where(span > 0, span, 1.0), 0.0)
    return np.where(rng.random(a.shape) < p, hi64, lo64)


def _level_fp32(oracle, F, M, u, n, alpha, sigma_up, sigma_f, rng):
    r = lambda a: round32(a, rng)
    gx, gy = (r(g) for g in oracle.gradient(F))
    for _ in range(n):
        d = r(r(oracle.warp(M, u)) - F)
        den = r(r(gx * gx + gy * gy) + r(alpha * alpha * d * d))
        ok = den > 1e-9
        t = np.where(ok, r(d / np.where(ok, den, 1.0)), 0.0)
        du = (r(t * gx), r(t * gy))
        u = np.stack([r(oracle.smooth(r(u[c] + r(oracle.smooth(du[c], sigma_up))), sigma_f)) for c in range(2)])
    return u


def perturbed_register(oracle, ref, test, levels, iters, alpha=1.0, sigma_up=1.0, sigma_f=1.0, seed=0,
                       init=None, start_level=-1, input_ulps=0):
    """The oracle's multi-resolution registration replaying `iters` updates per level (finest first):
    seed < 0 runs the oracle itself (oracle.demons_level per level); seed >= 0 one FP32-storage
    execution with stochastic rounding seeded by `seed` (see the module docstring)."""
    rng = np.random.default_rng(seed if seed >= 0 else 0)
    r = (lambda a: round32(a, rng)) if seed >= 0 else (lambda a: np.asarray(a, np.float64))
    def noisy(img):
        img = r(img)
        if seed >= 0 and input_ulps:
            sp = np.spacing(np.abs(img).astype(np.float32)).astype(np.float64)
            img = img + rng.uniform(-input_ulps, input_ulps, img.shape) * sp
        return img
    Fp, Mp = [noisy(test)], [noisy(ref)]
    for _ in range(1, levels):
        Fp.append(r(oracle.reduce2(Fp[-1])))
        Mp.append(r(oracle.reduce2(Mp[-1])))
    s = levels - 1 if start_level < 0 or start_level >= levels else start_level
    h, w = Fp[s].shape
    u = np.zeros((2, h, w)) if init is None else r(np.array(init, dtype=np.float64))
    for l in range(s, -1, -1):
        n = int(iters[l])
        if seed >= 0:
            u = _level_fp32(oracle, Fp[l], Mp[l], u, n, alpha, sigma_up, sigma_f, rng)
        else:
            u, k, _ = oracle.demons_level(Fp[l], Mp[l], u, alpha, sigma_up, sigma_f, max(n, 1), 0, 0.0, n)
            assert k == n
        if l > 0:
            u = r(oracle.prolong(u, *Fp[l - 1].shape))
    return u


def preprocess_ulps(got, exp):
    """Largest difference between two preprocessed patterns in FP32 units at the values' magnitude
    (at least that of 1.0): the input error an end-to-end field comparison inherits."""
    exp = np.asarray(exp, np.float64)
    sp = np.spacing(np.maximum(np.abs(exp), 1.0).astype(np.float32)).astype(np.float64)
    return float(np.max(np.abs(np.asarray(got, np.float64) - exp) / sp))


def perturbed_fields(oracle, ref, test, levels, iters, members=4, seed0=1000, **kw):
    return [perturbed_register(oracle, ref, test, levels, iters, seed=seed0 + m, **kw) for m in range(members)]


def _smooth_ops32(img, sigma, r):
    """The oracle's separable Gaussian (x pass, then y pass; replicated borders) with every product and
    every partial sum rounded by r."""
    if sigma <= 0:
        return img
    k = int(np.ceil(3 * sigma))
    j = np.arange(-k, k + 1)
    t = np.exp(-j * j / (2.0 * sigma * sigma))
    t = t / t.sum()
    out = img
    for axis in (1, 0):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (k, k)
        p = np.pad(out, pad, mode="edge")
        n = out.shape[axis]
        sl = (lambda i: p[:, i:i + n]) if axis == 1 else (lambda i: p[i:i + n, :])
        acc = r(t[0] * sl(0))
        for i in range(1, 2 * k + 1):
            acc = r(acc + r(t[i] * sl(i)))
        out = acc
    return out


def _level_ops32(oracle, F, M, u, n, alpha, sigma_up, sigma_f, r):
    """n updates of Eq. 1 at one level, every elementary operation rounded by r."""
    h, w = F.shape
    gx, gy = (r(g) for g in oracle.gradient(F))
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    a2 = alpha * alpha
    for _ in range(n):
        # bilinear sample of M at x - u with replicated borders, each product and sum rounded
        x = np.clip(r(X - u[0]), 0, w - 1)
        y = np.clip(r(Y - u[1]), 0, h - 1)
        x0 = np.minimum(np.floor(x), w - 2).astype(int)
        y0 = np.minimum(np.floor(y), h - 2).astype(int)
        fx, fy = r(x - x0), r(y - y0)
        omx, omy = r(1.0 - fx), r(1.0 - fy)
        top = r(r(omx * M[y0, x0]) + r(fx * M[y0, x0 + 1]))
        bot = r(r(omx * M[y0 + 1, x0]) + r(fx * M[y0 + 1, x0 + 1]))
        mw = r(r(omy * top) + r(fy * bot))
        d = r(mw - F)
        den = r(r(r(gx * gx) + r(gy * gy)) + r(r(a2 * d) * d))
        ok = den > 1e-9
        t = np.where(ok, r(d / np.where(ok, den, 1.0)), 0.0)
        du = (r(t * gx), r(t * gy))
        u = np.stack([_smooth_ops32(r(u[c] + _smooth_ops32(du[c], sigma_up, r)), sigma_f, r) for c in range(2)])
    return u


def arithmetic_register(oracle, ref, test, levels, iters, alpha=1.0, sigma_up=1.0, sigma_f=1.0, seed=0,
                        input_ulps=0):
    """One FP32-arithmetic execution of the registration replaying `iters` updates per level (finest
    first): the inputs, pyramid and prolongation as in perturbed_register, the iteration with every
    elementary operation rounded (module docstring); seed < 0 rounds nothing (FP64 throughout)."""
    rng = np.random.default_rng(seed if seed >= 0 else 0)
    r = (lambda a: round32(a, rng)) if seed >= 0 else (lambda a: np.asarray(a, np.float64))
    def noisy(img):
        img = r(img)
        if seed >= 0 and input_ulps:
            sp = np.spacing(np.abs(img).astype(np.float32)).astype(np.float64)
            img = img + rng.uniform(-input_ulps, input_ulps, img.shape) * sp
        return img
    Fp, Mp = [noisy(test)], [noisy(ref)]
    for _ in range(1, levels):
        Fp.append(r(oracle.reduce2(Fp[-1])))
        Mp.append(r(oracle.reduce2(Mp[-1])))
    u = np.zeros((2,) + Fp[-1].shape)
    for l in range(levels - 1, -1, -1):
        u = _level_ops32(oracle, Fp[l], Mp[l], u, int(iters[l]), alpha, sigma_up, sigma_f, r)
        if l > 0:
            u = r(oracle.prolong(u, *Fp[l - 1].shape))
    return u


def arithmetic_fields(oracle, ref, test, levels, iters, members=4, seed0=5000, **kw):
    return [arithmetic_register(oracle, ref, test, levels, iters, seed=seed0 + m, **kw) for m in range(members)]


def sensitivity(exp, members):
    return np.max([np.abs(m - exp) for m in members], axis=0)


QUANTILES = (0.99, 0.999, 0.9999, 1.0)
FACTOR = 3.0


def assert_field_parity(got, exp, members=None, tol=FIELD_TOL, what="", strict=False):
    """The field bar of the module docstring.  Returns a dict of the measured quantiles."""
    d = np.abs(np.asarray(got, np.float64) - exp)
    out = {"max": float(d.max()), "frac_over": float(np.mean(d > tol))}
    if strict:
        assert d.max() <= tol, (what, "max |d|", float(d.max()))
        return out
    dm = [np.abs(m - exp) for m in members]
    for q in QUANTILES:
        g = float(np.quantile(d, q))
        ref = float(np.max([np.quantile(x, q) for x in dm]))
        out[f"q{q}"] = (g, ref)
        assert g <= max(tol, FACTOR * ref), (what, f"quantile {q}", g, "oracle's own", ref)
    fref = float(np.max([np.mean(x > tol) for x in dm]))
    out["frac_over_oracle"] = fref
    floor = max(1e-4, 4.0 / d.size * 2)   # d holds both field components: four pixels
    assert out["frac_over"] <= FACTOR * fref + floor, (what, "pixels over", out["frac_over"], "oracle's own", fref)
    return out
