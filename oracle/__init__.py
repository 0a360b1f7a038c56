"""FP64 CPU oracle of the HR-EBSD demons-remapping method -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``hrebsd_oracle.c`` (plain C, FP64,
single-threaded) through ctypes; the wrappers below only marshal numpy arrays.
It shares no code with the CUDA library and never calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hrebsd_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    i, d, l_ = C.c_int, C.c_double, C.c_long
    sig = {
        "oracle_normalize": (None, [_D, l_, _D]),
        "oracle_preprocess": (None, [_D, i, i, i, _D]),
        "oracle_reduce2": (None, [_D, i, i, _D]),
        "oracle_gauss_taps": (i, [d, _D]),
        "oracle_smooth": (None, [_D, i, i, d, _D]),
        "oracle_gradient": (None, [_D, i, i, _D, _D]),
        "oracle_bilinear": (d, [_D, i, i, d, d]),
        "oracle_warp": (None, [_D, _D, i, i, _D]),
        "oracle_demons_force": (d, [_D, _D, _D, _D, _D, i, i, d, _D]),
        "oracle_demons_level": (i, [_D, _D, i, i, _D, d, d, d, i, i, d, i, C.c_void_p]),
        "oracle_prolong": (None, [_D, i, i, _D]),
        "oracle_prolong_to": (None, [_D, i, i, i, i, _D]),
        "oracle_demons_register": (i, [_D, _D, i, i, i, _I, d, d, d, i, d, i, C.c_void_p, C.c_void_p, _D, _I]),
        "oracle_fit_F": (i, [_D, _D, i, d, d, d, _D]),
        "oracle_polar": (None, [_D, _D]),
        "oracle_fit_rotation": (i, [_D, i, i, _D, i, d, d, d, _D, _D]),
        "oracle_remap": (None, [_D, i, i, _D, d, d, d, _D]),
        "oracle_fft": (None, [_D, _D, i, i]),
        "oracle_fft2": (None, [_D, _D, i, i]),
        "oracle_xcf_surface": (None, [_D, _D, i, i, i, i, i, _D, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "oracle_xcf_roi": (None, [_D, _D, i, i, _I, i, i, i, _D, _I, _D, _I]),
        "oracle_solve_F": (i, [_D, _D, i, i, i, d, d, d, C.c_void_p, _D]),
        "oracle_axis_angle": (None, [_D, _D, C.POINTER(C.c_double), _D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ wrappers
def normalize(img):
    a = _d(img)
    out = np.empty_like(a)
    _load().oracle_normalize(a, a.size, out)
    return out


def preprocess(img, flat=True):
    a = _d(img)
    H, W = a.shape
    out = np.empty_like(a)
    _load().oracle_preprocess(a, H, W, int(flat), out)
    return out


def reduce2(img):
    a = _d(img)
    H, W = a.shape
    out = np.empty((H // 2, W // 2))
    _load().oracle_reduce2(a, H, W, out)
    return out


def gauss_taps(sigma):
    taps = np.zeros(65)
    r = _load().oracle_gauss_taps(float(sigma), taps)
    return taps[: 2 * r + 1]


def smooth(img, sigma):
    a = _d(img)
    H, W = a.shape
    out = np.empty_like(a)
    _load().oracle_smooth(a, H, W, float(sigma), out)
    return out


def gradient(img):
    a = _d(img)
    H, W = a.shape
    gx, gy = np.empty_like(a), np.empty_like(a)
    _load().oracle_gradient(a, H, W, gx, gy)
    return gx, gy


def bilinear(img, x, y):
    a = _d(img)
    return _load().oracle_bilinear(a, a.shape[0], a.shape[1], float(x), float(y))


def warp(M, u):
    a, uu = _d(M), _d(u)
    H, W = a.shape
    out = np.empty_like(a)
    _load().oracle_warp(a, uu, H, W, out)
    return out


def demons_force(Fimg, M, u, alpha):
    f, m, uu = _d(Fimg), _d(M), _d(u)
    H, W = f.shape
    gx, gy = gradient(f)
    du = np.empty((2, H, W))
    ssd = _load().oracle_demons_force(f, gx, gy, m, uu, H, W, float(alpha), du)
    return du, ssd


def demons_level(Fimg, M, u0, alpha, sigma_up, sigma_f, cap, window=0, tol=0.0, replay=-1):
    f, m = _d(Fimg), _d(M)
    H, W = f.shape
    u = _d(u0).copy()
    trace = np.zeros(max(cap, 1))
    k = _load().oracle_demons_level(f, m, H, W, u, float(alpha), float(sigma_up), float(sigma_f), int(cap),
                                    int(window), float(tol), int(replay), _ptr(trace))
    return u, k, trace[:min(k + 1, cap)]


def prolong(uc, H=None, W=None):
    """Field of the next finer level: 2h x 2w, or the stored size H x W of that level (one more row or
    column where the size did not halve)."""
    a = _d(uc)
    _, h, w = a.shape
    H = 2 * h if H is None else int(H)
    W = 2 * w if W is None else int(W)
    out = np.empty((2, H, W))
    _load().oracle_prolong_to(a, h, w, H, W, out)
    return out


def demons_register(ref, test, levels, caps, alpha=1.0, sigma_up=1.0, sigma_f=1.0, window=0, tol=0.0,
                    start_level=-1, init=None, replay=None):
    r, t = _d(ref), _d(test)
    H, W = r.shape
    caps = _i(np.broadcast_to(np.asarray(caps), (levels,)))
    init_a = None if init is None else _d(init)
    replay_a = None if replay is None else _i(replay)
    field = np.empty((2, H, W))
    iters = np.zeros(levels, dtype=np.int32)
    st = _load().oracle_demons_register(r, t, H, W, int(levels), caps, float(alpha), float(sigma_up),
                                        float(sigma_f), int(window), float(tol), int(start_level),
                                        _ptr(init_a), _ptr(replay_a), field, iters)
    if st:
        raise ValueError(f"oracle_demons_register failed ({st})")
    return field, iters


def fit_F(ref_xy, test_xy, xpc, ypc, zs):
    a, b = _d(ref_xy), _d(test_xy)
    F = np.empty(9)
    st = _load().oracle_fit_F(a, b, a.shape[0], float(xpc), float(ypc), float(zs), F)
    if st:
        raise ValueError("oracle_fit_F: degenerate")
    return F.reshape(3, 3)


def polar(F):
    R = np.empty(9)
    _load().oracle_polar(_d(F).reshape(9), R)
    return R.reshape(3, 3)


def fit_rotation(field, roi_xy, geom):
    f = _d(field)
    _, H, W = f.shape
    roi = _d(roi_xy)
    F1, R = np.empty(9), np.empty(9)
    st = _load().oracle_fit_rotation(f, H, W, roi, roi.shape[0], geom.xstar, geom.ystar, geom.zstar, F1, R)
    if st:
        raise ValueError("oracle_fit_rotation: degenerate")
    return F1.reshape(3, 3), R.reshape(3, 3)


def remap(ref, R, geom):
    a = _d(ref)
    H, W = a.shape
    out = np.empty_like(a)
    _load().oracle_remap(a, H, W, _d(R).reshape(9), geom.xstar, geom.ystar, geom.zstar, out)
    return out


def fft(re, im, inverse=False):
    r, i = _d(re).copy(), _d(im).copy()
    _load().oracle_fft(r, i, r.size, int(inverse))
    return r, i


def fft2(re, im, inverse=False):
    r, i = _d(re).copy(), _d(im).copy()
    _load().oracle_fft2(r, i, r.shape[0], int(inverse))
    return r, i


def xcf_surface(ref_img, test_img, x0, y0, S, window=True):
    a, b = _d(ref_img), _d(test_img)
    c = np.empty((S, S))
    nr, nt = C.c_double(), C.c_double()
    _load().oracle_xcf_surface(a, b, a.shape[1], int(x0), int(y0), int(S), int(window), c, C.byref(nr),
                               C.byref(nt))
    return c, nr.value, nt.value


def xcf_roi(ref_img, test_img, roi_xy, S, window=True):
    a, b = _d(ref_img), _d(test_img)
    H, W = a.shape
    roi = _i(roi_xy)
    N = roi.shape[0]
    q = np.empty((N, 2))
    peak = np.empty((N, 2), dtype=np.int32)
    ph = np.empty(N)
    tie = np.empty(N, dtype=np.int32)
    _load().oracle_xcf_roi(a, b, H, W, roi, N, int(S), int(window), q, peak, ph, tie)
    return q, peak, ph, tie.astype(bool)


def solve_F(q, roi_xy, H, W, geom, R_finite=None):
    qq, roi = _d(q), _d(roi_xy)
    Rf = None if R_finite is None else _d(R_finite).reshape(9)
    F = np.empty(9)
    st = _load().oracle_solve_F(qq, roi, roi.shape[0], H, W, geom.xstar, geom.ystar, geom.zstar, _ptr(Rf), F)
    if st:
        raise ValueError("oracle_solve_F: degenerate")
    return F.reshape(3, 3)


def pipeline(ref, test, roi_xy, S, geom, levels, caps, alpha=1.0, sigma=1.0, window=0, tol=0.0,
             replay=None, init=None, start_level=-1, flat=True):
    """The whole hot path for one pair: preprocess, register, fit, remap, XCF, solve."""
    pref, ptest = preprocess(ref, flat), preprocess(test, flat)
    field, iters = demons_register(pref, ptest, levels, caps, alpha, sigma, sigma, window, tol,
                                   start_level, init, replay)
    F1, R = fit_rotation(field, roi_xy, geom)
    rem = remap(pref, R, geom)
    q, peak, ph, tie = xcf_roi(rem, ptest, roi_xy, S)
    F = solve_F(q, roi_xy, ref.shape[0], ref.shape[1], geom, R)
    return dict(field=field, iters=iters, F_first=F1, R_finite=R, remapped=rem, q=q, peak=peak, ph=ph,
                near_tie=tie, F=F, pref=pref, ptest=ptest)


def axis_angle(R):
    """(axis m, angle theta, lattice rotation tensor omega) of a rotation (Eq. 6-7)."""
    m, om = np.empty(3), np.empty(9)
    th = C.c_double()
    _load().oracle_axis_angle(_d(R).reshape(9), m, C.byref(th), om)
    return m, th.value, om.reshape(3, 3)
