"""GB300 (sm_103a) HR-EBSD demons remapping: Python binding of libhrebsd.

The binding marshals arguments only: every step of the method runs in the
CUDA kernels of ``libhrebsd.so`` behind the C ABI declared in
``include/hrebsd.h``.  Functions carry the ABI names and take either torch
CUDA tensors (their ``data_ptr``) or raw device addresses (ints).  A missing
or unloadable library raises immediately; there is no CPU fallback.

Method: Zhu, Kaufmann & Vecchio, "Novel Remapping Approach for HR-EBSD based
on Demons Registration" (arXiv 1907.05993).
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

__all__ = [
    "HrebsdError", "load", "hrebsd_geometry", "hrebsd_demons_params", "demons_params", "hrebsd_create",
    "hrebsd_destroy", "hrebsd_status_string", "hrebsd_launch_count", "hrebsd_preprocess_batch",
    "hrebsd_demons_register_batch", "hrebsd_demons_register_batch_noalloc", "hrebsd_fit_rotation", "hrebsd_remap", "hrebsd_xcf_roi_batch",
    "hrebsd_solve_F", "hrebsd_elastic", "elastic_params", "NORM_DET1", "NORM_TRACTION_FREE", "hrebsd_cnn_save", "hrebsd_cnn_load", "hrebsd_gauss_taps", "hrebsd_strain_stress", "hrebsd_profile_enable", "hrebsd_profile_read", "hrebsd_device_error", "hrebsd_set_option", "OPT_NO_TMA", "OPT_GRAPHS", "OPT_CNN_TC", "OPT_TEX_GATHER", "TILE_VARIANTS",
    "hrebsd_autotune", "hrebsd_probe_fp32_fma", "hrebsd_polar_batch", "hrebsd_tc_selftest", "hrebsd_wait_selftest", "hrebsd_cnn_get_state", "hrebsd_cnn_set_state", "hrebsd_fit_quality", "hrebsd_bandpass_batch", "hrebsd_mean_pattern",
    "hrebsd_background_batch", "hrebsd_shift_zoom_batch", "hrebsd_ssim_warped", "hrebsd_set_tile_variant", "hrebsd_get_tile_variant", "hrebsd_field_resample", "PROF_CLASSES", "PAIR_CAPPED", "PAIR_NONFINITE", "PAIR_FIT_FAILED",
]

PAIR_CAPPED, PAIR_NONFINITE, PAIR_FIT_FAILED = 1, 2, 4
ETIMEOUT, ESCRATCH, EIO, EFORMAT = -4, -5, -6, -7
NOALLOC_SCRATCH_BYTES = 16 << 20

_lib = None


class HrebsdError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().hrebsd_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} ({status})")
        self.status = status


class hrebsd_geometry(C.Structure):
    _fields_ = [("xstar", C.c_double), ("ystar", C.c_double), ("zstar", C.c_double)]


class hrebsd_elastic(C.Structure):
    _fields_ = [("tilt_rad", C.c_double), ("c11", C.c_double), ("c12", C.c_double), ("c44", C.c_double),
                ("g", C.c_void_p), ("ref_idx", C.c_void_p), ("R", C.c_int)]


NORM_DET1, NORM_TRACTION_FREE = 0, 1


class hrebsd_profile(C.Structure):
    _fields_ = [("ms", C.c_double * 9), ("launches", C.c_longlong * 9), ("pixel_iters", C.c_longlong)]


PROF_CLASSES = ("demons_iter", "demons_control", "demons_aux", "preprocess", "fit_rotation", "remap", "xcf",
                "solve_F", "cnn")


class hrebsd_demons_params(C.Structure):
    _fields_ = [("levels", C.c_int), ("max_iters", C.c_int * 8), ("alpha", C.c_float),
                ("sigma_update", C.c_float), ("sigma_field", C.c_float), ("stop_tol", C.c_float),
                ("stop_window", C.c_int), ("start_level", C.c_int)]


def demons_params(levels, max_iters, alpha=1.0, sigma_update=1.0, sigma_field=1.0, stop_tol=0.0, stop_window=0,
                  start_level=-1) -> hrebsd_demons_params:
    p = hrebsd_demons_params()
    p.levels = levels
    caps = list(max_iters) if hasattr(max_iters, "__len__") else [max_iters] * levels
    for i, c in enumerate(caps):
        p.max_iters[i] = int(c)
    p.alpha, p.sigma_update, p.sigma_field = alpha, sigma_update, sigma_field
    p.stop_tol, p.stop_window, p.start_level = stop_tol, stop_window, start_level
    return p


def load(build: bool = False):
    """Load libhrebsd.so (building it first if asked or if it is stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build or not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libhrebsd.so not found at {_build.LIB}: run __graft_entry__.build()")
    lib = C.CDLL(_build.LIB)
    vp, i, ll = C.c_void_p, C.c_int, C.c_longlong
    sig = {
        "hrebsd_create": (i, [C.POINTER(vp), i]),
        "hrebsd_destroy": (i, [vp]),
        "hrebsd_status_string": (C.c_char_p, [i]),
        "hrebsd_launch_count": (ll, [vp]),
        "hrebsd_profile_enable": (i, [vp, i]),
        "hrebsd_device_error": (i, [vp]),
        "hrebsd_set_option": (i, [vp, i, i]),
        "hrebsd_profile_read": (i, [vp, C.POINTER(hrebsd_profile)]),
        "hrebsd_preprocess_batch": (i, [vp, vp, i, i, i, i, vp, vp]),
        "hrebsd_demons_register_batch": (i, [vp, vp, vp, vp, i, i, i, i, C.POINTER(hrebsd_demons_params), vp, vp,
                                             vp, vp, vp]),
        "hrebsd_demons_register_batch_noalloc": (i, [vp, vp, vp, vp, i, i, i, i, C.POINTER(hrebsd_demons_params),
                                                     vp, vp, vp, vp, vp]),
        "hrebsd_fit_rotation": (i, [vp, vp, i, i, i, vp, i, C.POINTER(hrebsd_geometry), vp, vp, vp, vp]),
        "hrebsd_remap": (i, [vp, vp, vp, vp, i, i, i, C.POINTER(hrebsd_geometry), vp, vp]),
        "hrebsd_xcf_roi_batch": (i, [vp, vp, vp, i, i, i, vp, i, i, i, vp, vp, vp, vp, vp]),
        "hrebsd_solve_F": (i, [vp, vp, vp, i, i, i, i, C.POINTER(hrebsd_geometry), vp, i, C.POINTER(hrebsd_elastic), vp,
                               vp, vp]),
        "hrebsd_downsample_batch": (i, [vp, vp, i, i, i, i, vp, vp]),
        "hrebsd_field_resample": (i, [vp, vp, i, i, i, vp, i, i, vp]),
        "hrebsd_autotune": (i, [vp, i, i, i, C.POINTER(hrebsd_demons_params), vp, vp]),
        "hrebsd_probe_fp32_fma": (i, [vp, i, C.POINTER(C.c_double), vp]),
        "hrebsd_polar_batch": (i, [vp, vp, i, vp, vp]),
        "hrebsd_tc_selftest": (i, [vp, vp, vp, i, i, vp, vp]),
        "hrebsd_wait_selftest": (i, [vp, C.c_uint, vp]),
        "hrebsd_bandpass_batch": (i, [vp, vp, i, i, i, C.c_float, C.c_float, vp, vp]),
        "hrebsd_mean_pattern": (i, [vp, vp, i, i, i, vp, vp]),
        "hrebsd_background_batch": (i, [vp, vp, i, i, i, vp, C.c_float, vp, vp]),
        "hrebsd_shift_zoom_batch": (i, [vp, vp, i, i, i, vp, vp, C.POINTER(hrebsd_geometry), vp, vp]),
        "hrebsd_fit_quality": (i, [vp, vp, vp, vp, vp, vp, i, i, i, vp, i, C.POINTER(hrebsd_geometry), vp, vp, vp]),
        "hrebsd_ssim_warped": (i, [vp, vp, vp, vp, vp, i, i, i, vp, vp]),
        "hrebsd_set_tile_variant": (i, [vp, i, i, i]),
        "hrebsd_get_tile_variant": (i, [vp, i, i]),
        "hrebsd_strain_stress": (i, [vp, vp, vp, vp, i, i, C.c_double, C.c_double, C.c_double, C.c_double, i, vp,
                                     vp, vp, vp]),
        "hrebsd_cnn_num_params": (ll, [vp]),
        "hrebsd_cnn_init": (i, [vp, vp, ll]),
        "hrebsd_cnn_get_params": (i, [vp, vp, vp]),
        "hrebsd_cnn_get_state": (i, [vp, vp, vp, C.POINTER(C.c_int)]),
        "hrebsd_cnn_set_state": (i, [vp, vp, vp, i]),
        "hrebsd_cnn_save": (i, [vp, C.c_char_p]),
        "hrebsd_gauss_taps": (i, [C.c_float, C.POINTER(C.c_float)]),
        "hrebsd_cnn_load": (i, [vp, C.c_char_p]),
        "hrebsd_cnn_infer": (i, [vp, vp, i, vp, vp]),
        "hrebsd_cnn_infer_patterns": (i, [vp, vp, vp, vp, i, i, i, vp, vp]),
        "hrebsd_cnn_train_step": (i, [vp, vp, vp, i, C.c_float, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def _p(x, dtype=None):
    """Device address of a torch CUDA tensor, an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor (the library takes device pointers)")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and x.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {x.dtype}")
    return x.data_ptr()


def _s(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _chk(st, where):
    if st != 0:
        raise HrebsdError(st, where)


def _t():
    import torch
    return torch


def hrebsd_create(device: int = 0):
    h = C.c_void_p()
    _chk(load().hrebsd_create(C.byref(h), device), "hrebsd_create")
    return h


def hrebsd_destroy(ctx):
    _chk(load().hrebsd_destroy(ctx), "hrebsd_destroy")


def hrebsd_status_string(status: int) -> str:
    return load().hrebsd_status_string(status).decode()


def hrebsd_launch_count(ctx) -> int:
    return int(load().hrebsd_launch_count(ctx))


OPT_NO_TMA = 1
OPT_GRAPHS = 2
OPT_CNN_TC = 3
OPT_TEX_GATHER = 4


def hrebsd_device_error(ctx):
    """Raise if a kernel gave up a bounded wait since the last check (synchronises)."""
    _chk(load().hrebsd_device_error(ctx), "hrebsd_device_error")


def hrebsd_set_option(ctx, option: int, value: int):
    _chk(load().hrebsd_set_option(ctx, option, int(value)), "hrebsd_set_option")


def hrebsd_profile_enable(ctx, enable: bool):
    _chk(load().hrebsd_profile_enable(ctx, int(enable)), "hrebsd_profile_enable")


def hrebsd_profile_read(ctx) -> dict:
    """Per kernel class: {'ms', 'launches'}, plus 'pixel_iters' (synchronises the device)."""
    p = hrebsd_profile()
    _chk(load().hrebsd_profile_read(ctx, C.byref(p)), "hrebsd_profile_read")
    out = {name: {"ms": p.ms[i], "launches": p.launches[i]} for i, name in enumerate(PROF_CLASSES)}
    out["pixel_iters"] = p.pixel_iters
    return out


def hrebsd_preprocess_batch(ctx, inp, n, H, W, flat, out, stream=None):
    f32 = _t().float32
    _chk(load().hrebsd_preprocess_batch(ctx, _p(inp, f32), n, H, W, int(flat), _p(out, f32), _s(stream)),
         "hrebsd_preprocess_batch")


def hrebsd_downsample_batch(ctx, inp, n, H, W, f, out, stream=None):
    f32 = _t().float32
    _chk(load().hrebsd_downsample_batch(ctx, _p(inp, f32), n, H, W, f, _p(out, f32), _s(stream)),
         "hrebsd_downsample_batch")


def hrebsd_demons_register_batch(ctx, ref, test, ref_idx, R, B, H, W, params, init_field, field, iters,
                                 pair_status, stream=None):
    t = _t()
    _chk(load().hrebsd_demons_register_batch(ctx, _p(ref, t.float32), _p(test, t.float32), _p(ref_idx, t.int32), R,
                                             B, H, W, C.byref(params), _p(init_field, t.float32),
                                             _p(field, t.float32), _p(iters, t.int32), _p(pair_status, t.int32),
                                             _s(stream)), "hrebsd_demons_register_batch")


def hrebsd_demons_register_batch_noalloc(ctx, ref, test, ref_idx, R, B, H, W, params, init_field, field, iters,
                                         pair_status, stream=None):
    """Same as hrebsd_demons_register_batch with the library's static scratch (no device allocation)."""
    t = _t()
    _chk(load().hrebsd_demons_register_batch_noalloc(ctx, _p(ref, t.float32), _p(test, t.float32),
                                                     _p(ref_idx, t.int32), R, B, H, W, C.byref(params),
                                                     _p(init_field, t.float32), _p(field, t.float32),
                                                     _p(iters, t.int32), _p(pair_status, t.int32), _s(stream)),
         "hrebsd_demons_register_batch_noalloc")


def hrebsd_fit_rotation(ctx, field, B, H, W, roi_xy, N, geom, F_first, R_finite, pair_status, stream=None):
    t = _t()
    _chk(load().hrebsd_fit_rotation(ctx, _p(field, t.float32), B, H, W, _p(roi_xy, t.int32), N, C.byref(geom),
                                    _p(F_first, t.float64), _p(R_finite, t.float64), _p(pair_status, t.int32),
                                    _s(stream)), "hrebsd_fit_rotation")


def hrebsd_remap(ctx, ref, ref_idx, R_finite, B, H, W, geom, remapped, stream=None):
    t = _t()
    _chk(load().hrebsd_remap(ctx, _p(ref, t.float32), _p(ref_idx, t.int32), _p(R_finite, t.float64), B, H, W,
                             C.byref(geom), _p(remapped, t.float32), _s(stream)), "hrebsd_remap")


def hrebsd_xcf_roi_batch(ctx, remapped, test, B, H, W, roi_xy, N, S, window, q, peak, peak_height, near_tie,
                         stream=None):
    t = _t()
    _chk(load().hrebsd_xcf_roi_batch(ctx, _p(remapped, t.float32), _p(test, t.float32), B, H, W, _p(roi_xy, t.int32),
                                     N, S, int(window), _p(q, t.float32), _p(peak, t.int32),
                                     _p(peak_height, t.float32), _p(near_tie, t.int32), _s(stream)),
         "hrebsd_xcf_roi_batch")


def hrebsd_solve_F(ctx, q, roi_xy, N, B, H, W, geom, R_finite, F, pair_status, stream=None,
                   normalization=0, elastic=None):
    """normalization: NORM_DET1 (default) or NORM_TRACTION_FREE, which needs ``elastic``
    (an hrebsd_elastic, see ``elastic_params``)."""
    t = _t()
    _chk(load().hrebsd_solve_F(ctx, _p(q, t.float32), _p(roi_xy, t.int32), N, B, H, W, C.byref(geom),
                               _p(R_finite, t.float64), int(normalization),
                               None if elastic is None else C.byref(elastic), _p(F, t.float64),
                               _p(pair_status, t.int32), _s(stream)),
         "hrebsd_solve_F")


def elastic_params(g, R, tilt_rad, stiffness=None, ref_idx=None):
    """hrebsd_elastic for the traction-free normalisation: g [R, 9] float64 CUDA orientation matrices,
    ref_idx [B] int32 CUDA or None.  The struct holds raw device addresses: keep g and ref_idx alive."""
    t = _t()
    c11, c12, c44 = NI_STIFFNESS if stiffness is None else stiffness
    return hrebsd_elastic(float(tilt_rad), float(c11), float(c12), float(c44), _p(g, t.float64),
                          _p(ref_idx, t.int32), int(R))


TILE_VARIANTS = 8
# 5: the row sweep; 6: the row sweep with a level's iterations after the first in one launch;
# 7: the whole level (at most 64 x 64) in shared memory, one launch
TILE_SHAPES = ((64, 32), (32, 32), (64, 16), (64, 32), (64, 64), ("w", "rows"), ("w", "rows"), ("h", "w"))
TILE_THREADS = (256, 256, 256, 512, 768, "w", "w", 512)
TILE_AREAS = (2048, 1024, 1024, 2048, 4096, 65536, 65536, 4096)   # outputs per work item (at most)


def hrebsd_autotune(ctx, B, H, W, params, stream=None):
    """Time every tile shape per pyramid level and keep the fastest; returns ms [levels][TILE_VARIANTS]."""
    import numpy as np
    ms = (C.c_float * (params.levels * TILE_VARIANTS))()
    _chk(load().hrebsd_autotune(ctx, B, H, W, C.byref(params), ms, _s(stream)), "hrebsd_autotune")
    return np.array(ms[:], dtype=np.float32).reshape(params.levels, TILE_VARIANTS)


def hrebsd_bandpass_batch(ctx, inp, n, H, W, sigma_lp, sigma_hp, out, stream=None):
    f32 = _t().float32
    _chk(load().hrebsd_bandpass_batch(ctx, _p(inp, f32), n, H, W, float(sigma_lp), float(sigma_hp), _p(out, f32),
                                      _s(stream)), "hrebsd_bandpass_batch")


def hrebsd_mean_pattern(ctx, inp, n, H, W, out, stream=None):
    f32 = _t().float32
    _chk(load().hrebsd_mean_pattern(ctx, _p(inp, f32), n, H, W, _p(out, f32), _s(stream)), "hrebsd_mean_pattern")


def hrebsd_background_batch(ctx, inp, n, H, W, static_bg, sigma_dyn, out, stream=None):
    f32 = _t().float32
    _chk(load().hrebsd_background_batch(ctx, _p(inp, f32), n, H, W, _p(static_bg, f32), float(sigma_dyn),
                                        _p(out, f32), _s(stream)), "hrebsd_background_batch")


def hrebsd_shift_zoom_batch(ctx, inp, n, H, W, shift, zoom, geom, out, stream=None):
    f32 = _t().float32
    _chk(load().hrebsd_shift_zoom_batch(ctx, _p(inp, f32), n, H, W, _p(shift, f32), _p(zoom, f32), C.byref(geom),
                                        _p(out, f32), _s(stream)), "hrebsd_shift_zoom_batch")


def hrebsd_tc_selftest(ctx, A, B, N, KS, D, stream=None):
    t = _t()
    _chk(load().hrebsd_tc_selftest(ctx, _p(A, t.bfloat16), _p(B, t.bfloat16), N, KS, _p(D, t.float32), _s(stream)),
         "hrebsd_tc_selftest")


def hrebsd_wait_selftest(ctx, max_polls, stream=None):
    _chk(load().hrebsd_wait_selftest(ctx, int(max_polls), _s(stream)), "hrebsd_wait_selftest")


def hrebsd_polar_batch(ctx, F, B, R, stream=None):
    t = _t()
    _chk(load().hrebsd_polar_batch(ctx, _p(F, t.float64), B, _p(R, t.float64), _s(stream)), "hrebsd_polar_batch")


def hrebsd_fit_quality(ctx, F, R, q, field, ph, B, H, W, roi_xy, N, geom, mae, ph_mean=None, stream=None):
    t = _t()
    _chk(load().hrebsd_fit_quality(ctx, _p(F, t.float64), _p(R, t.float64), _p(q, t.float32), _p(field, t.float32),
                                   _p(ph, t.float32), B, H, W, _p(roi_xy, t.int32), N, C.byref(geom),
                                   _p(mae, t.float64), _p(ph_mean, t.float64), _s(stream)), "hrebsd_fit_quality")


def hrebsd_ssim_warped(ctx, ref, ref_idx, test, field, B, H, W, ssim, stream=None):
    t = _t()
    _chk(load().hrebsd_ssim_warped(ctx, _p(ref, t.float32), _p(ref_idx, t.int32), _p(test, t.float32),
                                   _p(field, t.float32), B, H, W, _p(ssim, t.float64), _s(stream)),
         "hrebsd_ssim_warped")


def hrebsd_probe_fp32_fma(ctx, iters, stream=None):
    """Launch the FP32 FMA probe; returns the floating-point operations of the launch."""
    f = C.c_double()
    _chk(load().hrebsd_probe_fp32_fma(ctx, iters, C.byref(f), _s(stream)), "hrebsd_probe_fp32_fma")
    return f.value


def hrebsd_set_tile_variant(ctx, h, w, variant):
    _chk(load().hrebsd_set_tile_variant(ctx, h, w, variant), "hrebsd_set_tile_variant")


def hrebsd_get_tile_variant(ctx, h, w):
    v = load().hrebsd_get_tile_variant(ctx, h, w)
    if v < 0:
        _chk(v, "hrebsd_get_tile_variant")
    return v


def hrebsd_field_resample(ctx, field, B, h, w, out, h2, w2, stream=None):
    t = _t()
    _chk(load().hrebsd_field_resample(ctx, _p(field, t.float32), B, h, w, _p(out, t.float32), h2, w2, _s(stream)),
         "hrebsd_field_resample")


NI_STIFFNESS = (276e9, 159e9, 132e9)


def hrebsd_strain_stress(ctx, F, ref_idx, g, R, B, tilt_rad, stiffness=NI_STIFFNESS, traction_free=True, F_S=None,
                         eps=None, sigma=None, stream=None):
    t = _t()
    c11, c12, c44 = stiffness
    _chk(load().hrebsd_strain_stress(ctx, _p(F, t.float64), _p(ref_idx, t.int32), _p(g, t.float64), R, B,
                                     float(tilt_rad), c11, c12, c44, int(traction_free), _p(F_S, t.float64),
                                     _p(eps, t.float64), _p(sigma, t.float64), _s(stream)), "hrebsd_strain_stress")


# ------------------------------------------------------------------ learned initialiser
def hrebsd_cnn_num_params(ctx) -> int:
    n = int(load().hrebsd_cnn_num_params(ctx))
    if n < 0:
        raise HrebsdError(-2, "hrebsd_cnn_num_params")
    return n


def hrebsd_cnn_init(ctx, params=None):
    """params: host float32 numpy vector in the library's layout (None keeps the current ones)."""
    import numpy as np
    if params is None:
        _chk(load().hrebsd_cnn_init(ctx, None, 0), "hrebsd_cnn_init")
        return
    a = np.ascontiguousarray(params, dtype=np.float32)
    _chk(load().hrebsd_cnn_init(ctx, a.ctypes.data, a.size), "hrebsd_cnn_init")


def hrebsd_cnn_get_params(ctx):
    """(params, grads of the last training step) as float32 numpy vectors."""
    import numpy as np
    n = hrebsd_cnn_num_params(ctx)
    p, g = np.empty(n, np.float32), np.empty(n, np.float32)
    _chk(load().hrebsd_cnn_get_params(ctx, p.ctypes.data, g.ctypes.data), "hrebsd_cnn_get_params")
    return p, g


def hrebsd_cnn_get_state(ctx):
    """(Adam first moment, second moment, step) of the network in the context."""
    import numpy as np
    n = hrebsd_cnn_num_params(ctx)
    m, v, step = np.empty(n, np.float32), np.empty(n, np.float32), C.c_int(0)
    _chk(load().hrebsd_cnn_get_state(ctx, m.ctypes.data, v.ctypes.data, C.byref(step)), "hrebsd_cnn_get_state")
    return m, v, step.value


def hrebsd_cnn_set_state(ctx, m, v, step):
    import numpy as np
    n = hrebsd_cnn_num_params(ctx)
    m, v = np.ascontiguousarray(m, np.float32), np.ascontiguousarray(v, np.float32)
    if m.size != n or v.size != n:
        raise ValueError(f"Adam moments need {n} entries each")
    _chk(load().hrebsd_cnn_set_state(ctx, m.ctypes.data, v.ctypes.data, int(step)), "hrebsd_cnn_set_state")


def hrebsd_gauss_taps(sigma):
    """FP32 taps of the registration's Gaussian (numpy float32 [2r + 1]); host only."""
    import numpy as np
    buf = (C.c_float * 13)()
    r = load().hrebsd_gauss_taps(float(sigma), buf)
    _chk(min(r, 0), "hrebsd_gauss_taps")
    return np.array(buf[: 2 * r + 1], dtype=np.float32)


def hrebsd_cnn_save(ctx, path):
    """Write the network's weights, Adam moments and step to ``path`` (the library's model file)."""
    _chk(load().hrebsd_cnn_save(ctx, os.fsencode(path)), "hrebsd_cnn_save")


def hrebsd_cnn_load(ctx, path):
    """Replace the network state of the context by the model file at ``path``."""
    _chk(load().hrebsd_cnn_load(ctx, os.fsencode(path)), "hrebsd_cnn_load")


def hrebsd_cnn_infer(ctx, x_bf16, B, field64, stream=None):
    t = _t()
    _chk(load().hrebsd_cnn_infer(ctx, _p(x_bf16, t.bfloat16), B, _p(field64, t.float32), _s(stream)),
         "hrebsd_cnn_infer")


def hrebsd_cnn_infer_patterns(ctx, ref, test, ref_idx, B, H, W, field64, stream=None):
    t = _t()
    _chk(load().hrebsd_cnn_infer_patterns(ctx, _p(ref, t.float32), _p(test, t.float32), _p(ref_idx, t.int32), B, H, W,
                                          _p(field64, t.float32), _s(stream)), "hrebsd_cnn_infer_patterns")


def hrebsd_cnn_train_step(ctx, x_bf16, target, B, lr, loss_out=None, stream=None):
    t = _t()
    _chk(load().hrebsd_cnn_train_step(ctx, _p(x_bf16, t.bfloat16), _p(target, t.float32), B, float(lr),
                                      _p(loss_out, t.float32), _s(stream)), "hrebsd_cnn_train_step")
