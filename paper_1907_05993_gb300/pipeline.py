"""The whole hot path for a batch of pattern pairs, chained through the C ABI.

``Pipeline.run`` calls, in order: hrebsd_autotune (first batch of a size
only), hrebsd_preprocess_batch (references and tests), hrebsd_demons_register_batch, hrebsd_fit_rotation, hrebsd_remap,
hrebsd_xcf_roi_batch and hrebsd_solve_F, all on one stream.  This module
only allocates the output tensors and passes pointers; every step runs in
the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import (demons_params, hrebsd_autotune, hrebsd_cnn_infer_patterns, hrebsd_create, hrebsd_demons_register_batch, hrebsd_destroy,
               hrebsd_fit_rotation, hrebsd_geometry, hrebsd_preprocess_batch, hrebsd_remap, hrebsd_solve_F,
               hrebsd_field_resample, hrebsd_strain_stress, hrebsd_xcf_roi_batch, NI_STIFFNESS)


@dataclass
class PipelineConfig:
    H: int
    W: int
    roi_xy: np.ndarray          # int32 [N, 2] ROI centres (continuous pixels)
    S: int                      # ROI size of the second pass
    levels: int
    max_iters: tuple
    alpha: float = 1.0
    sigma: float = 1.0
    stop_tol: float = 0.0
    stop_window: int = 0
    xstar: float = 0.5
    ystar: float = 0.5
    zstar: float = 0.6
    flat: bool = True
    window: bool = True
    autotune: bool = True       # pick the demons tile shape per level on the first batch of a size


class Pipeline:
    def __init__(self, cfg: PipelineConfig, device: int = 0):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.dev = torch.device("cuda", device)
        self.ctx = hrebsd_create(device)
        self.geom = hrebsd_geometry(cfg.xstar, cfg.ystar, cfg.zstar)
        self.params = demons_params(cfg.levels, cfg.max_iters, cfg.alpha, cfg.sigma, cfg.sigma, cfg.stop_tol,
                                    cfg.stop_window)
        self.roi = torch.as_tensor(np.ascontiguousarray(cfg.roi_xy, dtype=np.int32), device=self.dev)
        self.N = int(cfg.roi_xy.shape[0])
        self._bufs = {}
        self._tuned = {}

    def close(self):
        if self.ctx is not None:
            hrebsd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _buf(self, name, shape, dtype):
        t = self._bufs.get(name)
        if t is None or tuple(t.shape) != tuple(shape) or t.dtype != dtype:
            t = self.torch.empty(shape, dtype=dtype, device=self.dev)
            self._bufs[name] = t
        return t

    def preprocess(self, raw, out=None, stream=None):
        n, H, W = raw.shape
        out = self._buf(f"pre{n}", (n, H, W), self.torch.float32) if out is None else out
        hrebsd_preprocess_batch(self.ctx, raw, n, H, W, self.cfg.flat, out, stream)
        return out

    def run(self, refs_raw, tests_raw, ref_idx, stream=None, init_field=None, start_level=-1, out=None,
            learned_caps=None, learned_start_res=128):
        """refs_raw [R,H,W], tests_raw [B,H,W] float32 CUDA; ref_idx [B] int32 CUDA.

        learned_caps (per level, finest first): start the registration at the level of
        learned_start_res x learned_start_res pixels from the learned initialiser's 64x64
        field (hrebsd_cnn_infer_patterns, resampled by hrebsd_field_resample; the network
        must be loaded in this pipeline's context) with these iteration caps."""
        t = self.torch
        c = self.cfg
        R, B = refs_raw.shape[0], tests_raw.shape[0]
        H, W, N, L = c.H, c.W, self.N, c.levels
        o = {} if out is None else out

        def get(name, shape, dtype):
            if name not in o:
                o[name] = self._buf(name, shape, dtype)
            return o[name]
        ref_p = get("ref_pre", (R, H, W), t.float32)
        test_p = get("test_pre", (B, H, W), t.float32)
        if c.autotune and (B, H, W) not in self._tuned:
            self._tuned[(B, H, W)] = hrebsd_autotune(self.ctx, B, H, W, self.params, stream)
        hrebsd_preprocess_batch(self.ctx, refs_raw, R, H, W, c.flat, ref_p, stream)
        hrebsd_preprocess_batch(self.ctx, tests_raw, B, H, W, c.flat, test_p, stream)
        field = get("field", (B, 2, H, W), t.float32)
        iters = get("iters", (B, L), t.int32)
        status = get("status", (B,), t.int32)
        params = self.params
        params.start_level = start_level
        if learned_caps is not None:
            r = learned_start_res
            lvl = int(round(np.log2(H / r)))
            net = get("field64", (B, 2, 64, 64), t.float32)
            hrebsd_cnn_infer_patterns(self.ctx, ref_p, test_p, ref_idx, B, H, W, net, stream)
            if r == 64:
                init_field = net
            else:
                init_field = get(f"field_init{r}", (B, 2, r, r), t.float32)
                hrebsd_field_resample(self.ctx, net, B, 64, 64, init_field, r, r, stream)
            params = demons_params(c.levels, learned_caps, c.alpha, c.sigma, c.sigma, c.stop_tol, c.stop_window, lvl)
        hrebsd_demons_register_batch(self.ctx, ref_p, test_p, ref_idx, R, B, H, W, params, init_field, field,
                                     iters, status, stream)
        F1 = get("F_first", (B, 9), t.float64)
        Rf = get("R_finite", (B, 9), t.float64)
        hrebsd_fit_rotation(self.ctx, field, B, H, W, self.roi, N, self.geom, F1, Rf, status, stream)
        rem = get("remapped", (B, H, W), t.float32)
        hrebsd_remap(self.ctx, ref_p, ref_idx, Rf, B, H, W, self.geom, rem, stream)
        q = get("q", (B, N, 2), t.float32)
        peak = get("peak", (B, N, 2), t.int32)
        ph = get("ph", (B, N), t.float32)
        tie = get("near_tie", (B, N), t.int32)
        hrebsd_xcf_roi_batch(self.ctx, rem, test_p, B, H, W, self.roi, N, c.S, c.window, q, peak, ph, tie, stream)
        F = get("F", (B, 9), t.float64)
        hrebsd_solve_F(self.ctx, q, self.roi, N, B, H, W, self.geom, Rf, F, status, stream)
        return o

    def strain_stress(self, out, g, ref_idx, tilt_rad, stiffness=NI_STIFFNESS, traction_free=True, stream=None):
        """Post-processing of Eq. 13-16 on the F of ``run``: adds F_S, eps, sigma [B, 9] (FP64) to ``out``.

        g: [R, 9] float64 CUDA passive orientation matrices of the references."""
        t = self.torch
        F = out["F"]
        B = F.shape[0]
        for name in ("F_S", "eps", "sigma"):
            if name not in out:
                out[name] = self._buf(name, (B, 9), t.float64)
        hrebsd_strain_stress(self.ctx, F, ref_idx, g, g.shape[0], B, tilt_rad, stiffness, traction_free, out["F_S"],
                             out["eps"], out["sigma"], stream)
        return out
