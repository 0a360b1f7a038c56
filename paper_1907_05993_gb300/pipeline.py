"""The whole hot path for a batch of pattern pairs, chained through the C ABI.

``Pipeline.run`` calls, in order: hrebsd_autotune (first batch of a size
only), hrebsd_preprocess_batch (references and tests), hrebsd_demons_register_batch, hrebsd_fit_rotation, hrebsd_remap,
hrebsd_xcf_roi_batch and hrebsd_solve_F, all on one stream.  ``Pipeline.run_host``
takes pinned host inputs and overlaps their copy with the processing, slice
by slice.  This module only allocates the output tensors and passes
pointers; every step runs in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import (demons_params, hrebsd_autotune, hrebsd_background_batch, hrebsd_bandpass_batch, hrebsd_mean_pattern, hrebsd_cnn_infer_patterns, hrebsd_fit_quality, hrebsd_polar_batch,
               hrebsd_ssim_warped, hrebsd_create, hrebsd_demons_register_batch, hrebsd_destroy,
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
    # preprocessing for real scans (Section 3.2-3.3), off by default: static background = the
    # batch's mean test pattern, dynamic background blur sigma, band-pass (sigma_lp, sigma_hp)
    static_background: bool = False
    dynamic_background: float = 0.0
    bandpass: tuple = (0.0, 0.0)


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
        self._copy_stream = None
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
        src_r, src_t = refs_raw, tests_raw
        if c.static_background or c.dynamic_background > 0 or c.bandpass[0] > 0 or c.bandpass[1] > 0:
            src_r, src_t = get("ref_filtered", (R, H, W), t.float32), get("test_filtered", (B, H, W), t.float32)
            bg = None
            if c.static_background:
                bg = get("static_background", (H, W), t.float32)
                hrebsd_mean_pattern(self.ctx, tests_raw, B, H, W, bg, stream)
            hrebsd_background_batch(self.ctx, refs_raw, R, H, W, bg, c.dynamic_background, src_r, stream)
            hrebsd_background_batch(self.ctx, tests_raw, B, H, W, bg, c.dynamic_background, src_t, stream)
            if c.bandpass[0] > 0 or c.bandpass[1] > 0:
                hrebsd_bandpass_batch(self.ctx, src_r, R, H, W, c.bandpass[0], c.bandpass[1], src_r, stream)
                hrebsd_bandpass_batch(self.ctx, src_t, B, H, W, c.bandpass[0], c.bandpass[1], src_t, stream)
        hrebsd_preprocess_batch(self.ctx, src_r, R, H, W, c.flat, ref_p, stream)
        hrebsd_preprocess_batch(self.ctx, src_t, B, H, W, c.flat, test_p, stream)
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

    @staticmethod
    def slice_bounds(B: int, chunks: int, growth: float = 2.0):
        """Boundaries of ``chunks`` consecutive slices of B items whose sizes grow by ``growth``
        (1 : 2 : 4 ... by default): the first slice, whose copy nothing hides, is small, and each
        later copy runs while the (smaller) slice before it is processed.  Every slice has at
        least one item; returns [0, b1, ..., B]."""
        k = max(1, min(int(chunks), B))
        w = [growth ** i for i in range(k)]
        cuts = [0]
        for i in range(1, k):
            c = int(round(B * sum(w[:i]) / sum(w)))
            cuts.append(min(max(c, cuts[-1] + 1), B - (k - i)))
        cuts.append(B)
        return cuts

    def run_host(self, refs_host, tests_host, ref_idx_host, chunks=2, out=None, growth=4.0):
        """Host-resident inputs: refs [R,H,W] and tests [B,H,W] float32, ref_idx [B] int32, in pinned CPU
        memory.  The batch runs through ``run`` as ``chunks`` consecutive slices (sizes growing by
        ``growth``, see slice_bounds) on the current stream; the host -> device copy of slice k + 1 runs
        on a side stream while slice k is processed, and F, R_finite (FP64 [B, 9]) and status ([B]) of
        every slice are copied into pinned host tensors, returned in a dict (valid once the current
        stream has synchronised).  Each pair's result is the one ``run`` gives on the whole batch (pairs
        are independent); the static background, a statistic of the whole batch, needs chunks=1.
        Two slices of 1 : 4 by default: every slice is a registration of its own, whose last iterations
        (the pairs that run to the cap) leave CTAs idle once fewer pairs remain than CTAs, so more,
        smaller slices lose more there than they hide of the copy (10,000 pairs of 256x256 on GB300 at
        211 GB/s host to device: 4 slices 1:2:4:8 418 ms, 2 slices 1:4 388 ms, device-resident 373 ms)."""
        t = self.torch
        if self.cfg.static_background and chunks > 1:
            raise ValueError("the static background is a whole-batch statistic: use chunks=1")
        B, H, W = tests_host.shape
        R = refs_host.shape[0]
        cuts = self.slice_bounds(B, chunks, growth)
        nk = len(cuts) - 1
        n = max(cuts[i + 1] - cuts[i] for i in range(nk))
        cs = t.cuda.current_stream(self.dev)
        if self._copy_stream is None:
            self._copy_stream = t.cuda.Stream(self.dev)
        xs = self._copy_stream
        d_refs = self._buf("host_refs", (R, H, W), t.float32)
        d_refs.copy_(refs_host, non_blocking=True)
        slots = [(self._buf(f"host_tests{k}", (n, H, W), t.float32), self._buf(f"host_idx{k}", (n,), t.int32))
                 for k in range(2)]
        o = {} if out is None else out
        for name, shape, dtype in (("F", (B, 9), t.float64), ("R_finite", (B, 9), t.float64),
                                   ("status", (B,), t.int32)):
            if name not in o or tuple(o[name].shape) != shape or o[name].is_cuda:
                o[name] = t.empty(shape, dtype=dtype).pin_memory()
        copied = [t.cuda.Event(), t.cuda.Event()]
        freed = [None, None]

        def issue_copy(k):
            sl, a, b = k % 2, cuts[k], cuts[k + 1]
            with t.cuda.stream(xs):
                if freed[sl] is not None:   # the slice two back is done with this staging slot
                    xs.wait_event(freed[sl])
                slots[sl][0][: b - a].copy_(tests_host[a:b], non_blocking=True)
                slots[sl][1][: b - a].copy_(ref_idx_host[a:b], non_blocking=True)
                copied[sl].record(xs)

        issue_copy(0)
        for k in range(nk):
            sl, a, b = k % 2, cuts[k], cuts[k + 1]
            if k + 1 < nk:
                issue_copy(k + 1)
            cs.wait_event(copied[sl])
            r = self.run(d_refs, slots[sl][0][: b - a], slots[sl][1][: b - a])
            ev = t.cuda.Event()
            ev.record(cs)
            freed[sl] = ev
            for name in ("F", "R_finite", "status"):
                o[name][a:b].copy_(r[name], non_blocking=True)
        return o

    def run_scan(self, refs_host, tests_host, ref_idx_host, out_dir, chunk=10_000, slices=2):
        """A whole scan from pinned host inputs, resumable: chunks of ``chunk`` points go through
        ``run_host`` (``slices`` overlapped slices each) and F, R_finite and status of every chunk are
        written to ``out_dir`` (see scan.run_resumable); calling it again after an interruption
        computes only the missing chunks.  Returns (results as numpy arrays, chunks computed now)."""
        from .scan import run_resumable
        t = self.torch
        cs = t.cuda.current_stream(self.dev)

        def process(a, b):
            o = self.run_host(refs_host, tests_host[a:b], ref_idx_host[a:b], chunks=slices)
            cs.synchronize()
            return {k: o[k].numpy().copy() for k in ("F", "R_finite", "status")}

        tag = f"{tuple(tests_host.shape)} levels={self.cfg.levels} caps={tuple(self.cfg.max_iters)}"
        return run_resumable(int(tests_host.shape[0]), int(chunk), out_dir, process, tag)

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

    def compare(self, refs_raw, tests_raw, ref_idx, stream=None, out=None):
        """The four rotation measurements of Fig. 2 and the quality measures of Fig. 3 (Section 3.1).

        Runs the method of the paper (d) through ``run`` and adds: (a) XCF without remapping
        (the per-pair reference obtained by hrebsd_remap with identity rotations), (b) the demons
        fit alone (F_first), (c) remapping by polar((a)) then the second pass.  Per method m in
        a, b, c, d: F_m [B, 9], mae_m [B] (rad); ph_a, ph_c, ph_d [B]; ssim_b [B] of the warped
        reference and ssim_none [B] without warp.  Every step is a library call."""
        t = self.torch
        c = self.cfg
        o = self.run(refs_raw, tests_raw, ref_idx, stream=stream, out=out)
        B, H, W, N = tests_raw.shape[0], c.H, c.W, self.N

        def get(name, shape, dtype):
            if name not in o:
                o[name] = self._buf(name, shape, dtype)
            return o[name]
        eye = get("R_identity", (B, 9), t.float64)
        eye.copy_(t.eye(3, dtype=t.float64, device=self.dev).reshape(1, 9).expand(B, 9))
        ref_i = get("ref_per_pair", (B, H, W), t.float32)
        hrebsd_remap(self.ctx, o["ref_pre"], ref_idx, eye, B, H, W, self.geom, ref_i, stream)
        q_a, pk_a = get("q_a", (B, N, 2), t.float32), get("peak_a", (B, N, 2), t.int32)
        ph_a, tie_a = get("ph_a", (B, N), t.float32), get("near_tie_a", (B, N), t.int32)
        hrebsd_xcf_roi_batch(self.ctx, ref_i, o["test_pre"], B, H, W, self.roi, N, c.S, c.window, q_a, pk_a, ph_a,
                             tie_a, stream)
        st_a = get("status_a", (B,), t.int32)
        st_a.zero_()
        F_a = get("F_a", (B, 9), t.float64)
        hrebsd_solve_F(self.ctx, q_a, self.roi, N, B, H, W, self.geom, None, F_a, st_a, stream)
        R_a = get("R_a", (B, 9), t.float64)
        hrebsd_polar_batch(self.ctx, F_a, B, R_a, stream)
        rem_c = get("remapped_c", (B, H, W), t.float32)
        hrebsd_remap(self.ctx, o["ref_pre"], ref_idx, R_a, B, H, W, self.geom, rem_c, stream)
        q_c, pk_c = get("q_c", (B, N, 2), t.float32), get("peak_c", (B, N, 2), t.int32)
        ph_c, tie_c = get("ph_c", (B, N), t.float32), get("near_tie_c", (B, N), t.int32)
        hrebsd_xcf_roi_batch(self.ctx, rem_c, o["test_pre"], B, H, W, self.roi, N, c.S, c.window, q_c, pk_c, ph_c,
                             tie_c, stream)
        F_c = get("F_c", (B, 9), t.float64)
        hrebsd_solve_F(self.ctx, q_c, self.roi, N, B, H, W, self.geom, R_a, F_c, st_a, stream)
        o["F_b"], o["F_d"] = o["F_first"], o["F"]
        for m, F, R, q, field, ph in (("a", F_a, None, q_a, None, ph_a), ("b", o["F_first"], None, None, o["field"], None),
                                      ("c", F_c, R_a, q_c, None, ph_c), ("d", o["F"], o["R_finite"], o["q"], None, o["ph"])):
            mae = get(f"mae_{m}", (B,), t.float64)
            phm = get(f"phm_{m}", (B,), t.float64) if ph is not None else None
            hrebsd_fit_quality(self.ctx, F, R, q, field, ph, B, H, W, self.roi, N, self.geom, mae, phm, stream)
        for name, field in (("ssim_b", o["field"]), ("ssim_none", None)):
            hrebsd_ssim_warped(self.ctx, o["ref_pre"], ref_idx, o["test_pre"], field, B, H, W,
                               get(name, (B,), t.float64), stream)
        return o
