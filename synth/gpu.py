"""GPU twin of the seeded Kikuchi generator (input generation for large batches).

Per pattern the host computes the 25 deformed plane normals, Bragg angles and
amplitudes exactly as ``synth.kikuchi.render`` does; the kernel in
``csrc/kikuchi_gen.cu`` evaluates the bands, background, scaling and noise
per pixel.  Results agree with the numpy generator to FP32 rounding (noisy
patterns: to +-1 count at a small fraction of pixels).
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np

from . import kikuchi as K

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "kikuchi_gen.cu")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc, "-O3", "-shared", "-Xcompiler", "-fPIC", "-gencode",
                               "arch=compute_103a,code=sm_103a", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp, i, f = C.c_void_p, C.c_int, C.c_float
        lib.synth_kikuchi.restype = i
        lib.synth_kikuchi.argtypes = [vp, vp, i, i, i, f, f, f, f, i, i, vp, vp]
        _lib = lib
    return _lib


def plane_table(g: np.ndarray, F: np.ndarray) -> np.ndarray:
    """[25, 5] float32: unit normal (3), Bragg angle, amplitude of each band."""
    hkl = K.fcc_planes()
    G = (g @ (hkl / K.LATTICE_A).T).T
    G = (np.linalg.inv(F).T @ G.T).T
    gn = np.linalg.norm(G, axis=1)
    lam = K.electron_wavelength_angstrom(K.KV)
    out = np.empty((len(hkl), 5))
    out[:, :3] = G / gn[:, None]
    out[:, 3] = np.arcsin(lam * gn / 2.0)
    out[:, 4] = 3.0 / np.sum(hkl * hkl, axis=1)
    return out.astype(np.float32)


def render_batch(gs, Fs, keys, H, W, geom: K.Geometry, counts: float, noise=True, background=True, out=None,
                 stream=None):
    """Render len(gs) patterns on the current CUDA device into a float32 tensor [n, H, W]."""
    import torch
    n = len(gs)
    planes = np.stack([plane_table(g, F) for g, F in zip(gs, Fs)]) if n else np.zeros((0, 25, 5), np.float32)
    pl = torch.from_numpy(np.ascontiguousarray(planes)).cuda()
    ks = torch.from_numpy(np.asarray(keys, dtype=np.uint64).view(np.int64)).cuda()
    if out is None:
        out = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    rc = _load().synth_kikuchi(pl.data_ptr(), ks.data_ptr(), n, H, W, geom.xstar * W, geom.ystar * H, geom.zstar * W,
                               counts, int(noise), int(background), out.data_ptr(), st)
    if rc:
        raise RuntimeError("synth_kikuchi launch failed")
    return out


def make_scan_gpu(spec: K.ScanSpec, pairs=None, noise=True, chunk=4096):
    """GPU counterpart of kikuchi.make_scan: (refs, tests, ref_idx, F_true) as CUDA tensors / numpy truth."""
    import torch
    pairs = list(range(spec.n_pairs)) if pairs is None else list(pairs)
    g_refs = [K.ref_orientation(spec, r) for r in range(spec.n_refs)]
    ref_keys = [int(K.stream_key(spec.seed, 16 * (1_000_000 + r) + K.P_NOISE)) for r in range(spec.n_refs)]
    refs = render_batch(g_refs, [np.eye(3)] * spec.n_refs, ref_keys, spec.H, spec.W, spec.geom, spec.counts, noise)
    ridx = np.array([K.ref_index(spec, p) for p in pairs], dtype=np.int32)
    Ft = np.stack([K.pair_truth(spec, p) for p in pairs]) if pairs else np.zeros((0, 3, 3))
    tests = torch.empty((len(pairs), spec.H, spec.W), dtype=torch.float32, device="cuda")
    for c0 in range(0, len(pairs), chunk):
        sl = slice(c0, min(len(pairs), c0 + chunk))
        ps = pairs[sl]
        keys = [int(K.stream_key(spec.seed, 16 * p + K.P_NOISE)) for p in ps]
        render_batch([g_refs[r] for r in ridx[sl]], Ft[sl], keys, spec.H, spec.W, spec.geom, spec.counts, noise,
                     out=tests[sl])
    return refs, tests, torch.from_numpy(ridx).cuda(), Ft
