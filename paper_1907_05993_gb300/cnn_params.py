"""Parameter vector of the learned initialiser <-> per-layer arrays.

The library keeps each 3x3 layer as weights [cout][ky*3+kx][cin padded to 16]
followed by the bias, in the order e1a e1b e2a e2b e3a e3b ba bb d3a d3b d2a
d2b d1a d1b, then the 1x1 head [2][16] and its bias.  These helpers only
reorder numbers (no arithmetic of the network).
"""
from __future__ import annotations

import numpy as np

LAYERS = [("e1a", 2, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32), ("e3a", 32, 64), ("e3b", 64, 64),
          ("ba", 64, 128), ("bb", 128, 128), ("d3a", 192, 64), ("d3b", 64, 64), ("d2a", 96, 32), ("d2b", 32, 32),
          ("d1a", 48, 16), ("d1b", 16, 16)]


def _pad16(c):
    return (c + 15) // 16 * 16


def num_params() -> int:
    return sum(co * 9 * _pad16(ci) + co for _, ci, co in LAYERS) + 2 * 16 + 2


def pack(p: dict) -> np.ndarray:
    """{name.w [co, ci, 3, 3], name.b [co], head.w [2, 16, 1, 1], head.b [2]} -> flat float32 vector."""
    out = []
    for name, ci, co in LAYERS:
        w = np.zeros((co, 9, _pad16(ci)))
        w[:, :, :ci] = np.asarray(p[name + ".w"]).reshape(co, ci, 9).transpose(0, 2, 1)
        out += [w.ravel(), np.asarray(p[name + ".b"]).ravel()]
    out += [np.asarray(p["head.w"]).reshape(2, 16).ravel(), np.asarray(p["head.b"]).ravel()]
    return np.concatenate(out).astype(np.float32)


def unpack(v: np.ndarray) -> dict:
    v = np.asarray(v, dtype=np.float64)
    p, o = {}, 0
    for name, ci, co in LAYERS:
        n = co * 9 * _pad16(ci)
        w = v[o:o + n].reshape(co, 9, _pad16(ci))[:, :, :ci]
        p[name + ".w"] = w.transpose(0, 2, 1).reshape(co, ci, 3, 3)
        o += n
        p[name + ".b"] = v[o:o + co].copy()
        o += co
    p["head.w"] = v[o:o + 32].reshape(2, 16, 1, 1)
    o += 32
    p["head.b"] = v[o:o + 2].copy()
    return p
