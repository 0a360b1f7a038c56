"""Resumable scans: a long scan runs in chunks of consecutive points, and each chunk's results
are written to their own file as soon as the chunk is done (temporary name, then an atomic
rename).  A run that stops part way (a crash, a killed job, a lost node) is resumed by calling
the same function again: chunks whose file exists are skipped, the rest are computed, and the
result is assembled from the files.  A manifest pins the scan's size and chunking, so that a
directory of another scan is never mixed in."""
from __future__ import annotations

import json
import os

import numpy as np


def chunk_path(out_dir: str, k: int) -> str:
    return os.path.join(out_dir, f"chunk_{k:06d}.npz")


def _write_atomic_npz(path: str, arrays: dict):
    tmp = path + ".tmp.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def run_resumable(n_items: int, chunk: int, out_dir: str, process, tag: str = ""):
    """Process items [0, n_items) in chunks of ``chunk``.  ``process(a, b)`` returns a dict of numpy
    arrays whose first dimension is b - a.  Returns (results assembled over all items, indices of
    the chunks computed by this call)."""
    if n_items < 1 or chunk < 1:
        raise ValueError("n_items and chunk must be positive")
    os.makedirs(out_dir, exist_ok=True)
    manifest = {"n_items": int(n_items), "chunk": int(chunk), "tag": str(tag)}
    mpath = os.path.join(out_dir, "manifest.json")
    if os.path.exists(mpath):
        with open(mpath) as f:
            if json.load(f) != manifest:
                raise ValueError(f"{out_dir} holds another scan (manifest differs from {manifest})")
    else:
        tmp = mpath + ".tmp"
        with open(tmp, "w") as f:
            json.dump(manifest, f)
        os.replace(tmp, mpath)
    nk = -(-n_items // chunk)
    computed = []
    for k in range(nk):
        path = chunk_path(out_dir, k)
        if os.path.exists(path):
            continue
        a, b = k * chunk, min(n_items, (k + 1) * chunk)
        res = process(a, b)
        for name, arr in res.items():
            if np.shape(arr)[0] != b - a:
                raise ValueError(f"chunk {k}: '{name}' has {np.shape(arr)[0]} rows, expected {b - a}")
        _write_atomic_npz(path, {n: np.asarray(v) for n, v in res.items()})
        computed.append(k)
    parts = []
    for k in range(nk):
        with np.load(chunk_path(out_dir, k)) as z:
            parts.append({n: z[n] for n in z.files})
    out = {n: np.concatenate([p[n] for p in parts]) for n in parts[0]}
    return out, computed
