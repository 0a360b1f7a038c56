"""Checkpoint/resume of a long scan (host logic, CPU): chunks written atomically, an interrupted
run resumed without recomputing finished chunks, another scan's directory refused."""
import os

import numpy as np
import pytest

from paper_1907_05993_gb300 import scan


def _process_factory(calls, fail_at=None):
    def process(a, b):
        k = a // 3
        if fail_at is not None and k == fail_at:
            raise RuntimeError("node lost")
        calls.append(k)
        idx = np.arange(a, b)
        return {"F": np.stack([idx * 1.0] * 9, axis=1), "status": (idx % 4).astype(np.int32)}
    return process


def test_resume_after_interruption(tmp_path):
    d = str(tmp_path / "scan")
    ref, _ = scan.run_resumable(11, 3, str(tmp_path / "ref"), _process_factory([]))
    calls = []
    with pytest.raises(RuntimeError):
        scan.run_resumable(11, 3, d, _process_factory(calls, fail_at=2))
    assert calls == [0, 1] and sorted(os.listdir(d)) == ["chunk_000000.npz", "chunk_000001.npz", "manifest.json"]
    # a write that died half way leaves only a temporary file, which is not taken as done
    open(scan.chunk_path(d, 2) + ".tmp.npz", "wb").write(b"partial")
    calls2 = []
    out, computed = scan.run_resumable(11, 3, d, _process_factory(calls2))
    assert computed == [2, 3] and calls2 == [2, 3]
    for k in ref:
        assert np.array_equal(out[k], ref[k])
    assert out["F"].shape == (11, 9) and np.array_equal(out["F"][:, 0], np.arange(11.0))
    # a finished scan: nothing recomputed
    out2, computed2 = scan.run_resumable(11, 3, d, _process_factory([]))
    assert computed2 == [] and np.array_equal(out2["status"], ref["status"])


def test_other_scan_refused_and_shapes_checked(tmp_path):
    d = str(tmp_path / "scan")
    scan.run_resumable(6, 3, d, _process_factory([]))
    with pytest.raises(ValueError):
        scan.run_resumable(6, 2, d, _process_factory([]))      # other chunking
    with pytest.raises(ValueError):
        scan.run_resumable(7, 3, d, _process_factory([]))      # other size
    with pytest.raises(ValueError):
        scan.run_resumable(4, 2, str(tmp_path / "bad"), lambda a, b: {"F": np.zeros((1, 9))})


def test_slice_bounds_cover_the_batch_with_growing_slices():
    from paper_1907_05993_gb300.pipeline import Pipeline
    assert Pipeline.slice_bounds(10_000, 4) == [0, 667, 2000, 4667, 10_000]
    for B in range(1, 40):
        for chunks in range(1, 7):
            cuts = Pipeline.slice_bounds(B, chunks)
            sizes = np.diff(cuts)
            assert cuts[0] == 0 and cuts[-1] == B and len(sizes) == min(chunks, B) and (sizes >= 1).all()
    assert Pipeline.slice_bounds(12, 3, growth=1.0) == [0, 4, 8, 12]
