"""Checkpoint/resume on the GPU: the learned initialiser's training state (weights, Adam moments,
step), written by hrebsd_cnn_save and restored by hrebsd_cnn_load into a new context, continues
training as the uninterrupted run does, and damaged model files are refused; a scan
resumed after losing a chunk recomputes only that chunk and gives the same results."""
import os

import numpy as np
import pytest

from synth import kikuchi as K

pytestmark = pytest.mark.gpu


def test_training_checkpoint_resumes(tmp_path):
    import torch
    import paper_1907_05993_gb300 as P
    from paper_1907_05993_gb300 import learned as LN
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.normal(size=(16, 2, 64, 64)).astype(np.float32)).cuda().to(torch.bfloat16)
    tgt = torch.from_numpy(rng.normal(0, 0.5, (16, 2, 64, 64)).astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    path = str(tmp_path / "ckpt.hrcnn")
    ctxs = [P.hrebsd_create(0) for _ in range(3)]
    try:
        a = ctxs[0]
        P.hrebsd_cnn_init(a, LN.init_params(1))
        for _ in range(3):
            P.hrebsd_cnn_train_step(a, x, tgt, 16, 1e-3, loss)
        LN.save_checkpoint(a, path, epoch=np.int64(3))
        for _ in range(2):
            P.hrebsd_cnn_train_step(a, x, tgt, 16, 1e-3, loss)
        wa, _ = P.hrebsd_cnn_get_params(a)
        # resumed: weights, moments and step from the file
        b = ctxs[1]
        d = LN.load_checkpoint(b, path)
        assert int(d["epoch"]) == 3 and P.hrebsd_cnn_get_state(b)[2] == 3
        for _ in range(2):
            P.hrebsd_cnn_train_step(b, x, tgt, 16, 1e-3, loss)
        wb, _ = P.hrebsd_cnn_get_params(b)
        # weights only (Adam restarted): a different trajectory
        c = ctxs[2]
        P.hrebsd_cnn_init(c, d["params"])
        for _ in range(2):
            P.hrebsd_cnn_train_step(c, x, tgt, 16, 1e-3, loss)
        wc, _ = P.hrebsd_cnn_get_params(c)
        P.hrebsd_device_error(a)
        # gradients are summed with float atomics, so the runs agree to rounding, not bit for bit
        assert np.abs(wa - wb).max() <= 0.02 * np.abs(wa - wc).max()
        assert np.abs(wa - wc).max() > 1e-4
        # the model file is checked before anything is loaded
        raw = open(path, "rb").read()
        for bad in (raw[:-9], raw[:100] + bytes([raw[100] ^ 1]) + raw[101:], b"HRCNN002" + raw[8:]):
            with open(path + ".bad", "wb") as fh:
                fh.write(bad)
            before = P.hrebsd_cnn_get_params(c)[0]
            with pytest.raises(P.HrebsdError) as err:
                P.hrebsd_cnn_load(c, path + ".bad")
            assert err.value.status == P.EFORMAT
            assert np.array_equal(P.hrebsd_cnn_get_params(c)[0], before)
        with pytest.raises(P.HrebsdError) as err:
            P.hrebsd_cnn_load(c, str(tmp_path / "missing.hrcnn"))
        assert err.value.status == P.EIO
    finally:
        for ctx in ctxs:
            P.hrebsd_destroy(ctx)


def test_scan_resume_recomputes_only_missing_chunks(tmp_path):
    import torch
    from paper_1907_05993_gb300 import scan
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    spec = K.ScanSpec(n_pairs=6, H=128, W=128, n_refs=2, mis_lo_deg=0.5, mis_hi_deg=4.0, seed=9)
    refs, tests, ridx, _ = K.make_scan(spec)
    roi = K.roi_grid(128, 128, 32, True)
    pipe = Pipeline(PipelineConfig(128, 128, roi, 32, 3, (40, 40, 40), stop_tol=1e-4, stop_window=5))
    whole = pipe.run(torch.from_numpy(refs).cuda(), torch.from_numpy(tests).cuda(), torch.from_numpy(ridx).cuda())
    exp = {k: whole[k].cpu().numpy().copy() for k in ("F", "R_finite", "status")}
    h = (torch.from_numpy(refs).pin_memory(), torch.from_numpy(tests).pin_memory(), torch.from_numpy(ridx).pin_memory())
    d = str(tmp_path / "scan")
    out, computed = pipe.run_scan(*h, d, chunk=2, slices=2)
    assert computed == [0, 1, 2]
    os.remove(scan.chunk_path(d, 1))               # a lost chunk
    out2, computed2 = pipe.run_scan(*h, d, chunk=2, slices=2)
    assert computed2 == [1]
    for k, v in exp.items():
        assert np.array_equal(out[k], v) and np.array_equal(out2[k], v), k
    pipe.close()
