"""Failure detection on the GPU without a fault: a bounded wait that runs out reports
HREBSD_ETIMEOUT and leaves the context usable; degenerate and non-finite inputs are
flagged per pair (status bits) instead of stopping the batch."""
import numpy as np
import pytest

from synth import kikuchi as K

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1907_05993_gb300 as P
    assert torch.cuda.is_available()
    ctx = P.hrebsd_create(0)
    yield torch, P, ctx
    P.hrebsd_destroy(ctx)


def test_bounded_wait_runs_out_and_context_stays_usable(env):
    torch, P, ctx = env
    P.hrebsd_device_error(ctx)                     # nothing pending
    P.hrebsd_wait_selftest(ctx, 20000)             # a barrier nothing completes: gives up after 20k polls
    with pytest.raises(P.HrebsdError) as e:
        P.hrebsd_device_error(ctx)
    assert e.value.status == P.ETIMEOUT
    P.hrebsd_device_error(ctx)                     # the flag was cleared by the report
    with pytest.raises(P.HrebsdError):
        P.hrebsd_wait_selftest(ctx, 0)             # limit outside the range: EINVAL, nothing launched
    # the context still runs a registration, and reports no error afterwards
    spec = K.ScanSpec(n_pairs=2, H=64, W=64, n_refs=1, mis_lo_deg=0.5, mis_hi_deg=2.0, seed=3)
    refs, tests, ridx, _ = K.make_scan(spec)
    field = torch.empty((2, 2, 64, 64), dtype=torch.float32, device="cuda")
    iters = torch.empty((2, 2), dtype=torch.int32, device="cuda")
    status = torch.zeros((2,), dtype=torch.int32, device="cuda")
    P.hrebsd_demons_register_batch(ctx, torch.from_numpy(refs).cuda(), torch.from_numpy(tests).cuda(),
                                   torch.from_numpy(ridx).cuda(), 1, 2, 64, 64, P.demons_params(2, [10, 10]), None,
                                   field, iters, status)
    P.hrebsd_device_error(ctx)
    assert np.isfinite(field.cpu().numpy()).all() and (iters.cpu().numpy() == 10).all()


def test_degenerate_fit_sets_fit_failed(env):
    """All ROI centres at one point: the normal matrix of Eq. 3 is singular; that pair gets
    FIT_FAILED and identity matrices, the well-posed pair of the same batch is unaffected."""
    torch, P, ctx = env
    H = W = 64
    geom = P.hrebsd_geometry(0.5, 0.5, 0.6)
    field = torch.zeros((2, 2, H, W), dtype=torch.float32, device="cuda")
    good = K.roi_grid(H, W, 16, True)
    same = np.repeat(good[:1], len(good), axis=0)
    st = torch.zeros((2,), dtype=torch.int32, device="cuda")
    F1 = torch.empty((2, 9), dtype=torch.float64, device="cuda")
    Rf = torch.empty((2, 9), dtype=torch.float64, device="cuda")
    for b, roi in enumerate((good, same)):
        r = torch.from_numpy(np.ascontiguousarray(roi, dtype=np.int32)).cuda()
        P.hrebsd_fit_rotation(ctx, field[b:b + 1], 1, H, W, r, len(roi), geom, F1[b:b + 1], Rf[b:b + 1], st[b:b + 1])
    P.hrebsd_device_error(ctx)
    s = st.cpu().numpy()
    assert s[0] == 0 and (s[1] & P.PAIR_FIT_FAILED) and not (s[1] & P.PAIR_NONFINITE)
    eye = np.eye(3).ravel()
    assert np.abs(F1.cpu().numpy()[0] - eye).max() < 1e-12      # zero field: F = I by the fit
    assert np.array_equal(F1.cpu().numpy()[1], eye) and np.array_equal(Rf.cpu().numpy()[1], eye)
    # the second-pass solve flags the same way
    q = torch.zeros((1, len(same), 2), dtype=torch.float32, device="cuda")
    F = torch.empty((1, 9), dtype=torch.float64, device="cuda")
    st2 = torch.zeros((1,), dtype=torch.int32, device="cuda")
    r = torch.from_numpy(np.ascontiguousarray(same, dtype=np.int32)).cuda()
    P.hrebsd_solve_F(ctx, q, r, len(same), 1, H, W, geom, None, F, st2)
    P.hrebsd_device_error(ctx)
    assert st2.cpu().numpy()[0] & P.PAIR_FIT_FAILED
