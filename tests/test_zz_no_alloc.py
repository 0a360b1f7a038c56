"""The allocation-free registration entry point against the regular one.

hrebsd_demons_register_batch_noalloc serves callers that cannot allocate
device memory: hosts that fix the device-memory budget before they start,
plugins whose host application owns the allocator, and services that may not
allocate while serving a request.  Its workspace is a static 16 MiB array
inside the library.  It runs the same kernels with the same tile shapes as the
regular entry point, so its results must be bit-identical to it, on calls in a
row (the array keeps the previous call's contents: a call with other inputs in
between must leave no trace), with and without an initial field, and a batch
that does not fit must be refused.  This file is collected last so that a
failing run has already executed every other test.
"""
import numpy as np
import pytest

from synth import kikuchi as K

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point():
    import torch
    import oracle
    import paper_1907_05993_gb300 as P
    assert torch.cuda.is_available()
    ctx = P.hrebsd_create(0)
    try:
        spec = K.ScanSpec(n_pairs=10, H=128, W=128, n_refs=2, mis_lo_deg=0.5, mis_hi_deg=3.0, seed=41)
        refs = np.stack([oracle.preprocess(K.render_ref(spec, r).astype(np.float64)) for r in range(2)])
        tests = np.stack([oracle.preprocess(K.render_test(spec, p).astype(np.float64)) for p in range(10)])
        ridx = np.array([K.ref_index(spec, p) for p in range(10)], np.int32)
        d_ref = torch.from_numpy(refs.astype(np.float32)).cuda()
        d_test = torch.from_numpy(tests.astype(np.float32)).cuda()
        d_ridx = torch.from_numpy(ridx).cuda()
        params = P.demons_params(3, [30, 30, 30], 1.0, 1.0, 1.0, 1e-4, 5)
        params_init = P.demons_params(3, [20, 20, 20], 1.0, 1.0, 1.0, 1e-4, 5, 1)
        rng = np.random.default_rng(5)
        init = torch.from_numpy(rng.normal(0, 0.3, (10, 2, 64, 64)).astype(np.float32)).cuda()

        def run(fn, sl, prm, init_field=None):
            B = sl.stop - sl.start
            field = torch.full((B, 2, 128, 128), float("nan"), device="cuda")
            iters = torch.full((B, 3), -1, dtype=torch.int32, device="cuda")
            status = torch.full((B,), -1, dtype=torch.int32, device="cuda")
            fn(ctx, d_ref, d_test[sl].contiguous(), d_ridx[sl].contiguous(), 2, B, 128, 128, prm,
               None if init_field is None else init_field[sl].contiguous(), field, iters, status)
            torch.cuda.synchronize()
            return field.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy()

        def same(a, b):
            assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
            assert np.isfinite(a[0]).all() and np.array_equal(a[0], b[0])

        first, other = slice(0, 6), slice(6, 10)
        reg = P.hrebsd_demons_register_batch
        noa = P.hrebsd_demons_register_batch_noalloc
        ref0 = run(reg, first, params)
        ref_init = run(reg, first, params_init, init)
        same(run(noa, first, params), ref0)
        # another call with other patterns, another batch size and an initial field in between
        run(noa, other, params_init, init)
        same(run(noa, first, params), ref0)
        # the initial field goes through the static array too
        same(run(noa, first, params_init, init), ref_init)
        same(run(noa, first, params), ref0)

        # a batch beyond the static array is refused before any launch
        # (the host-side size check rejects it, so the undersized buffers are never touched)
        field, iters, status = (torch.empty(1, device="cuda"), torch.empty(1, dtype=torch.int32, device="cuda"),
                                torch.empty(1, dtype=torch.int32, device="cuda"))
        with pytest.raises(P.HrebsdError) as err:
            noa(ctx, d_ref, d_test, d_ridx, 2, 4096, 128, 128, params, None, field, iters, status)
        assert err.value.status == P.ESCRATCH
    finally:
        P.hrebsd_destroy(ctx)
