"""Batching machinery (project addition): tile-shape variants, the autotuner and the
per-level CUDA graphs.  None of them may change the registration's result."""
import numpy as np
import pytest

from synth import kikuchi as K

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def lib(torch):
    import paper_1907_05993_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def pairs(oracle):
    """Four noisy pairs of the batched-scan kind at 256x256, two references."""
    spec = K.ScanSpec(n_pairs=4, H=256, W=256, n_refs=2, mis_lo_deg=0.5, mis_hi_deg=5.0, seed=71)
    refs = np.stack([oracle.preprocess(K.render_ref(spec, r).astype(np.float64), True) for r in range(2)])
    tests = np.stack([oracle.preprocess(K.render_test(spec, p).astype(np.float64), True) for p in range(4)])
    ridx = np.array([K.ref_index(spec, p) for p in range(4)], dtype=np.int32)
    return refs.astype(np.float32), tests.astype(np.float32), ridx


def _register(torch, lib, ctx, pairs, params):
    refs, tests, ridx = pairs
    R, H, W = refs.shape
    B = tests.shape[0]
    field = torch.empty((B, 2, H, W), dtype=torch.float32, device="cuda")
    iters = torch.empty((B, params.levels), dtype=torch.int32, device="cuda")
    status = torch.empty((B,), dtype=torch.int32, device="cuda")
    lib.hrebsd_demons_register_batch(ctx, torch.from_numpy(refs).cuda(), torch.from_numpy(tests).cuda(),
                                     torch.from_numpy(ridx).cuda(), R, B, H, W, params, None, field, iters, status)
    lib.hrebsd_device_error(ctx)   # raises if a bounded wait gave up
    return field.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy()


def test_tile_shapes_give_the_same_field(torch, lib, pairs):
    """Fixed iteration counts: every tile shape yields a bit-identical field."""
    params = lib.demons_params(4, [12] * 4, 1.0, 1.0, 1.0)
    out = []
    for v in range(lib.TILE_VARIANTS):
        ctx = lib.hrebsd_create(0)
        for l in range(4):
            lib.hrebsd_set_tile_variant(ctx, 256 >> l, 256 >> l, v)
            assert lib.hrebsd_get_tile_variant(ctx, 256 >> l, 256 >> l) == v
        out.append(_register(torch, lib, ctx, pairs, params))
        lib.hrebsd_destroy(ctx)
    for f, it, st in out[1:]:
        assert np.array_equal(f, out[0][0])
        assert np.array_equal(it, out[0][1]) and np.array_equal(st, out[0][2])


def test_tile_shapes_agree_on_ragged_tiles(torch, lib, oracle):
    """96x96 patterns (levels 96, 48, 24): 64x64 and 64x32 tiles run past the image edge, so the
    border replication of partial tiles is exercised; with fixed iteration counts every shape gives
    a bit-identical field."""
    spec = K.ScanSpec(n_pairs=3, H=96, W=96, n_refs=1, mis_lo_deg=0.5, mis_hi_deg=3.0, seed=77)
    refs = np.stack([oracle.preprocess(K.render_ref(spec, 0).astype(np.float64), True)]).astype(np.float32)
    tests = np.stack([oracle.preprocess(K.render_test(spec, p).astype(np.float64), True)
                      for p in range(3)]).astype(np.float32)
    ridx = np.zeros(3, dtype=np.int32)
    params = lib.demons_params(3, [15] * 3, 1.0, 1.0, 1.0)
    out = []
    for v in range(lib.TILE_VARIANTS):
        ctx = lib.hrebsd_create(0)
        for l in range(3):
            lib.hrebsd_set_tile_variant(ctx, 96 >> l, 96 >> l, v)
        out.append(_register(torch, lib, ctx, (refs, tests, ridx), params))
        lib.hrebsd_destroy(ctx)
    assert np.isfinite(out[0][0]).all() and np.abs(out[0][0]).max() > 0
    for f, it, st in out[1:]:
        assert np.array_equal(f, out[0][0])
        assert np.array_equal(it, out[0][1]) and np.array_equal(st, out[0][2])


def test_autotune_records_the_fastest_shape(torch, lib):
    ctx = lib.hrebsd_create(0)
    params = lib.demons_params(4, [100] * 4, 1.0, 1.0, 1.0, 1e-4, 5)
    ms = lib.hrebsd_autotune(ctx, 64, 256, 256, params)
    assert ms.shape == (4, lib.TILE_VARIANTS)
    # the row sweep (shapes 5 and 6) covers levels 64, 128 and 256 pixels wide, not 32; the level in
    # shared memory (7) levels of at most 64 x 64
    assert np.isfinite(ms[:, :5]).all() and (ms[:, :5] > 0).all(), ms
    assert np.isfinite(ms[:3, 5:7]).all() and np.isnan(ms[3, 5:7]).all(), ms
    assert np.isnan(ms[:2, 7]).all() and np.isfinite(ms[2:, 7]).all(), ms
    area = np.array(lib.TILE_AREAS, dtype=np.float64)
    ctrl = np.where(np.arange(lib.TILE_VARIANTS) < 7, 0.005, 0.0)   # the control launch of shapes 0-6
    score = (ms + ctrl) * (1.0 + 0.01 * np.maximum(0.0, np.log2(4096.0 / area)))   # and the small-tile handicap
    score[:, 6] = np.nan   # shape 6 is timed but never chosen
    for l in range(4):
        assert lib.hrebsd_get_tile_variant(ctx, 256 >> l, 256 >> l) == int(np.nanargmin(score[l]))
    # radius 0 (no smoothing): nothing to tune
    ms0 = lib.hrebsd_autotune(ctx, 8, 64, 64, lib.demons_params(2, [5, 5], 1.0, 0.0, 0.0))
    assert np.isnan(ms0).all()
    with pytest.raises(lib.HrebsdError):
        lib.hrebsd_autotune(ctx, 8, 60, 64, lib.demons_params(4, [5] * 4))   # coarsest level 7 x 8
    lib.hrebsd_destroy(ctx)


def test_level_in_one_launch_matches_row_sweep_with_stop_rule(torch, lib, pairs):
    """Shape 6 runs a level's iterations after the first in one launch and applies the stop rule in
    each pair's CTA; with the same SSD partials as shape 5 (one per pair) it must stop every pair at
    the same iteration and give the same field, bit for bit, also with a cap that ends some pairs.
    The four pairs are repeated to 1,600, more than the resident CTAs of any level, so that shape 5
    runs one launch per iteration (with fewer pairs it takes the one-launch form itself)."""
    refs, tests, ridx = pairs
    big = (refs, np.tile(tests, (400, 1, 1)), np.tile(ridx, 400))
    for caps in ([100] * 4, [9, 30, 100, 100]):
        params = lib.demons_params(4, caps, 1.0, 1.0, 1.0, 1e-4, 5)
        out = []
        for v in (5, 6):
            ctx = lib.hrebsd_create(0)
            for l in range(4):
                lib.hrebsd_set_tile_variant(ctx, 256 >> l, 256 >> l, v)
            out.append(_register(torch, lib, ctx, big, params))
            lib.hrebsd_destroy(ctx)
        (f5, it5, st5), (f6, it6, st6) = out
        assert np.array_equal(it5, it6) and np.array_equal(st5, st6), (it5, it6, st5, st6)
        assert np.array_equal(f5, f6)
        assert it5.max() > 1
        assert np.array_equal(f5[:4], f5[4:8]) and np.array_equal(it5[:4], it5[-4:])


def test_texture_gathers_match_plain_loads(torch, lib, pairs):
    """The row sweep's moving image by texture gathers from the context's CUDA-array copy of the
    references (the default) equals plain loads, per-iteration launches (shape 5) and the loop form
    (shape 6), stop rule on.  Ten references, the pairs pointing at the last two: texture rows beyond
    the array's first allocation (8 references), so the array grows between calls (device synchronised,
    cached graphs dropped) and the row offset of a reference is exercised."""
    params = lib.demons_params(4, [40] * 4, 1.0, 1.0, 1.0, 1e-4, 5)
    refs, tests, ridx = pairs
    many = (np.concatenate([refs] * 5), tests, (ridx + 8).astype(np.int32))
    for v in (5, 6):
        res = {}
        for tex in (0, 1):
            ctx = lib.hrebsd_create(0)
            lib.hrebsd_set_option(ctx, lib.OPT_TEX_GATHER, tex)
            for l in range(4):
                lib.hrebsd_set_tile_variant(ctx, 256 >> l, 256 >> l, v)
            res[tex] = (_register(torch, lib, ctx, pairs, params), _register(torch, lib, ctx, many, params),
                        _register(torch, lib, ctx, pairs, params))
            lib.hrebsd_destroy(ctx)
        for run in range(3):
            for a, b in zip(res[0][run], res[1][run]):
                assert np.array_equal(a, b), (v, run)
        for a, b in zip(res[1][0], res[1][1]):
            assert np.array_equal(a, b), v
        assert res[1][0][1].max() > 5   # the stop rule ran


def test_graph_replay_matches_direct_launches(torch, lib, pairs):
    """Stop rule on: the graph path (captured, then replayed from the cache) equals direct launches."""
    params = lib.demons_params(4, [60] * 4, 1.0, 1.0, 1.0, 1e-4, 5)
    res = {}
    for graphs in (0, 1):
        ctx = lib.hrebsd_create(0)
        lib.hrebsd_set_option(ctx, lib.OPT_GRAPHS, graphs)
        first = _register(torch, lib, ctx, pairs, params)
        n1 = lib.hrebsd_launch_count(ctx)
        second = _register(torch, lib, ctx, pairs, params)
        n2 = lib.hrebsd_launch_count(ctx)
        for a, b in zip(first, second):
            assert np.array_equal(a, b)
        res[graphs] = (first, n1, n2 - n1)
        lib.hrebsd_destroy(ctx)
    for a, b in zip(res[0][0], res[1][0]):
        assert np.array_equal(a, b)
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]   # same kernel launches counted


def test_graphs_on_a_side_stream(torch, lib, pairs):
    params = lib.demons_params(2, [8, 8], 1.0, 1.0, 1.0)
    refs, tests, ridx = pairs
    ctx = lib.hrebsd_create(0)
    ref_ = lib.demons_params(2, [8, 8], 1.0, 1.0, 1.0)
    base = _register(torch, lib, ctx, pairs, ref_)
    s = torch.cuda.Stream()
    R, H, W = refs.shape
    B = tests.shape[0]
    with torch.cuda.stream(s):
        field = torch.empty((B, 2, H, W), dtype=torch.float32, device="cuda")
        iters = torch.empty((B, 2), dtype=torch.int32, device="cuda")
        status = torch.empty((B,), dtype=torch.int32, device="cuda")
        r_d, t_d, i_d = (torch.from_numpy(refs).cuda(), torch.from_numpy(tests).cuda(),
                         torch.from_numpy(ridx).cuda())
        for _ in range(2):
            lib.hrebsd_demons_register_batch(ctx, r_d, t_d, i_d, R, B, H, W, params, None, field, iters, status,
                                             stream=s)
    s.synchronize()
    assert np.array_equal(field.cpu().numpy(), base[0])
    lib.hrebsd_destroy(ctx)


def test_run_host_matches_run(torch, lib):
    """Pinned host inputs processed in slices with overlapped copies (3 slices of 2, 2 and 1 pairs,
    staging slots reused): the same F, rotation and status as one run on the whole batch."""
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    spec = K.ScanSpec(n_pairs=5, H=128, W=128, n_refs=2, mis_lo_deg=0.5, mis_hi_deg=4.0, seed=5)
    refs, tests, ridx, _ = K.make_scan(spec)
    roi = K.roi_grid(128, 128, 32, True)
    pipe = Pipeline(PipelineConfig(128, 128, roi, 32, 3, (40, 40, 40), stop_tol=1e-4, stop_window=5))
    whole = pipe.run(torch.from_numpy(refs).cuda(), torch.from_numpy(tests).cuda(), torch.from_numpy(ridx).cuda())
    exp = {k: whole[k].cpu().numpy().copy() for k in ("F", "R_finite", "status")}
    h = pipe.run_host(torch.from_numpy(refs).pin_memory(), torch.from_numpy(tests).pin_memory(),
                      torch.from_numpy(ridx).pin_memory(), chunks=3)
    torch.cuda.synchronize()
    lib.hrebsd_device_error(pipe.ctx)
    for k, v in exp.items():
        assert np.array_equal(h[k].numpy(), v), k
    pipe.close()
