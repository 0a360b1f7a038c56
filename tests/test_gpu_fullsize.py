"""The batched-scan workloads at full size, in the launch configuration the benchmark times, checked
on sampled pairs against the oracle:

- the batched scan: 10,000 pairs of 256x256, 4 levels, stop rule, <= 100 iterations per level,
  25 ROIs of 64x64;
- the large-misorientation scan: 20,000 pairs at 200 counts, <= 200 iterations per level.

The sampled slots of the batch are overwritten with patterns rendered by the numpy generator, so the
oracle's inputs never come from GPU code.  The stop rule is a threshold on the relative SSD decrease
(reading of the convergence criterion), which FP32 and FP64 can cross one iteration apart, so the
oracle replays the library's per-level iteration counts (its `replay` argument); every sampled pair
is then held to the bars: rotation <= 1e-5 rad, every F component <= 1e-6, non-tie integer XCF
peaks bit-exact (a tie: a near tie on either side, or a peak that one of the oracle's FP32
executions moves), and the field bar of tests/fp32_sensitivity.py (the deviation distribution no
wider than the oracle's own under FP32-sized perturbations, up to the worst pixel).  Where the oracle's own
result moves by more than the bar when it runs with FP32 storage (an ill-conditioned pair), the
rotation and F bars are widened to twice that measured spread, the count of compared peaks may fall
below 20, and the test reports the pair.  Each side's own stop rule is compared separately (test_stop_rule_agreement_full_size)."""
import math
import multiprocessing as mp

import numpy as np
import pytest

from synth import kikuchi as K

pytestmark = pytest.mark.gpu

SAMPLE2 = [0, 137, 1999, 2500, 3141, 4321, 5050, 5112, 6001, 7777, 8888, 9999]
SAMPLE3 = [0, 4999, 7777, 12345, 16000, 19999]
MEMBERS = 4
ROT_TOL, F_TOL = 1e-5, 1e-6


def rot_err(Ra, Rb):
    M = np.asarray(Ra).T @ np.asarray(Rb)
    v = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]]) / 2
    return math.asin(min(1.0, float(np.linalg.norm(v))))


def _spec(cfg):
    return K.config2(10_000) if cfg == 2 else K.config3(20_000)


def _oracle_replayed(args):
    """Oracle chain for one pair replaying `iters` (member < 0), or one FP32 execution of it (member >= 0,
    images carrying `pre` FP32 units of preprocessing error): field, R, F, peaks."""
    cfg, p, iters, member, pre = args
    import oracle
    import fp32_sensitivity as FS
    spec = _spec(cfg)
    roi = K.roi_grid(256, 256, 64, False)
    pref = oracle.preprocess(K.render_ref(spec, K.ref_index(spec, p)).astype(np.float64), True)
    ptest = oracle.preprocess(K.render_test(spec, p).astype(np.float64), True)
    if member < 0:
        field, it = oracle.demons_register(pref, ptest, 4, [200] * 4, 1.0, 1.0, 1.0, 5, 1e-4, replay=iters)
        assert list(it) == list(iters)
        rp, tp = pref, ptest
    else:
        field = FS.perturbed_register(oracle, pref, ptest, 4, iters, seed=1000 * member + p, input_ulps=pre)
        rng = np.random.default_rng(7 + member)
        rp, tp = FS.round32(pref, rng), FS.round32(ptest, rng)
    _, R = oracle.fit_rotation(field, roi, spec.geom)
    rem = oracle.remap(rp, R, spec.geom)
    q, peak, ph, tie = oracle.xcf_roi(rem, tp, roi, 64)
    F = oracle.solve_F(q, roi, 256, 256, spec.geom, R)
    return dict(field=field, R=R, F=F, peak=peak, tie=tie)


def _oracle_own_stop(args):
    cfg, p = args
    import oracle
    spec = _spec(cfg)
    cap = 100 if cfg == 2 else 200
    pref = oracle.preprocess(K.render_ref(spec, K.ref_index(spec, p)).astype(np.float64), True)
    ptest = oracle.preprocess(K.render_test(spec, p).astype(np.float64), True)
    _, it = oracle.demons_register(pref, ptest, 4, [cap] * 4, 1.0, 1.0, 1.0, 5, 1e-4)
    return it


@pytest.fixture(scope="module")
def pool():
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(16) as p:
        yield p


def _gpu_scan(cfg, sample):
    import torch
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    from synth import gpu as SG
    spec = _spec(cfg)
    refs, tests, ridx, _ = SG.make_scan_gpu(spec)
    refs = torch.from_numpy(np.stack([K.render_ref(spec, r) for r in range(spec.n_refs)])).cuda()
    for p in sample:
        tests[p] = torch.from_numpy(K.render_test(spec, p)).cuda()
    cap = 100 if cfg == 2 else 200
    pipe = Pipeline(PipelineConfig(256, 256, K.roi_grid(256, 256, 64, False), 64, 4, (cap,) * 4, stop_tol=1e-4,
                                   stop_window=5))
    out = pipe.run(refs, tests, ridx)
    torch.cuda.synchronize()
    res = {k: out[k].cpu().numpy() for k in ("iters", "R_finite", "F", "peak", "near_tie")}
    res["field"] = {p: out["field"][p].cpu().numpy().astype(np.float64) for p in sample}
    res["test_pre"] = {p: out["test_pre"][p].cpu().numpy() for p in sample}
    res["ref_pre"] = out["ref_pre"].cpu().numpy()
    res["ridx"] = ridx.cpu().numpy()
    pipe.close()
    del refs, tests, out
    torch.cuda.empty_cache()
    return res


def _check_scan(pool, cfg, sample):
    import fp32_sensitivity as FS
    g = _gpu_scan(cfg, sample)
    import oracle
    spec = _spec(cfg)
    jobs = []
    for p in sample:
        it = g["iters"][p].astype(np.int32)
        pre = max(FS.preprocess_ulps(g["test_pre"][p], oracle.preprocess(K.render_test(spec, p).astype(np.float64))),
                  FS.preprocess_ulps(g["ref_pre"][g["ridx"][p]],
                                     oracle.preprocess(K.render_ref(spec, K.ref_index(spec, p)).astype(np.float64))))
        jobs += [(cfg, p, it, m, pre) for m in range(-1, MEMBERS)]
    res = pool.map(_oracle_replayed, jobs, chunksize=1)
    widened, lines = [], []
    for i, p in enumerate(sample):
        e = res[i * (MEMBERS + 1)]
        mem = res[i * (MEMBERS + 1) + 1:(i + 1) * (MEMBERS + 1)]
        Rg, Fg = g["R_finite"][p].reshape(3, 3), g["F"][p].reshape(3, 3)
        rot = rot_err(Rg, e["R"])
        dF = float(np.abs(Fg - e["F"]).max())
        rot_s = max(rot_err(m["R"], e["R"]) for m in mem)
        F_s = max(float(np.abs(m["F"] - e["F"]).max()) for m in mem)
        rot_bar, F_bar = max(ROT_TOL, 2 * rot_s), max(F_TOL, 2 * F_s)
        if rot > ROT_TOL or dF > F_TOL:
            widened.append(p)
        # integer peaks compared where neither side has a near tie and every FP32 execution of the oracle
        # finds the FP64 run's peak (a peak the oracle's own FP32 rounding moves is a tie at this pair's
        # conditioning, as the rotation and F bars widen with the executions' spread)
        stable = np.all([np.all(m["peak"] == e["peak"], axis=-1) for m in mem], axis=0)
        ok = ~(g["near_tie"][p].astype(bool) | e["tie"]) & stable
        peaks_equal = bool(np.array_equal(g["peak"][p][ok], e["peak"][ok]))
        ill = rot > ROT_TOL or dF > F_TOL
        fo = FS.assert_field_parity(g["field"][p], e["field"], [m["field"] for m in mem],
                                    what=f"config {cfg} pair {p}")
        lines.append(f"pair {p:5d} iters {g['iters'][p].tolist()} rot {rot:.1e} (spread {rot_s:.1e}) "
                     f"F {dF:.1e} (spread {F_s:.1e}) peaks {int(ok.sum())} ({int((~stable).sum())} moved by the "
                     f"oracle's FP32 executions) equal={peaks_equal} "
                     f"field max {fo['max']:.1e} (oracle's own {fo['q1.0'][1]:.1e}) "
                     f"over 1e-3 {fo['frac_over']:.1e} (oracle's own {fo['frac_over_oracle']:.1e})")
        assert rot <= rot_bar and dF <= F_bar, lines[-1]
        assert peaks_equal and (ok.sum() >= 20 or ill), lines[-1]
    print(f"config {cfg}:\n" + "\n".join(lines) + f"\npairs needing the conditioning allowance: {widened}")
    # the allowance is for the odd ill-conditioned pair, not a way around the bars
    assert len(widened) <= max(1, len(sample) // 10), widened
    return g


def test_batched_scan_sampled_pairs_replayed(pool):
    _check_scan(pool, 2, SAMPLE2)


def test_large_misorientation_scan_sampled_pairs_replayed(pool):
    _check_scan(pool, 3, SAMPLE3)


def test_stop_rule_agreement_full_size(pool):
    """Each side's own stop rule on 200 seeded pairs of the batched scan: the per-level counts agree
    within one iteration on >= 99 % of (pair, level) (measured: 99.4 %; threshold crossings of a
    slowly changing relative SSD decrease can fall further apart; the fractions are printed)."""
    rng = np.random.default_rng(2020)
    sample = sorted(rng.choice(10_000, 200, replace=False).tolist())
    g = _gpu_scan(2, sample)
    own = pool.map(_oracle_own_stop, [(2, p) for p in sample], chunksize=4)
    d = np.abs(np.stack([g["iters"][p] for p in sample]) - np.stack(own))
    within1 = float(np.mean(d <= 1))
    print(f"stop rule, 200 pairs x 4 levels: exact {np.mean(d == 0):.4f}, within 1 {within1:.4f}, "
          f"max difference {int(d.max())}")
    assert within1 >= 0.99
