"""The GPU twin of the seeded Kikuchi generator (synth/csrc/kikuchi_gen.cu, input generation for
large batches) against the numpy generator synth/kikuchi.py, whose pins are in
tests/test_generator_pins.py.  The random counters are the same, so the two agree to FP32 rounding
of the band arithmetic: noise-free patterns to a relative 2e-5, noisy patterns to at most one count,
at a small fraction of the pixels (where the rounding moves lambda + sqrt(lambda) z + (z^2 - 1)/6
across a half-integer)."""
import numpy as np
import pytest

from synth import kikuchi as K

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [2, 3])
def test_gpu_generator_matches_numpy(cfg):
    import torch
    from synth import gpu as SG
    spec = K.config2(10_000) if cfg == 2 else K.config3(20_000)
    pairs = [0, 1, 4321, spec.n_pairs - 1]
    for noise in (False, True):
        refs, tests, ridx, Ft = SG.make_scan_gpu(spec, pairs=pairs, noise=noise)
        torch.cuda.synchronize()
        refs, tests = refs.cpu().numpy(), tests.cpu().numpy()
        for r in range(spec.n_refs):
            exp = K.render_ref(spec, r, noise)
            _check(refs[r], exp, noise)
        for i, p in enumerate(pairs):
            assert int(ridx[i]) == K.ref_index(spec, p)
            assert np.array_equal(Ft[i], K.pair_truth(spec, p))
            _check(tests[i], K.render_test(spec, p, noise), noise)


def _check(got, exp, noise):
    if not noise:
        assert np.abs(got - exp).max() <= 2e-5 * np.abs(exp).max()
        return
    d = np.abs(got.astype(np.float64) - exp)
    assert d.max() <= 1.0
    assert np.mean(d > 0) <= 2e-3, np.mean(d > 0)
