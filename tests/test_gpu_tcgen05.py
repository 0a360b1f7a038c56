"""The tcgen05 building blocks (shared-memory descriptors, BF16 MMA into tensor memory, commit,
TMEM loads) on one GEMM tile against a float64 product of the same BF16 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,KS", [(16, 1), (32, 2), (64, 4), (16, 3)])
def test_tcgen05_gemm_tile(N, KS):
    import torch
    import paper_1907_05993_gb300 as P
    ctx = P.hrebsd_create(0)
    rng = np.random.default_rng(N * 10 + KS)
    K = 16 * KS
    A = torch.from_numpy(rng.normal(size=(128, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    B = torch.from_numpy(rng.normal(size=(N, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    D = torch.full((128, N), float("nan"), device="cuda")
    P.hrebsd_tc_selftest(ctx, A, B, N, KS, D)
    P.hrebsd_device_error(ctx)
    exp = A.float().cpu().numpy().astype(np.float64) @ B.float().cpu().numpy().astype(np.float64).T
    got = D.cpu().numpy()
    assert np.abs(got - exp).max() <= 1e-4 * np.abs(exp).max(), np.abs(got - exp).max()
    P.hrebsd_destroy(ctx)
