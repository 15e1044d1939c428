"""The element kernels' FP64 sin(pi x) against CUDA's sinpi (GPU)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_sinpi_matches_cuda_library():
    import torch
    from paper_1802_03433_gb300 import fea
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.uniform(-4, 4, 1 << 20), rng.uniform(0, 1, 1 << 18),
        np.arange(-8, 8.5, 0.5), np.arange(-8, 8.5, 0.25), [0.0, -0.0, 1e-300, -1e-300, 5e-324],
        [2.0 ** 51 - 0.5, 2.0 ** 51, 2.0 ** 53 + 2, 1e300, -1e300, np.inf, -np.inf, np.nan],
        np.nextafter(0.5, 1) + np.arange(16) * 1e-16, rng.uniform(-1e6, 1e6, 4096)])
    xt = torch.as_tensor(x, device="cuda")
    mine, ref = (t.cpu().numpy() for t in fea.fea_diag_sinpi(xt))
    finite = np.isfinite(x)
    assert np.array_equal(np.isnan(mine), np.isnan(ref))
    err = np.abs(mine[finite] - ref[finite])
    assert err.max() <= 4.5e-16, err.max()
    # odd symmetry and exact values at half-integers and zeros
    half = np.arange(-8, 8.5, 0.5)
    m = fea.fea_diag_sinpi(torch.as_tensor(half, device="cuda"))[0].cpu().numpy()
    np.testing.assert_array_equal(np.abs(m[(half * 2) % 2 == 0]), 0.0)
    np.testing.assert_allclose(np.abs(m[(half * 2) % 2 == 1]), 1.0, rtol=0, atol=4.5e-16)
    assert np.signbit(fea.fea_diag_sinpi(torch.tensor([-0.0], device="cuda", dtype=torch.float64))[0].item())
