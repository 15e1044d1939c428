"""The element kernels' FP64-accurate sin(pi x) helpers against CUDA's sinpi
(GPU): the fixed-point evaluation (variant 0), the FP64-pipe polynomial
(variant 1, its fallback), the 62-fractional-bit integer value (variant 2)
and that value from an argument already in fixed point (variant 3, the FP64
load path)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _args():
    rng = np.random.default_rng(0)
    ints = np.arange(-8, 9, dtype=np.float64)
    near = np.concatenate([ints + d for d in (2.0 ** -40, -2.0 ** -40, 1e-3, -1e-3, 1e-9, -1e-9)])
    return np.concatenate([
        rng.uniform(-4, 4, 1 << 20), rng.uniform(0, 1, 1 << 18),
        np.arange(-8, 8.5, 0.5), np.arange(-8, 8.5, 0.25), [0.0, -0.0, 1e-300, -1e-300, 5e-324],
        [2.0 ** 51 - 0.5, 2.0 ** 51, 2.0 ** 53 + 2, 1e300, -1e300, np.inf, -np.inf, np.nan],
        np.nextafter(0.5, 1) + np.arange(16) * 1e-16, rng.uniform(-1e6, 1e6, 4096), near,
        # both sides of the fixed-point path's lower bound 2^-10 and upper bound 2^51
        2.0 ** -10 * np.array([0.999999, 1.0, 1.000001]), -(2.0 ** -10) * np.array([0.999999, 1.0, 1.000001]),
        np.nextafter(2.0 ** 51, 0) - np.arange(4), rng.uniform(2.0 ** 40, 2.0 ** 51, 256)])


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_sinpi_matches_cuda_library(variant):
    import torch
    from paper_1802_03433_gb300 import fea
    x = _args()
    if variant == 3:  # its documented argument range
        x = x[np.isfinite(x) & (np.abs(x) < 2.0 ** 58)]
    xt = torch.as_tensor(x, device="cuda")
    mine, ref = (t.cpu().numpy() for t in fea.fea_diag_sinpi(xt, variant))
    finite = np.isfinite(x)
    if variant < 2:  # an integer cannot carry NaN; the kernels flag non-finite geometry through det J
        assert np.array_equal(np.isnan(mine), np.isnan(ref))
    err = np.abs(mine[finite] - ref[finite])
    assert err.max() <= 4.5e-16, err.max()
    # relative accuracy where the value is small (near the zeros of sin(pi x));
    # the fixed-point value (variant 2) has absolute accuracy 2^-62
    small = finite & (np.abs(ref) > (1e-3 if variant >= 2 else 0)) & (np.abs(ref) < 1e-2)
    rel = np.abs(mine[small] - ref[small]) / np.abs(ref[small])
    assert rel.max() <= 6e-16, rel.max()
    # odd symmetry and exact values at half-integers and zeros
    half = np.arange(-8, 8.5, 0.5)
    m = fea.fea_diag_sinpi(torch.as_tensor(half, device="cuda"), variant)[0].cpu().numpy()
    np.testing.assert_array_equal(np.abs(m[(half * 2) % 2 == 0]), 0.0)
    np.testing.assert_allclose(np.abs(m[(half * 2) % 2 == 1]), 1.0, rtol=0, atol=4.5e-16)
    if variant < 2:  # an integer has no negative zero
        assert np.signbit(fea.fea_diag_sinpi(torch.tensor([-0.0], device="cuda", dtype=torch.float64),
                                             variant)[0].item())
    sym = fea.fea_diag_sinpi(torch.as_tensor(-x[finite], device="cuda"), variant)[0].cpu().numpy()
    np.testing.assert_array_equal(sym, -mine[finite])
