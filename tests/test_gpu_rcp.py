"""The element kernels' FP64 reciprocal (the 1 / (6 |det J|) that scales
their gradient products) against CUDA's division 1.0 / x (GPU): within one
ulp on the fast path, exactly the division on its fallback, and exact on
powers of two so that a mesh scaled by a power of two scales its matrix
exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    ia, ib = a.view(np.int64), b.view(np.int64)
    return np.abs(ia - ib)


def test_reciprocal_within_one_ulp_of_the_division():
    import torch
    from paper_1802_03433_gb300 import fea
    rng = np.random.default_rng(3)
    m = rng.uniform(1.0, 2.0, 1 << 20)
    edges = np.array([1.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 1.5, 1.25, 3.0, 6.0])
    fast = np.concatenate([
        m, m * np.exp2(rng.integers(-990, 991, m.size)).astype(np.float64), edges,
        # the ends of the fast path's exponent range and the FP32 seed's breakpoints
        2.0 ** -1000 * np.array([1.0, 1.5, np.nextafter(2.0, 1.0)]), 2.0 ** 1000 * np.array([1.0, 1.75]),
        1.0 + np.arange(1, 4096) * 2.0 ** -23, 1.0 + np.arange(1, 4096) * 2.0 ** -23 - 2.0 ** -52])
    mine, ref = (t.cpu().numpy() for t in fea.fea_diag_rcp(torch.as_tensor(fast, device="cuda")))
    assert _ulps(mine, ref).max() <= 1
    assert (_ulps(mine, ref) == 0).mean() > 0.999  # one Newton step of third order: nearly always the rounded value


def test_reciprocal_fallback_and_powers_of_two():
    import torch
    from paper_1802_03433_gb300 import fea
    k = np.arange(-1074, 1024)
    pw = np.ldexp(1.0, k)
    odd = np.array([0.0, 5e-324, 1e-310, 2.0 ** -1001, 2.0 ** 1001, 1.7e308, np.inf, np.nan, -1.0, -3.5, -0.0])
    x = np.concatenate([pw, odd])
    mine, ref = (t.cpu().numpy() for t in fea.fea_diag_rcp(torch.as_tensor(x, device="cuda")))
    # powers of two: the exact reciprocal wherever it is a normal double
    normal = np.abs(k) <= 1022
    assert np.array_equal(mine[: pw.size][normal], np.ldexp(1.0, -k[normal]))
    # outside the fast path the helper is the division itself, bit for bit (NaN as NaN)
    tail = slice(pw.size, None)
    assert np.array_equal(np.isnan(mine[tail]), np.isnan(ref[tail]))
    ok = ~np.isnan(ref[tail])
    assert np.array_equal(mine[tail][ok].view(np.int64), ref[tail][ok].view(np.int64))
    assert _ulps(mine[: pw.size], ref[: pw.size]).max() <= 1
