"""GPU checks of the measurement probe and of the saturated RHS's reciprocal.

The reciprocal (a hardware estimate refined by one third-order Newton-Raphson step, with an
IEEE division outside [2^-1000, 2^1001)) is compared with the correctly rounded 1/x (numpy's
IEEE division on the host) over a seeded sweep: random normals over the whole exponent range,
both sides of the two switch points, powers of two, subnormals, zeros, infinities and NaN.
"""
import numpy as np
import pytest

from paper_2306_13002_gb300 import binding

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# The error bound the sweep establishes (and the library's documentation states): the refined
# reciprocal is within 1 ulp of the correctly rounded 1/x (faithful rounding); the fallback
# range is the IEEE division itself.
MAX_ULP_REFINED = 1


def _ulp_distance(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distance in units in the last place between doubles of the same sign (as ordered ints)."""
    ia = a.view(np.int64).astype(np.int64)
    ib = b.view(np.int64).astype(np.int64)
    return np.abs(ia - ib)


def _sweep(seed: int = 2306) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    # random normals over the whole exponent range, both signs
    m = rng.uniform(1.0, 2.0, 400_000)
    e = rng.integers(-1022, 1024, 400_000)
    parts.append(np.ldexp(m, e) * rng.choice([-1.0, 1.0], 400_000))
    # the densities the RHS sees
    parts.append(rng.uniform(0.5, 1.5, 200_000))
    # mantissas near 1 and near 2 (where the estimate's error is largest relative to the result)
    parts.append(1.0 + rng.uniform(0, 1e-6, 20_000))
    parts.append(2.0 - rng.uniform(0, 1e-6, 20_000))
    # both sides of the switch points 2^-1000 and 2^1001, a few ulps apart
    for edge in (2.0 ** -1000, 2.0 ** 1001):
        x = np.full(2001, edge)
        steps = np.arange(-1000, 1001)
        x = x.view(np.int64) + steps
        parts.append(x.view(np.float64))
        parts.append(-x.view(np.float64))
    # every power of two, and its neighbours
    p2 = np.ldexp(1.0, np.arange(-1074, 1024))
    parts += [p2, np.nextafter(p2, np.inf), np.nextafter(p2, 0.0), -p2]
    # the smallest normals and subnormals, zeros, infinities, NaN
    parts.append(np.array([2.0 ** -1022, 2.0 ** -1022 * 1.5, 5e-324, 1e-310, 0.0, -0.0, np.inf, -np.inf, np.nan,
                           np.finfo(np.float64).max, -np.finfo(np.float64).max]))
    return np.concatenate(parts)


def test_refined_reciprocal_is_faithful_and_falls_back_to_ieee_division():
    x = _sweep()
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    binding.acs_rcp_selftest(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x
    ax = np.abs(x)
    refined = (ax >= 2.0 ** -1000) & (ax < 2.0 ** 1001)
    assert refined.sum() > 500_000 and (~refined).sum() > 2_000
    # refined range: finite, same sign, within MAX_ULP_REFINED of the correctly rounded value
    assert np.all(np.isfinite(y[refined]))
    assert np.all(np.signbit(y[refined]) == np.signbit(ref[refined]))
    d = _ulp_distance(y[refined], ref[refined])
    assert d.max() <= MAX_ULP_REFINED, (int(d.max()), x[refined][np.argmax(d)])
    # most results are the correctly rounded value itself
    assert (d == 0).mean() > 0.99
    # fallback range (zero, subnormal, huge, inf, NaN, and the normals outside the range):
    # the IEEE division, bit for bit (NaN as NaN)
    fb = ~refined
    nan = np.isnan(ref[fb])
    assert np.array_equal(np.isnan(y[fb]), nan)
    assert np.array_equal(y[fb][~nan].view(np.int64), ref[fb][~nan].view(np.int64))


def test_rcp_selftest_rejects_overlap_and_accepts_empty():
    x = torch.ones(16, dtype=torch.float64, device="cuda")
    import ctypes
    L = binding.lib()
    assert L.acs_rcp_selftest(x.data_ptr(), x.data_ptr() + 64, 16, None) == 7      # ACS_ERR_ALIAS
    assert L.acs_rcp_selftest(x.data_ptr(), x.data_ptr(), 0, None) == 0
    del ctypes


def test_fp64_rate_probe_runs_and_counts_its_operations():
    blocks, threads, iters = 2 * 152, 256, 64
    sink = torch.full((blocks * threads,), float("nan"), dtype=torch.float64, device="cuda")
    ops = binding.acs_fp64_rate_probe(sink, blocks, threads, iters)
    torch.cuda.synchronize()
    assert ops == blocks * threads * iters * 8
    s = sink.cpu().numpy()
    # every chain tends to the fixed point 1 of a <- 0.75 a + 0.25: eight chains sum to ~8
    assert np.all(np.isfinite(s)) and np.all(np.abs(s - 8.0) < 1.0)
