"""The P2P kernel's own FP64 1/sqrt against CUDA's rsqrt (and exact rational checks)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def ulp_diff(a, b):
    ia, ib = a.view(np.int64), b.view(np.int64)
    return np.abs(ia - ib)


def test_own_rsqrt_within_one_ulp_of_cuda():
    import torch
    from paper_2005_12351_gb300 import fmm
    rng = np.random.default_rng(0)
    # log-uniform over 2^-1000 .. 2^1000, plus the P2P range and exact powers of 4
    x = np.concatenate([np.exp2(rng.uniform(-1000, 1000, 200_000)),
                        rng.uniform(1e-8, 4.0, 200_000),
                        np.exp2(2.0 * np.arange(-500, 500)),
                        np.nextafter(np.exp2(np.arange(-40.0, 40.0)), 0),
                        np.nextafter(np.exp2(np.arange(-40.0, 40.0)), np.inf)])
    own, ref = fmm.check_rsqrt(torch.from_numpy(x).cuda())
    own, ref = own.cpu().numpy(), ref.cpu().numpy()
    # both CUDA's rsqrt and ours are allowed 1 ulp from the true value
    assert ulp_diff(own, ref).max() <= 2
    # against an extended-precision host value (long double: 80-bit or binary128)
    exact = (1.0 / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    d = ulp_diff(own, exact)
    assert d.max() <= 1, d.max()
    assert (d == 0).mean() > 0.8
    # powers of four have exact reciprocal square roots
    p4 = np.exp2(2.0 * np.arange(-500, 500))
    own4, _ = fmm.check_rsqrt(torch.from_numpy(p4).cuda())
    assert np.array_equal(own4.cpu().numpy(), np.exp2(-np.arange(-500, 500, dtype=float)))


def test_own_rsqrt_subnormal_arguments():
    """Subnormal r^2 (0 < x < 2^-1022: particles closer than ~1.5e-154) are outside
    the exponent arithmetic of the fast path; they must still be within 1 ulp of
    the true value (and of CUDA's rsqrt)."""
    import torch
    from paper_2005_12351_gb300 import fmm
    rng = np.random.default_rng(1)
    tiny = np.float64(2.0 ** -1074)
    x = np.concatenate([np.exp2(rng.uniform(-1074, -1022, 50_000)),
                        np.array([tiny, 2 * tiny, 3 * tiny, np.nextafter(2.0 ** -1022, 0), 2.0 ** -1023]),
                        np.array([2.0 ** -1022, np.nextafter(2.0 ** -1022, 1)])])
    assert (x > 0).all() and (x[:-2] < 2.0 ** -1022).all()
    own, ref = fmm.check_rsqrt(torch.from_numpy(x).cuda())
    own, ref = own.cpu().numpy(), ref.cpu().numpy()
    assert np.isfinite(own).all()
    assert ulp_diff(own, ref).max() <= 2
    exact = (1.0 / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    assert ulp_diff(own, exact).max() <= 1
