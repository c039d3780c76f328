"""The face kernel's own FP64 reciprocal and reciprocal square root (an FP32
approximation refined by one third-order Newton-Raphson step) against CUDA's 1/x and
rsqrt and against a higher-precision reference: within one unit in the last place over
the whole normal range, and exactly CUDA's result where they fall back to it (zero,
subnormal, huge, non-finite and negative arguments)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_05489_gb300 import build

    build.build()
    from paper_2410_05489_gb300 import ase_df

    return ase_df


def run(A, x):
    import torch

    xd = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    out = torch.empty(4 * len(x), dtype=torch.float64, device="cuda")
    A.ase_df_check_recip(xd, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(-1, 4)
    return o[:, 0], o[:, 1], o[:, 2], o[:, 3]


def ulps(a, ref):
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def test_recip_and_rsqrt_within_one_ulp(A):
    rng = np.random.default_rng(11)
    x = np.concatenate([
        10.0 ** rng.uniform(-300, 300, 200000),                 # log-uniform over the normal range
        1.0 + rng.uniform(-1e-6, 1e-6, 20000),                   # near 1
        np.ldexp(1.0, np.arange(-1020, 1021)),                   # powers of two
        np.nextafter(np.ldexp(1.0, np.arange(-1019, 1021)), 0),  # all-ones mantissas
        rng.uniform(0.5, 4.0, 100000),                           # the scaled seed ranges
    ])
    r_own, r_cuda, s_own, s_cuda = run(A, x)
    ld = np.longdouble(x)
    r_ref = np.float64(np.longdouble(1) / ld)
    s_ref = np.float64(np.longdouble(1) / np.sqrt(ld))
    assert ulps(r_own, r_ref).max() <= 1.0
    assert ulps(s_own, s_ref).max() <= 1.0
    assert ulps(r_own, r_cuda).max() <= 1.0
    assert ulps(s_own, s_cuda).max() <= 1.0


def test_fallback_ranges_match_cuda(A):
    tiny = np.array([5e-324, 1e-310, 2.2250738585072014e-308, 4e-308, 1e-307])
    huge = np.array([1e307, 1.7976931348623157e308, 8.98846567431158e307])
    special = np.array([0.0, -0.0, -1.0, -2.5e-3, np.inf, -np.inf, np.nan])
    x = np.concatenate([tiny, huge, special])
    r_own, r_cuda, s_own, s_cuda = run(A, x)
    # below biased exponent 3 / above 2044 the reciprocal is CUDA's; the reciprocal
    # square root handles every positive normal value itself
    lo = (x > 0) & (x < np.ldexp(1.0, -1020))
    hi = x >= np.ldexp(1.0, 1021)
    bad = ~(x > 0) | np.isinf(x) | np.isnan(x)
    np.testing.assert_array_equal(r_own[lo | hi | bad], r_cuda[lo | hi | bad])
    sub = (x > 0) & (x < 2.2250738585072014e-308)
    np.testing.assert_array_equal(s_own[sub | bad], s_cuda[sub | bad])
    norm = (x >= 2.2250738585072014e-308) & np.isfinite(x)
    ld = np.longdouble(x[norm])
    assert ulps(s_own[norm], np.float64(np.longdouble(1) / np.sqrt(ld))).max() <= 1.0
