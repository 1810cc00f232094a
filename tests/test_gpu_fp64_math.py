"""The FP64 reciprocal and reciprocal square root of the device sweep (Newton-
Raphson iteration from the FP32 unit approximations) against the correctly
rounded values: within 1 ulp for 1/x and 2 ulp for 1/sqrt(x) (reference in
80-bit extended precision), over magnitudes 1e-30 ... 1e30, random mantissas,
powers of two and their neighbours, and arguments outside the float range (which
take the IEEE operations)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(71)
    x = [10.0 ** rng.uniform(-30, 30, 20000),
         rng.uniform(0.5, 2.0, 5000),
         2.0 ** np.arange(-60, 61).astype(np.float64)]
    p2 = 2.0 ** np.arange(-20, 21).astype(np.float64)
    x += [np.nextafter(p2, 0), np.nextafter(p2, np.inf)]
    x += [np.array([1e-40, 3e-39, 1e-300, 4.9e-324, 1e39, 1e300, 1.7e308, 1.0, 3.0, 7.0])]
    return np.concatenate(x)


def _ulps(v, ref):
    return np.abs(v - ref) / np.spacing(np.abs(ref))


def test_fp64_device_reciprocal_and_rsqrt():
    import torch
    from paper_2205_15000_b300 import sc
    x = _inputs()
    rcp, rsq = sc.sc_debug_fp64_math(torch.as_tensor(x, device="cuda"))
    rcp, rsq = rcp.cpu().numpy(), rsq.cpu().numpy()
    with np.errstate(over="ignore", divide="ignore"):
        ref_r = 1.0 / x
        xl = x.astype(np.longdouble)
        ref_q = (np.longdouble(1) / np.sqrt(xl)).astype(np.float64)
    fin = np.isfinite(ref_r) & (ref_r != 0)
    assert np.max(_ulps(rcp[fin], ref_r[fin])) <= 1.0, np.max(_ulps(rcp[fin], ref_r[fin]))
    assert np.max(_ulps(rsq, ref_q)) <= 2.0, np.max(_ulps(rsq, ref_q))
    # where 1/x overflows (denormal x), the IEEE fallback gives inf like the reference
    assert np.array_equal(rcp[~fin], ref_r[~fin])


def test_fp64_math_rejects_bad_arguments():
    from paper_2205_15000_b300 import sc
    assert sc.lib.sc_debug_fp64_math(None, -1, None, None, None) == sc.SC_EINVAL
    assert sc.lib.sc_debug_fp64_math(None, 4, None, None, None) == sc.SC_EINVAL
    assert sc.lib.sc_debug_fp64_math(None, 0, None, None, None) == sc.SC_OK
