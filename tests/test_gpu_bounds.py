"""The bounds-checked build (libsc_checked.so, compiled with -DSC_DEBUG_BOUNDS:
every line, line-group, slot, sample, exit-tap, slab-row, padded-grid and
rotate-back index of the kernels is compared with the size of its table, a
failed check skips the access and counts) stands in for a device memory
checker.  On the parity grains -- three convex and composite grains in both
precisions, an energy-blocked grain, the adjoint, the LDOS, a batch and a batch
with a member in two energy parts -- it
must count no violation and give the regular build's results bit for bit
(the adjoint, whose cotangents are added with atomics in no fixed order, to
rounding)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_counts_no_violation_and_matches(tmp_path):
    import _bounds_run as R
    from paper_2205_15000_b300 import build
    assert os.path.exists(build.LIB_CHECKED), "build the checked library first (build(checked=True))"
    out = tmp_path / "checked.npz"
    env = dict(os.environ, SC_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_bounds_run.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    chk = np.load(out)
    assert int(chk["checked"]) == 1
    assert int(chk["violations"]) == 0
    reg, v, checked = R.run()
    assert not checked and v == 0
    assert set(reg) == set(chk.files) - {"violations", "checked"}
    for k, a in reg.items():
        b = chk[k]
        if k.startswith("adj_"):
            tol = 1e-12 if "_fp64_" in k else 1e-5
            assert np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(a)), 1e-30), k
        else:
            np.testing.assert_array_equal(a, b, err_msg=k)
