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
    from paper_2205_15000_b300 import build
    assert os.path.exists(build.LIB_CHECKED), "build the checked library first (build(checked=True))"

    def run(checked_lib):
        # each library in its own process, whatever the test run itself loaded
        out = tmp_path / ("checked.npz" if checked_lib else "regular.npz")
        env = {k: v for k, v in os.environ.items() if k != "SC_LIBRARY"}
        if checked_lib:
            env["SC_LIBRARY"] = "checked"
        r = subprocess.run([sys.executable, os.path.join(HERE, "_bounds_run.py"), str(out)], env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
        return np.load(out)
    chk, regf = run(True), run(False)
    assert int(chk["checked"]) == 1 and int(chk["violations"]) == 0
    assert int(regf["checked"]) == 0 and int(regf["violations"]) == 0
    assert set(regf.files) == set(chk.files)
    reg = {k: regf[k] for k in regf.files if k not in ("violations", "checked")}
    for k, a in reg.items():
        b = chk[k]
        if k.startswith("adj_"):
            tol = 1e-12 if "_fp64_" in k else 1e-5
            assert np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(a)), 1e-30), k
        else:
            np.testing.assert_array_equal(a, b, err_msg=k)
