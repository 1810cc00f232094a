"""Error paths, all injected on the host: allocation failures (a fake of the
failing allocation), non-finite inputs, wrong call order.  Nothing here faults
or stalls the GPU."""
import math
import os

import numpy as np
import pytest

from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _grain():
    p = W.disc(4.0, 24, pairing=0, t=0.5, n_angles=8, n_energies=4, kappa=2.0)
    return p, W.noisy_delta(p, 0.25, 0.05, seed=5)


@pytest.mark.parametrize("n", [0, 1, 5, 12, 20, 30])
def test_allocation_failure_returns_enomem_and_leaks_nothing(n, monkeypatch):
    import torch
    from paper_2205_15000_b300 import sc
    p, d = _grain()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("SC_TEST_FAIL_ALLOC_AT", str(n))
    with pytest.raises(sc.ScError) as ei:
        c = sc.Context(p)
        # creation may need fewer than n + 1 allocations; then the lazy ones fail
        c.set_fields(d)
        c.sweep()
        c.outputs()
        sc.sc_update_vector_potential(c.h)
        c.adjoint(g_Ftotal=1.0)
    assert ei.value.status in (sc.SC_ENOMEM, sc.SC_ESTATE)
    monkeypatch.delenv("SC_TEST_FAIL_ALLOC_AT")
    import gc
    gc.collect()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)
    # the library is usable afterwards
    c = sc.Context(p)
    c.set_fields(d)
    c.sweep()
    assert math.isfinite(c.outputs()["F_total"])


def test_failed_context_rejects_later_calls(monkeypatch):
    from paper_2205_15000_b300 import sc
    p, d = _grain()
    # find how many allocations creation needs: the next one is the sweep's scratch
    c2 = None
    for n in range(0, 64):
        monkeypatch.setenv("SC_TEST_FAIL_ALLOC_AT", str(n))
        try:
            c2 = sc.Context(p)
        except sc.ScError as e:
            assert e.status == sc.SC_ENOMEM
            continue
        break
    monkeypatch.delenv("SC_TEST_FAIL_ALLOC_AT")
    assert c2 is not None
    c2.set_fields(d)
    with pytest.raises(sc.ScError) as ei:
        c2.sweep()
    assert ei.value.status == sc.SC_ENOMEM
    with pytest.raises(sc.ScError) as ei:
        c2.sweep()
    assert ei.value.status == sc.SC_ESTATE


def test_nan_in_delta_reports_enumeric():
    from paper_2205_15000_b300 import sc
    p, d = _grain()
    d = d.copy()
    d[p["ny"] // 2, p["nx"] // 2] = np.nan
    c = sc.Context(p)
    c.set_fields(d)
    c.sweep()
    with pytest.raises(sc.ScError) as ei:
        c.outputs()
    assert ei.value.status == sc.SC_ENUMERIC


def test_call_order_errors():
    from paper_2205_15000_b300 import sc
    p, d = _grain()
    c = sc.Context(p)
    c.set_fields(d)
    with pytest.raises(sc.ScError) as ei:
        c.outputs()  # no sweep since the fields were set
    assert ei.value.status == sc.SC_ESTATE
    with pytest.raises(sc.ScError) as ei:
        c.adjoint(g_Ftotal=1.0)
    assert ei.value.status == sc.SC_ESTATE
    with pytest.raises(sc.ScError) as ei:
        sc.sc_ldos(c.h, [-0.1, 0.2], 0.01, 2, None)
    assert ei.value.status == sc.SC_EINVAL
    with pytest.raises(sc.ScError) as ei:
        c.ldos([-0.1, 0.2], 0.01)  # not symmetric about zero
    assert ei.value.status == sc.SC_EINVAL
