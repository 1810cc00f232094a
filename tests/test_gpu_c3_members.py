"""The batched workload at full size (64 uneven grains, FP32, the layout
sc_batch_autotune picks): after two iterations from fresh boundary values, ten
members spread over the lower two thirds of the size order -- other energy
counts, lanes per line and energies-per-lane classes than the four grains the
benchmark checks -- equal two FP64 oracle sweeps within the production
tolerances (Delta_new 1e-5, j and F 1e-4 of the oracle's largest value)."""
import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_c3_members_match_oracle_in_the_tuned_layout():
    import torch
    from paper_2205_15000_b300 import sc
    grains = W.c3_batch()
    b = sc.Batch([p for p, _, _ in grains], precision="fp32")
    for (p, d, _), m in zip(grains, b.members):
        m.set_fields(d)
    b.autotune()
    b.reset_boundary()
    b.run(2, True)
    torch.cuda.synchronize()
    order = np.argsort([m.info.steps_per_sweep for m in b.members])
    check = [int(order[k]) for k in range(2, 42, 4)]
    for g in check:
        p, d, _ = grains[g]
        o = oracle.OracleGeom(p)
        mk = o.mask().astype(bool)
        r1 = o.full_sweep(d, None, None)
        ref = o.full_sweep(d, None, r1["exit"])
        got = b.members[g].outputs()
        for key, tol in (("delta_new", 1e-5), ("j", 1e-4), ("F", 1e-4)):
            a = got[key].cpu().numpy()[mk]
            e = ref[key][mk]
            err = np.max(np.abs(a - e)) / np.max(np.abs(e))
            assert err <= tol, (g, p["n_energies"], key, err)
    b.close()
