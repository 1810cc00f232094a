"""The FP32 sweep with 9 or 10 energies per lane (16 lanes per line): Matsubara
sums, the implicit midpoint stepper and Ozaki's weighted sums against the oracle
after two sweeps (FP32 tolerances as for every FP32 sweep: 1e-5 of the largest
Delta_new, 1e-4 of the largest F); the adjoint, which keeps at most 8 energies
per lane, refuses the layout when it is forced."""
import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _grain(n_e, **kw):
    kw.setdefault("pairing", 1)
    p = W.disc(3.0, 24, t=0.02, n_angles=8, n_energies=n_e, flux_quanta=0.4, **kw)
    d = W.vortex_delta(p, 0.24, [(0.5, -0.3)], [-1], seed=81, rel_noise=0.05)
    return p, d


def _outputs(ctx):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ctx.outputs().items()}


@pytest.mark.parametrize("n_e,ept,opts", [(150, 10, {}), (144, 9, {}), (150, 10, {"stepper": "midpoint"}),
                                          (150, 10, {"energy_sum": "ozaki"})])
def test_wide_layout_matches_oracle(n_e, ept, opts):
    from paper_2205_15000_b300 import sc
    p, d = _grain(n_e)
    p.update(opts)
    g = oracle.OracleGeom(p)
    m = g.mask().astype(bool)
    ctx = sc.Context(p, precision="fp32", lanes_per_line=16)
    info = sc.sc_get_info(ctx.h)
    assert (info.lanes_per_line, info.energies_per_lane) == (16, ept)
    ctx.set_fields(d)
    ex = None
    for _ in range(2):
        o = g.full_sweep(d, None, ex)
        ex = o["exit"]
        ctx.sweep()
    r = _outputs(ctx)
    assert np.max(np.abs(r["delta_new"][m] - o["delta_new"][m])) < 1e-5 * np.max(np.abs(o["delta_new"][m]))
    assert np.max(np.abs(r["j"][m] - o["j"][m])) < 1e-4 * np.max(np.abs(o["j"][m]))
    assert np.max(np.abs(r["F"][m] - o["F"][m])) < 1e-4 * np.max(np.abs(o["F"][m]))


def test_adjoint_refuses_a_forced_wide_layout():
    from paper_2205_15000_b300 import sc
    p, d = _grain(150)
    ctx = sc.Context(p, precision="fp32", lanes_per_line=16)
    ctx.set_fields(d)
    ctx.sweep()
    with pytest.raises(sc.ScError):
        ctx.adjoint(g_Ftotal=1.0)


@pytest.mark.parametrize("n_e,layout", [(160, (16, 10)), (80, (16, 5)), (144, (16, 9)), (128, (32, 4))])
def test_layout_choice_on_a_grain_that_fills_the_gpu(n_e, layout):
    """Least padding first; among equal padding the fewest issue units per line
    (16 x 10 rather than 32 x 5 for 160 energies; 32 x 4 and 16 x 8 tie and keep
    4 energies per lane)."""
    from paper_2205_15000_b300 import sc
    p, _, _ = W.c2_diamond_d(n=256, n_angles=64)
    p["n_energies"] = n_e
    ctx = sc.Context(p, precision="fp32")
    info = sc.sc_get_info(ctx.h)
    assert (info.lanes_per_line, info.energies_per_lane) == layout
    # FP64 keeps at most 8 energies per lane
    ctx64 = sc.Context(p, precision="fp64")
    assert sc.sc_get_info(ctx64.h).energies_per_lane <= 8


def test_batch_with_a_wide_member_matches_oracle():
    """A batch bounded by 10 energies per lane: the 150-energy member runs 16 x 10
    in its own class launch, the 40-energy member 8 x 5; both against the oracle
    after two sweeps (FP32 tolerances)."""
    from paper_2205_15000_b300 import sc
    p1, d1 = _grain(150)
    p2 = W.disc(4.0, 28, pairing=0, t=0.5, n_angles=16, n_energies=40, flux_quanta=0.7)
    d2 = W.noisy_delta(p2, 0.26, 0.1, seed=82)
    b = sc.Batch([p1, p2], precision="fp32", energies_per_lane=10)
    for m, d in zip(b.members, (d1, d2)):
        m.set_fields(d)
    for _ in range(2):
        b.sweep()
    for m, (p, d) in zip(b.members, ((p1, d1), (p2, d2))):
        g = oracle.OracleGeom(p)
        mask = g.mask().astype(bool)
        ex = None
        for _ in range(2):
            o = g.full_sweep(d, None, ex)
            ex = o["exit"]
        r = _outputs(m)
        assert np.max(np.abs(r["delta_new"][mask] - o["delta_new"][mask])) < 1e-5 * np.max(np.abs(o["delta_new"][mask]))
        assert np.max(np.abs(r["F"][mask] - o["F"][mask])) < 1e-4 * np.max(np.abs(o["F"][mask]))
    b.close()
