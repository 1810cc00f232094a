"""Batched form: many grains of uneven size, shape, pairing, temperature,
field and angle count in one persistent sweep launch must give every grain
exactly what its own context gives (and, in FP64, what the oracle gives)."""
import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _grains():
    out = []
    p = W.disc(4.0, 28, pairing=0, t=0.5, n_angles=16, n_energies=10, flux_quanta=0.7)
    out.append((p, W.noisy_delta(p, 0.26, 0.1, seed=31)))
    p = W.diamond(9.0, 36, pairing=1, t=0.2, n_angles=24, n_energies=40, flux_quanta=1.5)
    out.append((p, W.noisy_delta(p, 0.24, 0.1, seed=32)))
    p = W.polygon([0.0, 6.0, 7.0, 1.0], [0.0, -1.0, 5.0, 6.0], 0.25, pairing=1, t=0.3,
                  n_angles=12, n_energies=27)
    out.append((p, W.vortex_delta(p, 0.22, [(3.0, 2.5)], [-1], seed=33, rel_noise=0.05)))
    p = W.square(6.0, 24, pairing=0, t=0.8, n_angles=8, n_energies=3)
    out.append((p, W.noisy_delta(p, 0.15, 0.1, seed=34)))
    return out


def _outputs(ctx):
    r = ctx.outputs()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.items()}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("ept", [0, 3, 8])
def test_batch_equals_single_contexts(precision, tol, ept):
    from paper_2205_15000_b300 import sc
    grains = _grains()
    b = sc.Batch([p for p, _ in grains], precision=precision, energies_per_lane=ept)
    singles = [sc.Context(p, precision=precision) for p, _ in grains]
    for (p, d), m, s in zip(grains, b.members, singles):
        m.set_fields(d)
        s.set_fields(d)
    for it in range(3):
        b.sweep()
        for s in singles:
            s.sweep()
        for m, s in zip(b.members, singles):
            rm, rs = _outputs(m), _outputs(s)
            for k in ("delta_new", "j", "F"):
                scale = max(np.max(np.abs(rs[k])), 1e-3)
                assert np.max(np.abs(rm[k] - rs[k])) <= tol * scale, (it, k)
    b.close()


def test_batch_midpoint_equals_single_contexts():
    """A batch with the implicit-midpoint stepper gives what each member's own
    context gives (FP64)."""
    from paper_2205_15000_b300 import sc
    grains = _grains()
    prms = [dict(p, stepper="midpoint") for p, _ in grains]
    b = sc.Batch(prms, precision="fp64", energies_per_lane=8)
    singles = [sc.Context(p, precision="fp64") for p in prms]
    for (_, d), m, s in zip(grains, b.members, singles):
        m.set_fields(d)
        s.set_fields(d)
    for it in range(2):
        b.sweep()
        for s in singles:
            s.sweep()
        for m, s in zip(b.members, singles):
            rm, rs = _outputs(m), _outputs(s)
            for k in ("delta_new", "j", "F"):
                scale = max(np.max(np.abs(rs[k])), 1e-3)
                assert np.max(np.abs(rm[k] - rs[k])) <= 1e-12 * scale, (it, k)
    b.close()


def test_batch_ozaki_matches_oracle_fp64():
    """A batch with Ozaki energy sums: every member equals the oracle's weighted
    sweep (FP64)."""
    from paper_2205_15000_b300 import sc
    grains = _grains()
    prms = [dict(p, energy_sum="ozaki") for p, _ in grains]
    b = sc.Batch(prms, precision="fp64")
    for (_, d), m in zip(grains, b.members):
        m.set_fields(d)
    exits = [None] * len(grains)
    for it in range(2):
        b.sweep()
        for gi, ((_, d), q) in enumerate(zip(grains, prms)):
            o = oracle.OracleGeom(q).full_sweep(d, None, exits[gi])
            exits[gi] = o["exit"]
            r = _outputs(b.members[gi])
            np.testing.assert_allclose(r["delta_new"], o["delta_new"], atol=1e-10, rtol=0)
            np.testing.assert_allclose(r["j"], o["j"], atol=1e-10, rtol=0)
    b.close()


def test_batch_member_matches_oracle_fp64():
    from paper_2205_15000_b300 import sc
    grains = _grains()
    b = sc.Batch([p for p, _ in grains], precision="fp64")
    for (p, d), m in zip(grains, b.members):
        m.set_fields(d)
    exits = [None] * len(grains)
    for it in range(2):
        b.sweep()
        for g, (p, d) in enumerate(grains):
            o = oracle.OracleGeom(p).full_sweep(d, None, exits[g])
            exits[g] = o["exit"]
            r = _outputs(b.members[g])
            np.testing.assert_allclose(r["delta_new"], o["delta_new"], atol=1e-10, rtol=0)
            np.testing.assert_allclose(r["j"], o["j"], atol=1e-10, rtol=0)
    b.close()


def test_batch_graph_run_and_autotune():
    from paper_2205_15000_b300 import sc
    grains = _grains()
    b = sc.Batch([p for p, _ in grains], precision="fp32")
    ref = sc.Batch([p for p, _ in grains], precision="fp32")
    for (p, d), m, mr in zip(grains, b.members, ref.members):
        m.set_fields(d)
        mr.set_fields(d)
    ept = b.autotune()   # two timing sweeps per candidate
    assert 2 <= ept <= 8
    # reference: the same total number of eager sweeps
    n_auto = sum(2 for e in range(2, 9) if max(p["n_energies"] for p, _ in grains) <= 32 * e)
    for _ in range(n_auto):
        ref.sweep()
    b.run(5, with_outputs=True)        # graph replays
    for _ in range(5):
        ref.sweep()
    for m, mr in zip(b.members, ref.members):
        rm, rr = _outputs(m), _outputs(mr)
        scale = np.max(np.abs(rr["delta_new"]))
        assert np.max(np.abs(rm["delta_new"] - rr["delta_new"])) <= 2e-6 * scale
    info = b.info()
    assert info.n_grains == len(grains) and info.energies_per_lane == ept and info.steps_per_sweep > 0
    b.close()
    ref.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_energy_layout_per_member(precision):
    """Each member takes the layout with the fewest padded lane slots (at
    most energies_per_lane energies per lane); one sweep launch per distinct
    energies-per-lane count.  The batch reports the lane steps it executes."""
    from paper_2205_15000_b300 import sc
    grains = _grains()
    ept = 8
    b = sc.Batch([p for p, _ in grains], precision=precision, energies_per_lane=ept)
    expect, counts = 0, set()
    for (p, _), m in zip(grains, b.members):
        L = m.lines()
        steps = int(np.sum(2 * (np.maximum(L["m1"] - L["m0"] + 1, 0) + 1)))
        ne = p["n_energies"]
        slots, lanes = min((l * -(-ne // l), l) for l in (2, 4, 8, 16, 32) if -(-ne // l) <= ept)
        counts.add(slots // lanes)
        expect += steps * slots
    info = b.info()
    assert info.lane_steps_per_sweep == expect
    assert info.sweep_launches == len(counts)
    # FP32: field conversion, rotation, rotate-back (one component count), outputs and
    # final sums around the class launches; FP64: rotate and rotate-back per member
    extra = 5 if precision == "fp32" else 2 + 2 * len(grains)
    assert info.launches_per_iteration == info.sweep_launches + extra
    b.close()


def test_member_sweep_alone_is_rejected():
    from paper_2205_15000_b300 import sc
    grains = _grains()
    b = sc.Batch([p for p, _ in grains[:2]], precision="fp32")
    b.members[0].set_fields(grains[0][1])
    with pytest.raises(sc.ScError) as ei:
        b.members[0].sweep()
    assert ei.value.status == sc.SC_ESTATE
    b.close()


@pytest.mark.parametrize("precision,on_device", [("fp32", True), ("fp32", False), ("fp64", True)])
def test_batch_wide_fields_and_outputs_equal_member_calls(precision, on_device):
    """sc_batch_set_fields / sc_batch_get_outputs (every member's Delta in, every
    member's Delta_new, j, F out, members one after another) give bit for bit what
    the per-member calls give, with device and with host arrays; a two-component
    member carries both planes."""
    import torch
    from paper_2205_15000_b300 import sc
    p1 = W.disc(4.0, 28, pairing=0, t=0.5, n_angles=16, n_energies=10, flux_quanta=0.7)
    p2 = W.diamond(8.0, 30, pairing=1, t=0.3, n_angles=16, n_energies=12, flux_quanta=0.3)
    p3 = W.disc(4.0, 26, pairing=2, t=0.5, n_angles=16, n_energies=8)
    p3["components"] = [(2, 1.0), (1, 1.0)]
    d1 = W.noisy_delta(p1, 0.26, 0.1, seed=71)
    d2 = W.noisy_delta(p2, 0.23, 0.1, seed=72)
    d3 = np.stack([W.noisy_delta(p3, 0.2, 0.1, seed=73), 0.1j * W.noisy_delta(p3, 0.2, 0.1, seed=74)])
    prms, ds = [p1, p2, p3], [d1, d2, d3]
    ref = sc.Batch(prms, precision=precision)
    for m, d in zip(ref.members, ds):
        m.set_fields(d)
    ref.run(2, True)
    want = [m.outputs() for m in ref.members]
    b = sc.Batch(prms, precision=precision)
    flat = np.concatenate([np.ascontiguousarray(d, np.complex128).reshape(-1) for d in ds])
    arr = np.ascontiguousarray(flat.view(np.float64))
    src = torch.from_numpy(arr).cuda() if on_device else arr
    sc.sc_batch_set_fields(b.h, src, on_device)
    b.run(2, True)
    n_c = sum(d.size for d in ds)
    n_p = sum(p["nx"] * p["ny"] for p in prms)
    if on_device:
        dn, j, F = (torch.empty(k, dtype=torch.float64, device="cuda") for k in (2 * n_c, 2 * n_p, n_p))
    else:
        dn, j, F = np.zeros(2 * n_c), np.zeros(2 * n_p), np.zeros(n_p)
    sc.sc_batch_get_outputs(b.h, dn, j, F, on_device)
    torch.cuda.synchronize()
    dn, j, F = ((x.cpu().numpy() if on_device else x) for x in (dn, j, F))
    oc = op = 0
    for w, d, p in zip(want, ds, prms):
        npt = p["nx"] * p["ny"]
        got_dn = dn[2 * oc:2 * (oc + d.size)].view(np.complex128).reshape(d.shape)
        np.testing.assert_array_equal(got_dn, w["delta_new"].cpu().numpy())
        np.testing.assert_array_equal(j[2 * op:2 * (op + npt)].reshape(p["ny"], p["nx"], 2), w["j"].cpu().numpy())
        np.testing.assert_array_equal(F[op:op + npt].reshape(p["ny"], p["nx"]), w["F"].cpu().numpy())
        oc += d.size
        op += npt
    ref.close()
    b.close()


def test_batch_reset_boundary_restarts_from_fresh_values():
    """After sc_batch_reset_boundary two batch iterations give bit for bit the
    outputs of the first two (same fields, same layout, fresh boundary values);
    without the reset they differ (the boundary values were carried over)."""
    from paper_2205_15000_b300 import sc
    grains = _grains()
    b = sc.Batch([p for p, _ in grains], precision="fp32")
    for (p, d), m in zip(grains, b.members):
        m.set_fields(d)
    b.run(2, True)
    first = [_outputs(m)["delta_new"] for m in b.members]
    b.run(2, True)
    carried = [_outputs(m)["delta_new"] for m in b.members]
    b.reset_boundary()
    b.run(2, True)
    again = [_outputs(m)["delta_new"] for m in b.members]
    for x, y in zip(first, again):
        np.testing.assert_array_equal(x, y)
    assert any(np.max(np.abs(x - y)) > 0 for x, y in zip(first, carried))
    b.close()


def test_batch_member_in_two_energy_parts():
    """A member whose 132 energies would pad 16 x 9 lane slots runs as two parts in
    their own layouts (2 x 10 and 16 x 7) whose images are added after the sweep:
    three batch iterations equal the single FP32 context (16 x 9) to FP32 rounding
    and the FP64 oracle within the production tolerances; without parts the batch
    takes the single layout."""
    from paper_2205_15000_b300 import sc
    p = W.disc(3.0, 24, pairing=1, t=0.06, n_angles=16, n_energies=132, flux_quanta=0.4)
    d = W.vortex_delta(p, 0.24, [(0.5, -0.3)], [-1], seed=35, rel_noise=0.05)
    q = W.square(4.0, 20, pairing=0, t=0.5, n_angles=8, n_energies=12)
    dq = W.noisy_delta(q, 0.2, 0.1, seed=36)
    b = sc.Batch([p, q], precision="fp32", energies_per_lane=10)
    assert b.info().split_members == 0  # one layout per member unless asked for
    sc.sc_batch_set_energy_parts(b.h, True)
    info = b.info()
    assert info.split_members == 1 and info.launches_per_iteration == info.sweep_launches + 6
    for m, x in zip(b.members, (d, dq)):
        m.set_fields(x)
    ref = sc.Context(p, precision="fp32")
    ref.set_fields(d)
    g = oracle.OracleGeom(p)
    mk = g.mask().astype(bool)
    ex = None
    for it in range(3):
        b.run(1, True)
        ref.sweep()
        o = g.full_sweep(d, None, ex)
        ex = o["exit"]
        rb, rr = _outputs(b.members[0]), _outputs(ref)
        for k in ("delta_new", "j", "F"):
            scale = np.max(np.abs(rr[k]))
            assert np.max(np.abs(rb[k] - rr[k])) <= 2e-6 * scale, (it, k)
        assert np.max(np.abs(rb["delta_new"][mk] - o["delta_new"][mk])) <= 1e-5 * np.max(np.abs(o["delta_new"][mk]))
        assert np.max(np.abs(rb["j"][mk] - o["j"][mk])) <= 1e-4 * np.max(np.abs(o["j"][mk]))
        assert np.max(np.abs(rb["F"][mk] - o["F"][mk])) <= 1e-4 * np.max(np.abs(o["F"][mk]))
    sc.sc_batch_set_energy_parts(b.h, False)
    assert b.info().split_members == 0
    b.close()
    b64 = sc.Batch([q], precision="fp64")
    with pytest.raises(sc.ScError):
        sc.sc_batch_set_energy_parts(b64.h, True)
    b64.close()


def test_batch_with_ten_energies_per_lane_classes():
    """Ten members whose energy counts (2, 4, ..., 20 on 2 lanes per line) give ten
    energies-per-lane classes, each its own launch with its own work counter: three
    graph-replayed iterations equal the members' single FP32 contexts."""
    from paper_2205_15000_b300 import sc
    prms, ds = [], []
    for k in range(10):
        p = W.disc(2.5 + 0.1 * k, 16 + k, margin=0.2, pairing=k % 2, t=0.3, n_angles=8,
                   n_energies=2 * (k + 1), flux_quanta=0.2)
        prms.append(p)
        ds.append(W.noisy_delta(p, 0.2, 0.1, seed=60 + k))
    b = sc.Batch(prms, precision="fp32", energies_per_lane=10)
    info = b.info()
    assert info.sweep_launches == 10
    assert sorted(info.class_ept[k] for k in range(10)) == list(range(1, 11))
    refs = []
    for p, d, m in zip(prms, ds, b.members):
        m.set_fields(d)
        r = sc.Context(p, precision="fp32")
        r.set_fields(d)
        refs.append(r)
    b.run(3, True)
    for r in refs:
        for _ in range(3):
            r.sweep()
    for m, r in zip(b.members, refs):
        om, orf = _outputs(m), _outputs(r)
        for k in ("delta_new", "j", "F"):
            assert np.max(np.abs(om[k] - orf[k])) <= 2e-6 * np.max(np.abs(orf[k])), k
        r.close()
    b.close()
