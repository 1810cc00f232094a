"""FP32 batches whose sweep launches also run the members' lattice transfers
(rotation and rotate-back, Sec. 3.1) as work items: every member's images,
Delta_new, j and F are bit for bit those of the batch that runs the transfers
in launches of their own, sweep after sweep and under graph replay, with mixed
energy counts (several launch classes), gauges, a two-component member (whose
rotate-back stays in its own launch), both steppers, Ozaki sums and members in
two energy parts."""
import numpy as np
import pytest

from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _grains():
    out = []
    p = W.disc(4.0, 28, pairing=0, t=0.5, n_angles=16, n_energies=10, flux_quanta=0.7)
    out.append((p, W.noisy_delta(p, 0.26, 0.1, seed=41)))
    p = W.diamond(9.0, 36, pairing=1, t=0.2, n_angles=24, n_energies=40, flux_quanta=1.5)
    out.append((p, W.noisy_delta(p, 0.24, 0.1, seed=42)))
    p = W.polygon([0.0, 6.0, 7.0, 1.0], [0.0, -1.0, 5.0, 6.0], 0.25, pairing=1, t=0.3,
                  n_angles=12, n_energies=27)
    out.append((p, W.vortex_delta(p, 0.22, [(3.0, 2.5)], [-1], seed=43, rel_noise=0.05)))
    p = W.square(6.0, 24, pairing=0, t=0.8, n_angles=8, n_energies=3)
    out.append((p, W.noisy_delta(p, 0.15, 0.1, seed=44)))
    p = W.disc(5.0, 32, pairing=1, t=0.3, n_angles=20, n_energies=17, gauge="landau", flux_quanta=0.9)
    out.append((p, W.noisy_delta(p, 0.2, 0.1, seed=45)))
    p = W.annulus(5.0, 2.0, 40, margin=0.3, pairing=2, t=0.4, n_angles=16, n_energies=5, gauge="solenoid",
                  flux_quanta=0.7)
    p["components"] = [(2, 1.0), (1, 0.9)]
    X, Y = W.grid_xy(p)
    ph = np.exp(-1j * np.arctan2(Y, X))
    out.append((p, np.stack([0.15 * ph, 0.15j * ph])))
    p = W.diamond(12.0, 48, pairing=1, t=0.1, n_angles=32, n_energies=132, flux_quanta=0.5)
    out.append((p, W.noisy_delta(p, 0.24, 0.05, seed=46)))
    return out


def _state(b):
    res = []
    for m in b.members:
        r = {k: (v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)) for k, v in m.outputs().items()}
        r["images"] = np.asarray(m.images())
        res.append(r)
    return res


def _run(prms, deltas, fused, split, sweeps, graph):
    from paper_2205_15000_b300 import sc
    b = sc.Batch(prms, precision="fp32", energies_per_lane=10)
    if split:
        sc.sc_batch_set_energy_parts(b.h, 1)
    b.set_fused_transfers(fused)
    info = b.info()
    for m, d in zip(b.members, deltas):
        m.set_fields(d)
    states = []
    for _ in range(sweeps):
        b.sweep()
        states.append(_state(b))
    if graph:
        b.run(3, with_outputs=True)
        states.append(_state(b))
    b.close()
    return info, states


@pytest.mark.parametrize("stepper,energy_sum,split", [
    ("closed", "matsubara", False),
    ("closed", "matsubara", True),
    ("midpoint", "matsubara", False),
    ("closed", "ozaki", False),
])
def test_fused_transfers_bitwise_equal(stepper, energy_sum, split):
    grains = _grains()
    prms = [dict(p, stepper=stepper, energy_sum=energy_sum) for p, _ in grains]
    deltas = [d for _, d in grains]
    info_on, on = _run(prms, deltas, True, split, 3, True)
    info_off, off = _run(prms, deltas, False, split, 3, True)
    assert info_on.fused_transfers == 1 and info_on.transfer_items > 0
    assert info_off.fused_transfers == 0 and info_off.transfer_items == 0
    assert info_on.sweep_launches >= 2
    for it, (a, c) in enumerate(zip(on, off)):
        for g, (ra, rc) in enumerate(zip(a, c)):
            for k in ("images", "delta_new", "j", "F"):
                assert np.array_equal(ra[k], rc[k]), (it, g, k)
            assert np.isfinite(ra["delta_new"]).all()


def test_autotuned_blocks_per_sm_follow_their_class():
    """The autotune's blocks per SM belong to an energies-per-lane class, not to a
    launch position: switching the transfer layout afterwards (which reorders the
    launches) keeps each class's choice."""
    from paper_2205_15000_b300 import sc
    grains = _grains()
    b = sc.Batch([p for p, _ in grains], precision="fp32")
    for m, (_, d) in zip(b.members, grains):
        m.set_fields(d)
    b.autotune()

    def per_class(i):
        return {i.class_ept[k]: i.class_blocks_per_sm[k] for k in range(i.sweep_launches)}

    ref = per_class(b.info())
    for fused in (True, False, True):
        b.set_fused_transfers(fused)
        got = per_class(b.info())
        assert got == ref, (fused, got, ref)
    b.sweep()
    assert np.isfinite(b.members[0].outputs()["delta_new"].cpu().numpy()).all()
    b.close()


def test_transfer_items_only_where_the_layout_allows():
    """The fused layout needs two or more launch classes and no member in energy
    blocks; otherwise the transfers stay in launches of their own (and the
    results equal the separate layout's).  FP64 batches refuse it."""
    from paper_2205_15000_b300 import sc
    grains = _grains()
    # one class: two members with the same energies-per-lane count
    one = [grains[0], (dict(grains[0][0]), W.noisy_delta(grains[0][0], 0.26, 0.1, seed=47))]
    b = sc.Batch([p for p, _ in one], precision="fp32", energies_per_lane=10)
    b.set_fused_transfers(True)
    i = b.info()
    assert i.sweep_launches == 1 and i.fused_transfers == 0 and i.transfer_items == 0
    b.close()
    # a member whose 700 energies exceed one layout (three energy blocks)
    p = W.disc(3.0, 24, pairing=1, t=0.02, n_angles=8, n_energies=700, flux_quanta=0.4)
    blk = [grains[0], grains[1], (p, W.vortex_delta(p, 0.24, [(0.5, -0.3)], [-1], seed=48, rel_noise=0.05))]
    res = []
    for fused in (True, False):
        b = sc.Batch([q for q, _ in blk], precision="fp32", energies_per_lane=10)
        b.set_fused_transfers(fused)
        i = b.info()
        assert i.sweep_launches >= 2 and i.fused_transfers == 0
        for m, (_, d) in zip(b.members, blk):
            m.set_fields(d)
        b.sweep()
        b.sweep()
        res.append(_state(b))
        b.close()
    for ra, rc in zip(*res):
        for k in ("images", "delta_new", "j", "F"):
            assert np.array_equal(ra[k], rc[k]), k
    b = sc.Batch([q for q, _ in grains[:2]], precision="fp64")
    with pytest.raises(sc.ScError) as ei:
        b.set_fused_transfers(True)
    assert ei.value.status == sc.SC_EINVAL
    b.close()
