"""More energies than one lane layout holds (32 lanes x 8 energies per lane):
the work list carries one item per (line group, energy block); each block writes
its energy sums into its own image and the images are added in block order.  Sweeps, Ozaki sums, the
adjoint and the batch against the oracle, which has no such limit; the LDOS,
whose gamma~ at eps comes from gamma at -eps in the same warp, refuses more
than one block."""
import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _grain(n_e=300, **kw):
    kw.setdefault("pairing", 1)
    p = W.disc(3.0, 24, t=0.02, n_angles=8, n_energies=n_e, flux_quanta=0.4, **kw)
    d = W.vortex_delta(p, 0.24, [(0.5, -0.3)], [-1], seed=61, rel_noise=0.05)
    return p, d


def _outputs(ctx):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ctx.outputs().items()}


@pytest.mark.parametrize("energy_sum", ["matsubara", "ozaki"])
def test_blocked_sweep_matches_oracle(energy_sum):
    from paper_2205_15000_b300 import sc
    p, d = _grain()
    p["energy_sum"] = energy_sum
    g = oracle.OracleGeom(p)
    m = g.mask().astype(bool)
    for precision, tol in (("fp64", 1e-10), ("fp32", None)):
        ctx = sc.Context(p, precision=precision)
        ctx.set_fields(d)
        ex = None
        for _ in range(2):
            o = g.full_sweep(d, None, ex)
            ex = o["exit"]
            ctx.sweep()
            r = _outputs(ctx)
            if tol is not None:
                np.testing.assert_allclose(ctx.exits(), o["exit"][0], atol=tol, rtol=0)
                for k in ("delta_new", "j", "F"):
                    np.testing.assert_allclose(r[k], o[k], atol=tol, rtol=0)
            else:
                assert np.max(np.abs(r["delta_new"][m] - o["delta_new"][m])) < 1e-5 * np.max(np.abs(o["delta_new"][m]))
                assert np.max(np.abs(r["F"][m] - o["F"][m])) < 1e-4 * np.max(np.abs(o["F"][m]))


def test_blocked_adjoint_matches_oracle_fd():
    from paper_2205_15000_b300 import sc
    p, d = _grain()
    X, Y = W.grid_xy(p)
    a = np.stack([0.02 * np.sin(0.4 * X), -0.015 * np.cos(0.3 * Y)], axis=-1)
    g = oracle.OracleGeom(p)
    ex = None
    for _ in range(200):
        o = g.full_sweep(d, a, ex)
        done = ex is not None and np.max(np.abs(o["exit"] - ex)) < 1e-13
        ex = o["exit"]
        if done:
            break
    m = g.mask().astype(bool)
    rng = np.random.default_rng(62)
    idx = np.argwhere(m)
    probes = idx[rng.choice(len(idx), 6, replace=False)]
    hh = 1e-5
    fd = []
    for (j, i) in probes:
        row = []
        for comp in range(4):
            vals = []
            for s in (+1, -1):
                dd, aa = d.copy(), a.copy()
                if comp == 0:
                    dd[j, i] += s * hh
                elif comp == 1:
                    dd[j, i] += s * 1j * hh
                else:
                    aa[j, i, comp - 2] += s * hh
                vals.append(g.full_sweep(dd, aa, ex)["F_total"])
            row.append((vals[0] - vals[1]) / (2 * hh))
        fd.append(row)
    fd = np.array(fd)
    ctx = sc.Context(p, precision="fp64")
    ctx.set_fields(d, a)
    sc.sc_burnin(ctx.h, 300, 1e-13)
    ctx.sweep()
    gd, ga = ctx.adjoint(g_Ftotal=1.0)
    gd, ga = gd.cpu().numpy(), ga.cpu().numpy()
    adj = np.array([[gd[j, i].real, gd[j, i].imag, ga[j, i, 0], ga[j, i, 1]] for j, i in probes])
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(adj - fd)) <= 1e-6 * scale, np.max(np.abs(adj - fd)) / scale


def test_batch_with_a_blocked_member_equals_single_contexts():
    from paper_2205_15000_b300 import sc
    p1, d1 = _grain()
    p2 = W.disc(4.0, 28, pairing=0, t=0.5, n_angles=16, n_energies=10, flux_quanta=0.7)
    d2 = W.noisy_delta(p2, 0.26, 0.1, seed=63)
    grains = [(p1, d1), (p2, d2)]
    b = sc.Batch([q for q, _ in grains], precision="fp64")
    singles = [sc.Context(q, precision="fp64") for q, _ in grains]
    for (q, d), mb, s in zip(grains, b.members, singles):
        mb.set_fields(d)
        s.set_fields(d)
    for _ in range(2):
        b.sweep()
        for s in singles:
            s.sweep()
        for mb, s in zip(b.members, singles):
            rm, rs = _outputs(mb), _outputs(s)
            for k in ("delta_new", "j", "F"):
                scale = max(np.max(np.abs(rs[k])), 1e-3)
                assert np.max(np.abs(rm[k] - rs[k])) <= 1e-12 * scale
    b.close()


def test_ldos_refuses_more_than_one_block():
    from paper_2205_15000_b300 import sc
    p, d = _grain(n_e=4)
    ctx = sc.Context(p, precision="fp32")
    ctx.set_fields(d)
    with pytest.raises(sc.ScError):
        ctx.ldos(np.linspace(-0.3, 0.3, 300), 0.02)


def test_blocked_images_do_not_depend_on_scheduling():
    """700 energies take three blocks of 32 x 8: the sample images of two
    contexts swept from the same inputs are bit for bit equal (the blocks'
    images are added in a fixed order, not by atomics in the order the work
    items happen to finish), and the outputs match the oracle."""
    from paper_2205_15000_b300 import sc
    p, d = _grain(n_e=700)
    g = oracle.OracleGeom(p)
    m = g.mask().astype(bool)
    o = g.full_sweep(d, None, None)
    imgs = []
    for _ in range(2):
        ctx = sc.Context(p, precision="fp32")
        ctx.set_fields(d)
        ctx.sweep()
        imgs.append(ctx.images())
        r = _outputs(ctx)
        assert np.max(np.abs(r["delta_new"][m] - o["delta_new"][m])) < 1e-5 * np.max(np.abs(o["delta_new"][m]))
        ctx.close()
    np.testing.assert_array_equal(imgs[0], imgs[1])
