"""Parity of the CUDA path with the FP64 oracle on composite grains (Sec. 4
and App. B: discs and convex polygons added and removed in order; lattice
lines with several chords, boundary links through holes) and in the three
gauges (symmetric, landau, solenoid; Eq. solenoid_gauge).

FP64: images, exits and outputs within 1e-10; FP32: Delta_new within 1e-5,
j and F within 1e-4 relative to the oracle's maximum, as for convex grains."""
import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL_DELTA, TOL_J, TOL_F = 1e-5, 1e-4, 1e-4
J_FLOOR = 1e-6


def _smooth_a(p, amp):
    X, Y = W.grid_xy(p)
    return np.stack([amp * np.sin(0.3 * X + 0.2 * Y), -amp * np.cos(0.25 * Y - 0.15 * X)], axis=-1)


def case(name):
    if name == "annulus_s_solenoid":
        p = W.annulus(6.0, 2.5, 48, margin=0.3, pairing=0, t=0.5, n_angles=16, n_energies=6,
                      gauge="solenoid", flux_quanta=-0.7)
        X, Y = W.grid_xy(p)
        d = 0.26 * np.exp(1j * np.arctan2(Y, X)) * (1 + 0.05 * W.noisy_delta(p, 1.0, 1.0, seed=71))
        return p, d, None
    if name == "annulus_d_symmetric":
        p = W.annulus(7.0, 3.0, 56, margin=0.3, pairing=1, t=0.3, n_angles=20, n_energies=9,
                      flux_quanta=1.3)
        return p, W.noisy_delta(p, 0.23, 0.1, seed=72), _smooth_a(p, 0.02)
    if name == "square_hole_landau":
        vx, vy = W.regular_polygon((2.5, 0.5), 4, 3.0, rotation=0.07)
        p = W.composite([W.disc_part((0, 0), 6.0), W.polygon_part(vx, vy, add=False)], 0.25, pairing=2,
                        t=0.4, n_angles=12, n_energies=5, gauge="landau", flux_quanta=0.9,
                        crystal_rotation=0.1, charge_sign=1)
        return p, W.noisy_delta(p, 0.2, 0.1, seed=73), _smooth_a(p, 0.015)
    if name == "squid":
        vx, vy = W.regular_polygon((20.0, 0.0), 8, 6.0)
        p = W.composite([W.polygon_part([0, 40, 40, 0], [-2, -2, 2, 2]), W.polygon_part(vx, vy),
                         W.disc_part((20.0, 0.0), 3.5, add=False)], 0.4, pairing=0, t=0.5,
                        n_angles=16, n_energies=4, flux_quanta=2.0)
        return p, W.noisy_delta(p, 0.26, 0.1, seed=74), None
    if name == "two_discs_landau":
        p = W.composite([W.disc_part((0, 0), 4.0), W.disc_part((5.0, 1.0), 3.0)], 0.25, pairing=1, t=0.3,
                        n_angles=18, n_energies=7, gauge="landau", flux_quanta=1.1)
        return p, W.vortex_delta(p, 0.22, [(0.5, 0.0)], [-1], seed=75, rel_noise=0.05), None
    raise KeyError(name)


CASES = ["annulus_s_solenoid", "annulus_d_symmetric", "square_hole_landau", "squid", "two_discs_landau"]


def _rel(a, b, floor=0.0):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor, 1e-300))


def _run_both(p, delta, aind, precision, n_sweeps=3):
    from paper_2205_15000_b300 import sc
    g = oracle.OracleGeom(p)
    ctx = sc.Context(p, precision=precision)
    ctx.set_fields(delta, aind)
    ex = None
    res = []
    for _ in range(n_sweeps):
        o = g.full_sweep(delta, aind, ex)
        ex = o["exit"]
        ctx.sweep()
        r = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ctx.outputs().items()}
        res.append(dict(o=o, r=r, exits=ctx.exits(), images=ctx.images()))
    return g, g.mask().astype(bool), res


@pytest.mark.parametrize("stepper", ["closed", "midpoint"])
@pytest.mark.parametrize("name", CASES)
def test_fp64_composite_matches_oracle(name, stepper):
    p, delta, aind = case(name)
    p["stepper"] = stepper
    g, m, res = _run_both(p, delta, aind, "fp64")
    for R in res:
        o, r = R["o"], R["r"]
        np.testing.assert_allclose(R["images"], o["images"][: g.n_samples_all // 2], atol=TOL64, rtol=0)
        np.testing.assert_allclose(R["exits"], o["exit"][0], atol=TOL64, rtol=0)
        np.testing.assert_allclose(r["delta_new"], o["delta_new"], atol=TOL64, rtol=0)
        np.testing.assert_allclose(r["j"], o["j"], atol=TOL64, rtol=0)
        np.testing.assert_allclose(r["F"], o["F"], atol=TOL64, rtol=0)
        assert abs(r["F_total"] - o["F_total"]) < TOL64


@pytest.mark.parametrize("name", CASES)
def test_fp32_composite_within_tolerance(name):
    p, delta, aind = case(name)
    g, m, res = _run_both(p, delta, aind, "fp32")
    for R in res:
        o, r = R["o"], R["r"]
        assert _rel(r["delta_new"][m], o["delta_new"][m]) < TOL_DELTA
        assert _rel(r["j"][m], o["j"][m], J_FLOOR) < TOL_J
        assert _rel(r["F"][m], o["F"][m]) < TOL_F
        assert np.max(np.abs(R["exits"] - o["exit"][0])) < 2e-5


def test_solenoid_matching_flux_carries_no_current_on_the_gpu():
    """The paper's flux-quantisation check through the CUDA path: with
    alpha = -1 and one phase winding the superflow vanishes (Sec. 5.1.1), and
    the FP32 sweep gives the oracle's small residual current."""
    from paper_2205_15000_b300 import sc
    p = W.annulus(6.0, 2.5, 64, margin=0.3, pairing=0, t=0.5, n_angles=16, n_energies=6, gauge="solenoid",
                  flux_quanta=-1.0)
    X, Y = W.grid_xy(p)
    db = oracle.bulk_gap(0, 0.5, 6, 16)
    d = db * np.exp(1j * np.arctan2(Y, X))
    g = oracle.OracleGeom(p)
    ex = None
    for _ in range(10):
        o = g.full_sweep(d, None, ex)
        ex = o["exit"]
    ctx = sc.Context(p, precision="fp32")
    ctx.set_fields(d)
    for _ in range(10):
        ctx.sweep()
    r = ctx.outputs()
    j = r["j"].cpu().numpy()
    m = g.mask().astype(bool)
    assert np.max(np.abs(j[m] - o["j"][m])) < 2e-5
    eps = 0.5 * (np.arange(6) + 0.5)
    Y = 0.5 * float(np.sum(db * db / (eps * eps + db * db) ** 1.5))   # Yosida function (Eq. linearcurrent)
    assert np.max(np.abs(j[m])) < 0.25 * Y / (2 * 6.0)   # far below one unmatched quantum's current


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
def test_ldos_on_an_annulus_matches_oracle(precision, tol):
    from paper_2205_15000_b300 import sc
    p = W.annulus(5.0, 2.0, 40, margin=0.3, pairing=1, t=0.5, n_angles=16, n_energies=1, gauge="solenoid",
                  flux_quanta=0.4)
    d = W.noisy_delta(p, 0.22, 0.05, seed=76)
    e = np.linspace(-0.3, 0.3, 8)
    g = oracle.OracleGeom(p)
    acc, _ = g.ldos(d, None, e, 0.03, n_burnin=6, tol=0.0)
    ctx = sc.Context(p, precision=precision)
    ctx.set_fields(d)
    out = ctx.ldos(e, 0.03, n_burnin=6).cpu().numpy()
    m = g.mask().astype(bool)
    for c in range(len(e)):
        assert _rel(out[c][m], acc[c][m]) < tol, c


def test_adjoint_on_an_annulus_matches_oracle_fd():
    """d F_total / d(Delta, A_ind) through holes and the solenoid gauge:
    the adjoint sweep against central differences of the oracle, boundary
    values held at their burnt-in values on both sides."""
    from paper_2205_15000_b300 import sc
    p = W.annulus(5.0, 2.0, 36, margin=0.3, pairing=1, t=0.3, n_angles=16, n_energies=6, gauge="solenoid",
                  flux_quanta=0.6)
    X, Y = W.grid_xy(p)
    d = 0.22 * np.exp(-1j * np.arctan2(Y, X)) * (1 + 0.1 * W.noisy_delta(p, 1.0, 1.0, seed=77))
    a = _smooth_a(p, 0.02)
    g = oracle.OracleGeom(p)
    ex = None
    for _ in range(300):
        o = g.full_sweep(d, a, ex)
        done = ex is not None and np.max(np.abs(o["exit"] - ex)) < 1e-13
        ex = o["exit"]
        if done:
            break
    m = g.mask().astype(bool)
    rng = np.random.default_rng(78)
    idx = np.argwhere(m)
    probes = idx[rng.choice(len(idx), 10, replace=False)]
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
    assert scale > 0
    assert np.max(np.abs(adj - fd)) <= 1e-6 * scale, np.max(np.abs(adj - fd)) / scale


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_batch_with_composite_members_equals_single_contexts(precision, tol):
    from paper_2205_15000_b300 import sc
    grains = [case(n)[:2] for n in ("annulus_s_solenoid", "square_hole_landau", "squid")]
    p = W.disc(4.0, 28, pairing=0, t=0.5, n_angles=16, n_energies=10, flux_quanta=0.7)
    grains.append((p, W.noisy_delta(p, 0.26, 0.1, seed=79)))
    b = sc.Batch([q for q, _ in grains], precision=precision)
    singles = [sc.Context(q, precision=precision) for q, _ in grains]
    for (q, d), mb, s in zip(grains, b.members, singles):
        mb.set_fields(d)
        s.set_fields(d)
    for it in range(2):
        b.sweep()
        for s in singles:
            s.sweep()
        for mb, s in zip(b.members, singles):
            rm = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in mb.outputs().items()}
            rs = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in s.outputs().items()}
            for k in ("delta_new", "j", "F"):
                scale = max(np.max(np.abs(rs[k])), 1e-3)
                assert np.max(np.abs(rm[k] - rs[k])) <= tol * scale, (it, k)
    b.close()


def test_options_compose_fp64():
    """Every option at once -- two order-parameter components (chiral
    d_xy + i d_x2-y2), Ozaki sums, the implicit midpoint stepper, an annulus
    and the solenoid gauge with an induced field -- against the oracle to 1e-10."""
    p = W.annulus(5.0, 2.0, 40, margin=0.3, pairing=2, t=0.4, n_angles=16, n_energies=5, gauge="solenoid",
                  flux_quanta=0.7, charge_sign=-1)
    p["components"] = [(2, 1.0), (1, 0.9)]
    p["energy_sum"] = "ozaki"
    p["stepper"] = "midpoint"
    X, Y = W.grid_xy(p)
    d = np.stack([0.15 * np.exp(-1j * np.arctan2(Y, X)), 0.15j * np.exp(-1j * np.arctan2(Y, X))])
    d = d * (1 + 0.05 * W.noisy_delta(p, 1.0, 1.0, seed=80))
    g, m, res = _run_both(p, d, _smooth_a(p, 0.02), "fp64", n_sweeps=2)
    for R in res:
        o, r = R["o"], R["r"]
        np.testing.assert_allclose(R["exits"], o["exit"][0], atol=TOL64, rtol=0)
        np.testing.assert_allclose(r["delta_new"], o["delta_new"], atol=TOL64, rtol=0)
        np.testing.assert_allclose(r["j"], o["j"], atol=TOL64, rtol=0)
        np.testing.assert_allclose(r["F"], o["F"], atol=TOL64, rtol=0)


def test_batch_mixes_components_and_gauges():
    """Batch members may differ in components, gauge and geometry: each equals
    its own context (FP64)."""
    from paper_2205_15000_b300 import sc
    q1 = W.annulus(5.0, 2.0, 40, margin=0.3, pairing=2, t=0.4, n_angles=16, n_energies=5, gauge="solenoid",
                   flux_quanta=0.7)
    q1["components"] = [(2, 1.0), (1, 0.9)]
    X, Y = W.grid_xy(q1)
    d1 = np.stack([0.15 * np.exp(-1j * np.arctan2(Y, X)), 0.15j * np.exp(-1j * np.arctan2(Y, X))])
    q2, d2, _ = case("two_discs_landau")
    q3 = W.disc(4.0, 28, pairing=0, t=0.5, n_angles=16, n_energies=10, flux_quanta=0.7)
    d3 = W.noisy_delta(q3, 0.26, 0.1, seed=81)
    grains = [(q1, d1), (q2, d2), (q3, d3)]
    b = sc.Batch([q for q, _ in grains], precision="fp64")
    singles = [sc.Context(q, precision="fp64") for q, _ in grains]
    for (q, d), mb, s in zip(grains, b.members, singles):
        mb.set_fields(d)
        s.set_fields(d)
    for it in range(2):
        b.sweep()
        for s in singles:
            s.sweep()
        for mb, s in zip(b.members, singles):
            rm = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in mb.outputs().items()}
            rs = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in s.outputs().items()}
            for k in ("delta_new", "j", "F"):
                scale = max(np.max(np.abs(rs[k])), 1e-3)
                assert np.max(np.abs(rm[k] - rs[k])) <= 1e-12 * scale, (it, k)
    b.close()
