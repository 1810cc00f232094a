"""Multi-component order parameters (Eq. order_parameter, Delta(p, R) =
sum_Gamma Delta_Gamma(R) eta_Gamma(p), per-component gap equations with their
own T_c^Gamma) through the C ABI against the oracle: sweeps (FP64 to 1e-10,
FP32 within the production tolerances), the adjoint against central
differences, an accelerated self-consistency loop and the LDOS."""
import numpy as np
import pytest

import oracle
from oracle import accel as oaccel
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "d_plus_is":
        p = W.disc(5.0, 36, pairing=1, t=0.3, n_angles=16, n_energies=8, flux_quanta=0.7, kappa=3.0)
        p["components"] = [(1, 1.0), (0, 0.6)]
        d = W.vortex_delta(p, 0.22, [(1.0, -0.5)], [-1], seed=61, rel_noise=0.05)
        s = 0.05j * W.noisy_delta(p, 1.0, 0.2, seed=62)
        return p, np.stack([d, s])
    if name == "chiral_d":
        p = W.square(10.0, 32, pairing=2, t=0.5, n_angles=16, n_energies=6)
        p["components"] = [(2, 1.0), (1, 1.0)]
        a = W.noisy_delta(p, 0.2, 0.1, seed=63)
        return p, np.stack([a, 1j * W.noisy_delta(p, 0.2, 0.1, seed=64)])
    if name == "three_components":
        p = W.polygon([0.0, 7.0, 9.0, 2.0], [0.0, -1.0, 6.0, 8.0], 0.3, pairing=1, t=0.4, n_angles=12,
                      n_energies=5, flux_quanta=0.5)
        p["components"] = [(1, 1.0), (2, 0.9), (0, 0.5)]
        return p, np.stack([W.noisy_delta(p, a, 0.1, seed=65 + k) for k, a in enumerate((0.2, 0.08, 0.03))])
    raise KeyError(name)


CASES = ["d_plus_is", "chiral_d", "three_components"]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", CASES)
def test_components_sweep_matches_oracle(name, precision):
    from paper_2205_15000_b300 import sc
    p, d = _case(name)
    g = oracle.OracleGeom(p)
    ctx = sc.Context(p, precision=precision)
    ctx.set_fields(d)
    m = g.mask().astype(bool)
    ex = None
    for _ in range(2):
        o = g.full_sweep(d, None, ex)
        ex = o["exit"]
        ctx.sweep()
        r = ctx.outputs()
        dn = r["delta_new"].cpu().numpy()
        assert dn.shape == o["delta_new"].shape
        if precision == "fp64":
            np.testing.assert_allclose(dn, o["delta_new"], atol=1e-10, rtol=0)
            np.testing.assert_allclose(r["j"].cpu().numpy(), o["j"], atol=1e-10, rtol=0)
            np.testing.assert_allclose(r["F"].cpu().numpy(), o["F"], atol=1e-10, rtol=0)
            assert abs(r["eps_G"] - o["eps_G"]) < 1e-9
        else:
            scale = np.max(np.abs(o["delta_new"][:, m]))
            assert np.max(np.abs(dn[:, m] - o["delta_new"][:, m])) < 1e-5 * scale
            assert _rel(r["j"].cpu().numpy()[m], o["j"][m]) < 1e-4
            assert _rel(r["F"].cpu().numpy()[m], o["F"][m]) < 1e-4


def test_components_free_energy_gradient_matches_oracle_fd():
    """dF_total/d(Delta_Gamma(R)) for both components and dF/dA_ind against
    central differences of the oracle (boundary values held fixed)."""
    from paper_2205_15000_b300 import sc
    p, d = _case("d_plus_is")
    a = np.zeros((p["ny"], p["nx"], 2))
    X, Y = W.grid_xy(p)
    a[..., 0] = 0.02 * np.sin(0.4 * X + 0.1 * Y)
    g = oracle.OracleGeom(p)
    ex = None
    for _ in range(200):
        o = g.full_sweep(d, a, ex)
        if ex is not None and np.max(np.abs(o["exit"] - ex)) < 1e-13:
            break
        ex = o["exit"]
    rng = np.random.default_rng(71)
    m = g.mask().astype(bool)
    idx = np.argwhere(m & (np.hypot(X, Y) < 3.5))
    probes = idx[rng.choice(len(idx), 5, replace=False)]
    hstep = 1e-5
    ctx = sc.Context(p, precision="fp64")
    ctx.set_fields(d, a)
    sc.sc_burnin(ctx.h, 300, 1e-13)
    ctx.sweep()
    gd, ga = ctx.adjoint(g_Ftotal=1.0)
    gd, ga = gd.cpu().numpy(), ga.cpu().numpy()
    err, scale = 0.0, 0.0
    for (j, i) in probes:
        for comp in range(2):
            for part in (1.0, 1j):
                dp, dm = d.copy(), d.copy()
                dp[comp, j, i] += part * hstep
                dm[comp, j, i] -= part * hstep
                fd = (g.full_sweep(dp, a, ex)["F_total"] - g.full_sweep(dm, a, ex)["F_total"]) / (2 * hstep)
                adj = gd[comp, j, i].real if part == 1.0 else gd[comp, j, i].imag
                err = max(err, abs(adj - fd))
                scale = max(scale, abs(fd))
        ap, am = a.copy(), a.copy()
        ap[j, i, 0] += hstep
        am[j, i, 0] -= hstep
        fd = (g.full_sweep(d, ap, ex)["F_total"] - g.full_sweep(d, am, ex)["F_total"]) / (2 * hstep)
        err = max(err, abs(ga[j, i, 0] - fd))
    assert scale > 0 and err <= 1e-6 * scale, err / scale


def test_components_accelerated_loop_matches_oracle():
    from paper_2205_15000_b300 import sc
    p, d = _case("d_plus_is")
    n_iter = 5
    g = oracle.OracleGeom(p)
    ref = g.self_consistency(d, n_iter, oaccel.default_params("congacc"))
    ctx = sc.Context(p, precision="fp64")
    ctx.set_fields(d)
    hist = []
    prm = sc.accel_params("congacc")
    for _ in range(n_iter):
        ctx.sweep()
        hist.append(ctx.outputs()["eps_G"])
        ctx.accelerate(prm)
    np.testing.assert_allclose(hist, ref["history"], rtol=1e-9, atol=1e-12)
    it, alpha, w = sc.sc_accel_get_state(ctx.h)
    nc = len(ref["accelerator"].alpha_c)
    assert nc == 6
    np.testing.assert_allclose(alpha[:nc], ref["accelerator"].alpha_c, rtol=1e-9)


def test_components_ldos_matches_oracle():
    from paper_2205_15000_b300 import sc
    p, d = _case("chiral_d")
    e = np.linspace(-0.3, 0.3, 6)
    g = oracle.OracleGeom(p)
    acc, _ = g.ldos(d, None, e, 0.04, n_burnin=6, tol=0.0)
    ctx = sc.Context(p, precision="fp64")
    ctx.set_fields(d)
    out = ctx.ldos(e, 0.04, n_burnin=6).cpu().numpy()
    m = g.mask().astype(bool)
    for c in range(len(e)):
        assert _rel(out[c][m], acc[c][m]) < 1e-9
