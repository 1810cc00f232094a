"""Adjoint sweep: d(loss)/d(Delta(R), A_ind(R)) through the C ABI against
central finite differences of the FP64 oracle, with the boundary entry values
(converged by burn-in at the evaluation point) held fixed on both sides.

Gradients are taken at a non-self-consistent Delta (a vortex plus noise): at
self-consistency dF/dDelta vanishes (stationarity of the functional)."""
import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _grain(kappa=0.0):
    p = W.disc(5.0, 32, pairing=1, t=0.3, n_angles=16, n_energies=8, flux_quanta=0.6, kappa=kappa)
    d = W.vortex_delta(p, 0.22, [(1.0, 0.5)], [-1], seed=41, rel_noise=0.1)
    X, Y = W.grid_xy(p)
    a = np.stack([0.02 * np.sin(0.4 * X + 0.1 * Y), -0.015 * np.cos(0.3 * Y - 0.2 * X)], axis=-1)
    return p, d, a


def _oracle_converged_exits(g, d, a, n=200, tol=1e-13):
    ex = None
    for _ in range(n):
        o = g.full_sweep(d, a, ex)
        if ex is not None and np.max(np.abs(o["exit"] - ex)) < tol:
            return o["exit"]
        ex = o["exit"]
    return ex


def _probes(p, g, n, seed):
    rng = np.random.default_rng(seed)
    m = g.mask().astype(bool)
    X, Y = W.grid_xy(p)
    idx = np.argwhere(m & (np.hypot(X, Y) < 4.0))
    return idx[rng.choice(len(idx), n, replace=False)]


def _fd(loss, d, a, probes, h=1e-5):
    out = []
    for (j, i) in probes:
        row = []
        for comp in range(4):
            vals = []
            for s in (+1, -1):
                dd, aa = d.copy(), a.copy()
                if comp == 0:
                    dd[j, i] += s * h
                elif comp == 1:
                    dd[j, i] += s * 1j * h
                else:
                    aa[j, i, comp - 2] += s * h
                vals.append(loss(dd, aa))
            row.append((vals[0] - vals[1]) / (2 * h))
        out.append(row)
    return np.array(out)


def _adjoint(p, d, a, precision, **cot):
    from paper_2205_15000_b300 import sc
    ctx = sc.Context(p, precision=precision)
    ctx.set_fields(d, a)
    sc.sc_burnin(ctx.h, 300, 1e-13 if precision == "fp64" else 1e-6)
    ctx.sweep()
    gd, ga = ctx.adjoint(**cot)
    return gd.cpu().numpy(), ga.cpu().numpy()


@pytest.mark.parametrize("kappa", [0.0, 3.0])
def test_free_energy_gradient_matches_oracle_fd(kappa):
    p, d, a = _grain(kappa)
    g = oracle.OracleGeom(p)
    ex = _oracle_converged_exits(g, d, a)
    loss = lambda dd, aa: g.full_sweep(dd, aa, ex)["F_total"]  # noqa: E731
    probes = _probes(p, g, 10, 42)
    fd = _fd(loss, d, a, probes)
    gd, ga = _adjoint(p, d, a, "fp64", g_Ftotal=1.0)
    adj = np.array([[gd[j, i].real, gd[j, i].imag, ga[j, i, 0], ga[j, i, 1]] for j, i in probes])
    scale = np.max(np.abs(fd))
    assert scale > 0
    assert np.max(np.abs(adj - fd)) <= 1e-6 * scale, np.max(np.abs(adj - fd)) / scale


def test_midpoint_free_energy_gradient_matches_oracle_fd():
    """The adjoint of the implicit-midpoint sweep (App. C) against central
    differences of the oracle's midpoint sweep."""
    p, d, a = _grain()
    p["stepper"] = "midpoint"
    g = oracle.OracleGeom(p)
    ex = _oracle_converged_exits(g, d, a)
    loss = lambda dd, aa: g.full_sweep(dd, aa, ex)["F_total"]  # noqa: E731
    probes = _probes(p, g, 8, 46)
    fd = _fd(loss, d, a, probes)
    gd, ga = _adjoint(p, d, a, "fp64", g_Ftotal=1.0)
    adj = np.array([[gd[j, i].real, gd[j, i].imag, ga[j, i, 0], ga[j, i, 1]] for j, i in probes])
    scale = np.max(np.abs(fd))
    assert scale > 0
    assert np.max(np.abs(adj - fd)) <= 1e-6 * scale, np.max(np.abs(adj - fd)) / scale


def test_ozaki_free_energy_gradient_matches_oracle_fd():
    """The adjoint with Ozaki-weighted energy sums against central differences
    of the oracle's weighted sweep."""
    p, d, a = _grain()
    p["energy_sum"] = "ozaki"
    g = oracle.OracleGeom(p)
    ex = _oracle_converged_exits(g, d, a)
    loss = lambda dd, aa: g.full_sweep(dd, aa, ex)["F_total"]  # noqa: E731
    probes = _probes(p, g, 8, 47)
    fd = _fd(loss, d, a, probes)
    gd, ga = _adjoint(p, d, a, "fp64", g_Ftotal=1.0)
    adj = np.array([[gd[j, i].real, gd[j, i].imag, ga[j, i, 0], ga[j, i, 1]] for j, i in probes])
    scale = np.max(np.abs(fd))
    assert scale > 0
    assert np.max(np.abs(adj - fd)) <= 1e-6 * scale, np.max(np.abs(adj - fd)) / scale


def test_output_cotangent_gradient_matches_oracle_fd():
    p, d, a = _grain()
    g = oracle.OracleGeom(p)
    ex = _oracle_converged_exits(g, d, a)
    rng = np.random.default_rng(7)
    c1 = rng.standard_normal((p["ny"], p["nx"])) + 1j * rng.standard_normal((p["ny"], p["nx"]))
    c2 = rng.standard_normal((p["ny"], p["nx"], 2))
    c3 = rng.standard_normal((p["ny"], p["nx"]))

    def loss(dd, aa):
        o = g.full_sweep(dd, aa, ex)
        return (np.sum(c1.real * o["delta_new"].real + c1.imag * o["delta_new"].imag)
                + np.sum(c2 * o["j"]) + np.sum(c3 * o["F"]))
    probes = _probes(p, g, 8, 43)
    fd = _fd(loss, d, a, probes)
    gd, ga = _adjoint(p, d, a, "fp64", g_delta_new=c1, g_j=c2, g_F=c3)
    adj = np.array([[gd[j, i].real, gd[j, i].imag, ga[j, i, 0], ga[j, i, 1]] for j, i in probes])
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(adj - fd)) <= 1e-6 * scale, np.max(np.abs(adj - fd)) / scale


def test_fp32_adjoint_close_to_fp64():
    p, d, a = _grain()
    gd64, ga64 = _adjoint(p, d, a, "fp64", g_Ftotal=1.0)
    gd32, ga32 = _adjoint(p, d, a, "fp32", g_Ftotal=1.0)
    assert np.max(np.abs(gd32 - gd64)) <= 1e-3 * np.max(np.abs(gd64))
    assert np.max(np.abs(ga32 - ga64)) <= 1e-3 * np.max(np.abs(ga64))


@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_fp32_adjoint_in_forced_lane_layouts(lanes):
    """The FP32 adjoint in a forced layout (2 lanes per line: 16 lines per warp, 4
    energies per lane; 4 and 8 lanes) against the FP64 adjoint: the lines of a
    warp and the lane sums of the cotangents in every layout."""
    from paper_2205_15000_b300 import sc
    p, d, a = _grain()
    gd64, ga64 = _adjoint(p, d, a, "fp64", g_Ftotal=1.0)
    ctx = sc.Context(p, precision="fp32", lanes_per_line=lanes)
    assert sc.sc_get_info(ctx.h).lanes_per_line == lanes
    ctx.set_fields(d, a)
    sc.sc_burnin(ctx.h, 300, 1e-6)
    ctx.sweep()
    gd32, ga32 = (x.cpu().numpy() for x in ctx.adjoint(g_Ftotal=1.0))
    assert np.max(np.abs(gd32 - gd64)) <= 1e-3 * np.max(np.abs(gd64))
    assert np.max(np.abs(ga32 - ga64)) <= 1e-3 * np.max(np.abs(ga64))


def _oracle_ldos_fixed(g, d, a, e, dl, ex):
    im, _ = g.sweep(d, a, np.asarray(e) + 1j * dl, 1, ex)
    return g.rotate_back(im, 1, len(e))


def _oracle_ldos_exits(g, d, a, e, dl, n=400, tol=1e-13):
    ex = None
    z = np.asarray(e) + 1j * dl
    for _ in range(n):
        im, ex2 = g.sweep(d, a, z, 1, ex)
        if ex is not None and np.max(np.abs(ex2 - ex)) < tol:
            return ex2
        ex = ex2
    return ex


def test_ldos_map_gradient_matches_oracle_fd():
    """L2 misfit of the LDOS map to a synthetic target (another vortex position,
    1% noise): autograd gradient vs central differences of the oracle's LDOS
    with converged boundary values held fixed."""
    import torch
    from paper_2205_15000_b300 import sc
    from paper_2205_15000_b300.autograd import ldos_map
    p, d, a = _grain()
    e = np.linspace(-0.2, 0.2, 6)
    dl = 0.05
    g = oracle.OracleGeom(p)
    d_t = W.vortex_delta(p, 0.22, [(-1.0, -0.5)], [-1])
    ex_t = _oracle_ldos_exits(g, d_t, a, e, dl)
    rng = np.random.default_rng(9)
    target = _oracle_ldos_fixed(g, d_t, a, e, dl, ex_t)
    target = target * (1 + 0.01 * rng.standard_normal(target.shape))
    m = g.mask().astype(bool)
    ex = _oracle_ldos_exits(g, d, a, e, dl)

    def loss(dd, aa):
        N = _oracle_ldos_fixed(g, dd, aa, e, dl, ex)
        return float(np.sum(((N - target) ** 2)[:, m]))
    probes = _probes(p, g, 6, 44)
    fd = _fd(loss, d, a, probes)
    ctx = sc.Context(p, precision="fp64")
    dt = torch.tensor(d, dtype=torch.complex128, device="cuda", requires_grad=True)
    at = torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
    N = ldos_map(ctx, dt, list(e), dl, at, n_burnin=400)
    tgt = torch.tensor(target, device="cuda")
    mk = torch.tensor(m, device="cuda")
    L = (((N - tgt) ** 2) * mk).sum()
    L.backward()
    gd, ga = dt.grad.cpu().numpy(), at.grad.cpu().numpy()
    adj = np.array([[gd[j, i].real, gd[j, i].imag, ga[j, i, 0], ga[j, i, 1]] for j, i in probes])
    scale = np.max(np.abs(fd))
    assert scale > 0
    assert np.max(np.abs(adj - fd)) <= 1e-5 * scale, np.max(np.abs(adj - fd)) / scale


def test_autograd_free_energy_matches_oracle_fd():
    import torch
    from paper_2205_15000_b300 import sc
    from paper_2205_15000_b300.autograd import riccati_sweep
    p, d, a = _grain()
    g = oracle.OracleGeom(p)
    ex = _oracle_converged_exits(g, d, a)
    probes = _probes(p, g, 6, 45)
    fd = _fd(lambda dd, aa: g.full_sweep(dd, aa, ex)["F_total"], d, a, probes)
    ctx = sc.Context(p, precision="fp64")
    ctx.set_fields(d, a)
    sc.sc_burnin(ctx.h, 300, 1e-13)
    dt = torch.tensor(d, dtype=torch.complex128, device="cuda", requires_grad=True)
    at = torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
    dn, j, F, Ft = riccati_sweep(ctx, dt, at)
    Ft.backward()
    gd, ga = dt.grad.cpu().numpy(), at.grad.cpu().numpy()
    adj = np.array([[gd[j_, i].real, gd[j_, i].imag, ga[j_, i, 0], ga[j_, i, 1]] for j_, i in probes])
    assert np.max(np.abs(adj - fd)) <= 1e-6 * np.max(np.abs(fd))


@pytest.mark.parametrize("k", [2, 5, 32])
def test_checkpointed_fp32_adjoint_equals_parked(k):
    """The FP32 adjoint with the forward gamma kept every k samples and
    recomputed from there gives the parked adjoint's gradient (the recomputed
    gammas are the same FP32 values; only the order of the atomic cotangent
    sums differs), also on lines shorter than k."""
    from paper_2205_15000_b300 import sc
    p, d, a = _grain()
    ref = _adjoint(p, d, a, "fp32", g_Ftotal=1.0)
    got = _adjoint(dict(p, adjoint_checkpoint=k), d, a, "fp32", g_Ftotal=1.0)
    for x, y in zip(got, ref):
        assert np.max(np.abs(x - y)) <= 1e-5 * np.max(np.abs(y))
    with pytest.raises(sc.ScError):
        sc.Context(dict(p, adjoint_checkpoint=k), precision="fp64")
    with pytest.raises(sc.ScError):
        sc.Context(dict(p, adjoint_checkpoint=1), precision="fp32")
