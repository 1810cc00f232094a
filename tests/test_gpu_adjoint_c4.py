"""Adjoint sweep at the size of the adjoint workload: d_{x2-y2} disc of radius
25 xi0 on a 128 x 128 grid, 64 Fermi angles, t = 0.2 (40 Matsubara energies
below the cutoff 16 pi kB Tc), one vortex at a seeded position.

The gradients of the free energy F/Omega_A and of the L2 misfit of the LDOS
map (64 energies spanning [-Delta0, Delta0], broadening 0.05 Delta0) to a
synthetic target (the LDOS of a second seeded vortex position with 1 %
noise) with respect to Re Delta, Im Delta, A_x and A_y at 32 seeded probe
points are compared with central finite differences of the FP64 oracle, in
both library precisions: FP64 within 1e-6, FP32 within 1e-3 of the largest
difference quotient.  Boundary entry values are converged at the evaluation
point and held fixed on both sides (the adjoint's reading of the boundary
condition).  Gradients are taken at a non-self-consistent Delta, where they
do not vanish.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu

N_PROBES = 32
TOL = {"fp64": 1e-6, "fp32": 1e-3}


def _c4():
    p, d, _ = W.c4_disc_d()
    rng = np.random.default_rng(404)
    d = d * (1.0 + 0.05 * (rng.standard_normal(d.shape) + 1j * rng.standard_normal(d.shape)) / math.sqrt(2))
    a = np.zeros((p["ny"], p["nx"], 2))
    return p, d, a


def _probes(p, g, n, seed):
    rng = np.random.default_rng(seed)
    m = g.mask().astype(bool)
    X, Y = W.grid_xy(p)
    idx = np.argwhere(m & (np.hypot(X, Y) < 20.0))
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


def _at(gd, ga, probes):
    return np.array([[gd[j, i].real, gd[j, i].imag, ga[j, i, 0], ga[j, i, 1]] for j, i in probes])


def _converged_exits(step, n=400, tol=1e-13):
    ex = None
    for _ in range(n):
        ex2 = step(ex)
        if ex is not None and np.max(np.abs(ex2 - ex)) < tol:
            return ex2
        ex = ex2
    return ex


@pytest.fixture(scope="module")
def c4():
    p, d, a = _c4()
    return p, d, a, oracle.OracleGeom(p)


def test_c4_free_energy_gradient_matches_oracle_fd(c4):
    from paper_2205_15000_b300 import sc
    p, d, a, g = c4
    ex = _converged_exits(lambda e: g.full_sweep(d, a, e)["exit"])
    probes = _probes(p, g, N_PROBES, 4401)
    fd = _fd(lambda dd, aa: g.full_sweep(dd, aa, ex)["F_total"], d, a, probes)
    scale = np.max(np.abs(fd))
    assert scale > 0
    # FP32 also with the forward gamma kept every 32 samples and recomputed
    for precision, ckpt in (("fp64", 0), ("fp32", 0), ("fp32", 32)):
        ctx = sc.Context(dict(p, adjoint_checkpoint=ckpt), precision=precision)
        ctx.set_fields(d, a)
        sc.sc_burnin(ctx.h, 400, 1e-13 if precision == "fp64" else 1e-6)
        ctx.sweep()
        gd, ga = ctx.adjoint(g_Ftotal=1.0)
        err = np.max(np.abs(_at(gd.cpu().numpy(), ga.cpu().numpy(), probes) - fd)) / scale
        print(f"c4 free-energy gradient, {precision}, checkpoint {ckpt}: max error / max |FD| = {err:.3e}")
        assert err <= TOL[precision], (precision, ckpt, err)
        ctx.close()


def test_c4_ldos_misfit_gradient_matches_oracle_fd(c4):
    import torch
    from paper_2205_15000_b300 import sc
    from paper_2205_15000_b300.autograd import ldos_map
    p, d, a, g = c4
    d0 = math.sqrt(2.0) * oracle.bulk_gap(1, p["t"], p["n_energies"], p["n_angles"])
    e = np.linspace(-d0, d0, 64)
    dl = 0.05 * d0
    z = e + 1j * dl
    # the target: LDOS of a second seeded vortex position, 1 % multiplicative noise
    rng = np.random.default_rng(4402)
    r, th = 15.0 * math.sqrt(rng.uniform()), rng.uniform(0, 2 * math.pi)
    d_t = W.vortex_delta(p, W.BULK_GUESS[("dx2y2", 0.2)], [(r * math.cos(th), r * math.sin(th))], [-1])
    ex_t = _converged_exits(lambda x: g.sweep(d_t, a, z, 1, x)[1])
    target = g.rotate_back(g.sweep(d_t, a, z, 1, ex_t)[0], 1, len(e))
    target = target * (1 + 0.01 * rng.standard_normal(target.shape))
    m = g.mask().astype(bool)
    ex = _converged_exits(lambda x: g.sweep(d, a, z, 1, x)[1])

    def loss(dd, aa):
        N = g.rotate_back(g.sweep(dd, aa, z, 1, ex)[0], 1, len(e))
        return float(np.sum(((N - target) ** 2)[:, m]))
    probes = _probes(p, g, N_PROBES, 4403)
    fd = _fd(loss, d, a, probes)
    scale = np.max(np.abs(fd))
    assert scale > 0
    tgt = torch.tensor(target, device="cuda")
    mk = torch.tensor(m, device="cuda")
    for precision in ("fp64", "fp32"):
        ctx = sc.Context(p, precision=precision)
        dt = torch.tensor(d, dtype=torch.complex128, device="cuda", requires_grad=True)
        at = torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
        N = ldos_map(ctx, dt, list(e), dl, at, n_burnin=400)
        (((N - tgt) ** 2) * mk).sum().backward()
        err = np.max(np.abs(_at(dt.grad.cpu().numpy(), at.grad.cpu().numpy(), probes) - fd)) / scale
        print(f"c4 LDOS-misfit gradient, {precision}: max error / max |FD| = {err:.3e}")
        assert err <= TOL[precision], (precision, err)
        ctx.close()
