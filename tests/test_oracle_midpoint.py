"""Pins of the oracle's implicit midpoint stepper (App. C, Eq. riccati_midpoint)
against facts that do not come from the oracle: the implicit rule itself, its
linear (Cayley) limit, the homogeneous fixed point, second-order convergence
to the exact solution for constant coefficients, an independent fixed-point
solution of the rule along every segment of a tiny grain, the bulk map of a
full sweep, and O(h^2) agreement with the closed-form stepper.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W


def _f(P, Q, R, g):
    return 1j * (P * g * g + 2 * Q * g + R)


def _random_coeffs(rng, independent):
    D = complex(*rng.normal(0, 0.4, 2))
    z = complex(rng.normal(0, 0.4), rng.uniform(0.02, 1.5))
    if independent:  # Delta and Delta* as independent arguments
        return complex(*rng.normal(0, 0.4, 2)), z, D
    return D.conjugate(), z, D


@pytest.mark.parametrize("independent", [False, True])
def test_midpoint_step_satisfies_the_implicit_rule(independent):
    """gamma_{j+1} = gamma_j + h f((gamma_j + gamma_{j+1})/2): the quadratic's
    root is a solution of the update rule the paper states."""
    rng = np.random.default_rng(21)
    for _ in range(200):
        P, Q, R = _random_coeffs(rng, independent)
        ell = rng.uniform(1e-4, 0.8)
        g0 = complex(*rng.normal(0, 0.5, 2))
        g1 = oracle.step_midpoint(P, Q, R, ell, g0)
        res = g1 - g0 - ell * _f(P, Q, R, 0.5 * (g0 + g1))
        assert abs(res) < 1e-14 * max(1.0, abs(g1))


def test_midpoint_linear_limit_is_the_cayley_map():
    """Delta = 0: the rule is linear and its solution is the Cayley form
    g1 = (g0 (1 + i h z) + i h R)/(1 - i h z) (the root continuous in Delta)."""
    rng = np.random.default_rng(22)
    for _ in range(50):
        z = complex(rng.normal(0, 0.4), rng.uniform(0.02, 1.5))
        R = complex(*rng.normal(0, 0.3, 2))
        ell = rng.uniform(1e-3, 0.8)
        g0 = complex(*rng.normal(0, 0.5, 2))
        ref = (g0 * (1 + 1j * ell * z) + 1j * ell * R) / (1 - 1j * ell * z)
        assert abs(oracle.step_midpoint(0.0, z, R, ell, g0) - ref) < 1e-15 * max(1.0, abs(ref))


def test_midpoint_homogeneous_solution_is_a_fixed_point():
    """f(gamma_h) = 0 for constant coefficients, so gamma_h = -Delta/(z + i Omega)
    maps to itself (bulk: gamma = i Delta/(eps + sqrt(eps^2 + |Delta|^2)))."""
    for D in (0.27, 0.2 + 0.1j, -0.05j):
        for eps in (0.05, 0.3, 2.0):
            gh = 1j * D / (eps + math.sqrt(eps ** 2 + abs(D) ** 2))
            for ell in (0.01, 0.37, 1.5):
                assert abs(oracle.step_midpoint(complex(D).conjugate(), 1j * eps, D, ell, gh) - gh) < 1e-15


def test_midpoint_is_second_order():
    """Constant coefficients over a length L: n midpoint steps of L/n converge
    to the exact solution (the closed-form step over L) with error ~ n^-2."""
    rng = np.random.default_rng(23)
    for _ in range(6):
        P, Q, R = _random_coeffs(rng, False)
        L = rng.uniform(0.5, 2.0)
        g0 = complex(*rng.normal(0, 0.4, 2))
        exact = oracle.step(P, Q, R, L, g0)
        errs = []
        for n in (16, 32, 64, 128):
            g = g0
            for _ in range(n):
                g = oracle.step_midpoint(P, Q, R, L / n, g)
            errs.append(abs(g - exact))
        ratios = [errs[i] / errs[i + 1] for i in range(3)]
        assert all(3.6 < r < 4.4 for r in ratios), ratios
        assert errs[-1] < 1e-4


def _midpoint_by_iteration(P, Q, R, ell, g0):
    """The implicit rule solved by fixed-point iteration (a different solver)."""
    g1 = g0
    for _ in range(200):
        g1 = g0 + ell * _f(P, Q, R, 0.5 * (g0 + g1))
    return g1


def test_midpoint_sweep_segments_brute_force():
    """On a tiny grain with the midpoint stepper, gamma at every sample of the
    lines of one pair equals the implicit rule solved by iteration along the
    segments (half-step coefficients by linear interpolation between samples,
    nearest-sample values on the end segments, App. C), entry = homogeneous
    solution."""
    t, ne, N = 0.5, 2, 4
    p = W.disc(1.6, 8, pairing=0, t=t, n_angles=N, n_energies=ne, flux_quanta=0.7)
    p["stepper"] = "midpoint"
    g = oracle.OracleGeom(p)
    rng = np.random.default_rng(11)
    delta = 0.25 * (1 + 0.3 * (rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))))
    im, ex, gam = g.sweep(delta, None, g.matsubara(), 0, None, want_gammas=True)
    L = g.lines()
    w, vh, eta = g.quadrature()
    h = p["h"]
    eps = t * (np.arange(ne) + 0.5)
    off = 0
    pair = 0
    ds, av = g.sample_fields(delta, None, pair)
    e = vh[pair]
    checked = 0
    for l in range(L["l_lo"][pair], L["l_hi"][pair] + 1):
        i = l - L["l_lo"][pair]
        m0, m1 = L["m0"][i], L["m1"][i]
        ns = m1 - m0 + 1
        if ns < 2:
            off += max(ns, 0)
            continue
        dl = ds[off:off + ns] * eta[pair]
        al = -1 * (av[off:off + ns] @ e)
        segs = [(dl[0], al[0], m0 * h - L["smin"][i])]
        segs += [(0.5 * (dl[q - 1] + dl[q]), 0.5 * (al[q - 1] + al[q]), h) for q in range(1, ns)]
        for n in range(ne):
            z0 = 1j * eps[n]
            D0, a0, _ = segs[0]
            z = z0 + a0
            Om = np.sqrt(abs(D0) ** 2 - z * z)
            gm = -D0 / (z + 1j * Om)
            for q, (Dc, ac, ell) in enumerate(segs):
                gm = _midpoint_by_iteration(np.conj(Dc), z0 + ac, Dc, ell, gm)
                assert abs(gm - gam[0][off + q, n]) < 1e-13
                checked += 1
        off += ns
    assert checked > 10


@pytest.mark.parametrize("shape", ["square", "disc"])
def test_midpoint_sweep_bulk_maps_to_itself(shape):
    """Uniform real s-wave Delta at its bulk value, A = 0: with the midpoint
    stepper, too, gamma is the homogeneous solution everywhere and the gap
    equation returns Delta (Eq. gapeq_fixpoint)."""
    t, ne, N = 0.5, 16, 32
    kw = dict(pairing=0, t=t, n_angles=N, n_energies=ne)
    p = W.square(12.0, 48, **kw) if shape == "square" else W.disc(7.0, 48, **kw)
    p["stepper"] = "midpoint"
    d0 = oracle.bulk_gap(0, t, ne, N)
    g = oracle.OracleGeom(p)
    delta = np.full((p["ny"], p["nx"]), d0, complex)
    m = g.mask().astype(bool)
    ex = None
    for it in range(2):
        out = g.full_sweep(delta, None, ex)
        ex = out["exit"]
        assert np.max(np.abs(out["delta_new"][m] - d0)) < 1e-12
        assert np.max(np.abs(out["j"])) < 1e-12


def _smooth_grain(n):
    p = W.disc(5.0, n, pairing=1, t=0.5, n_angles=16, n_energies=6, flux_quanta=0.4)
    X, Y = W.grid_xy(p)
    delta = 0.22 * (1 + 0.3 * np.cos(0.5 * X) * np.sin(0.4 * Y)) * np.exp(0.35j * X + 0.2j * Y)
    return p, delta


def test_steppers_agree_to_second_order_in_h():
    """Both steppers approximate the same continuum equation to O(h^2): the
    difference of their free energies after two sweeps falls ~4x per halving of
    the grid spacing (smooth Delta, same grain)."""
    diffs = []
    for n in (24, 48, 96):
        p, delta = _smooth_grain(n)
        F = {}
        for st in ("closed", "midpoint"):
            q = dict(p)
            q["stepper"] = st
            g = oracle.OracleGeom(q)
            ex = None
            for _ in range(2):
                out = g.full_sweep(delta, None, ex)
                ex = out["exit"]
            F[st] = out["F_total"]
        diffs.append(abs(F["closed"] - F["midpoint"]))
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    assert 2.8 < r1 < 5.5 and 2.8 < r2 < 5.5, (diffs, r1, r2)
