"""Pins of the oracle's Ozaki energy sums (Sec. 3.1, Ozaki's continued-fraction
representation of the Fermi function) against closed forms: the Fermi
function itself, the first poles on the Matsubara frequencies, the BCS kernel
sum_n 1/(omega_n^2 + y^2) = tanh(y/2)/(2y), the bulk gap of the converged
Matsubara sum, and the bulk fixed point of a full weighted sweep."""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_2205_15000_b300 import workloads as W


def test_first_poles_are_matsubara_frequencies():
    z, R = oracle.ozaki_poles(32)
    n = np.arange(8)
    np.testing.assert_allclose(z[:8], math.pi * (2 * n + 1), rtol=1e-13)
    np.testing.assert_allclose(R[:8], 1.0, rtol=1e-12)
    assert np.all(np.diff(z) > 0) and np.all(R > 0)


@pytest.mark.parametrize("n", [16, 32])
def test_poles_reproduce_the_fermi_function(n):
    z, R = oracle.ozaki_poles(n)
    for x in np.linspace(-40.0, 40.0, 161):
        f = 0.5 - np.sum(R * 2 * x / (x * x + z * z))
        assert abs(f - 1.0 / (1.0 + math.exp(x))) < 1e-14


def test_pole_sum_of_the_bcs_kernel():
    """sum over all Matsubara frequencies of 1/(omega_n^2 + y^2) =
    tanh(y/2)/(2y) (omega_n = pi(2n+1)); the pole sum with weights R_p."""
    z, R = oracle.ozaki_poles(64)
    for y in (0.01, 0.5, 3.0, 20.0, 80.0):
        s = np.sum(R * 2.0 / (z * z + y * y))
        assert abs(s - math.tanh(y / 2) / (2 * y)) < 1e-13 * math.tanh(y / 2) / (2 * y)


def _bulk_gap(eps, w, t):
    """s-wave bulk gap of the regularised gap equation with energies eps and
    weights w: t sum w / sqrt(eps^2 + Delta^2) = ln t + t sum w / eps."""
    D = math.log(t) + t * np.sum(w / eps)
    return optimize.brentq(lambda d: t * np.sum(w / np.sqrt(eps ** 2 + d * d)) - D, 1e-9, 2.0,
                           xtol=1e-15, rtol=1e-15)


@pytest.mark.parametrize("t", [0.1, 0.5, 0.9])
def test_ozaki_bulk_gap_equals_converged_matsubara(t):
    """With the same regularisation, the Ozaki sum converges to the bulk gap of
    the cutoff-free Matsubara sum (10^6 energies; its tail is below 1e-12):
    within 5e-8 at 128 poles, and the error falls faster than N^-3."""
    n = np.arange(1_000_000)
    eps_m = t * (n + 0.5)
    d_m = _bulk_gap(eps_m, np.ones_like(eps_m), t)
    err = {}
    for npole in (32, 64, 128):
        eps_o, w_o = oracle.ozaki_energies(t, npole)
        err[npole] = abs(_bulk_gap(eps_o, w_o, t) - d_m) / d_m
    assert err[128] < 5e-8
    assert err[32] / err[64] > 8 and err[64] / err[128] > 8, err


def test_ozaki_sweep_bulk_maps_to_itself():
    """A uniform real s-wave Delta at the Ozaki bulk gap is a fixed point of a
    full sweep with Ozaki energies and weights (weighted image sums and the
    weighted normalisation D), through the specular boundary links."""
    t, npole, N = 0.5, 12, 32
    p = W.disc(7.0, 40, pairing=0, t=t, n_angles=N, n_energies=npole)
    p["energy_sum"] = "ozaki"
    eps, w = oracle.ozaki_energies(t, npole)
    d0 = _bulk_gap(eps, w, t)
    g = oracle.OracleGeom(p)
    delta = np.full((p["ny"], p["nx"]), d0, complex)
    m = g.mask().astype(bool)
    ex = None
    for _ in range(2):
        out = g.full_sweep(delta, None, ex)
        ex = out["exit"]
        assert np.max(np.abs(out["delta_new"][m] - d0)) < 1e-12
        assert np.max(np.abs(out["j"])) < 1e-12
