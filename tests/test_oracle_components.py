"""Pins of the oracle's multi-component order parameter (Eq. order_parameter,
Delta(p, R) = sum_Gamma Delta_Gamma(R) eta_Gamma(p); per-component gap
equation Eq. gapeq_fixpoint with D_Gamma = ln(T/T_c^Gamma) + pi T sum 1/|eps_n|;
free energy Eq. qcLWFE) against closed forms written here from the paper's
basis-function table, and reductions to the single-component oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

# Table basis_functions (circular Fermi surface): eta of each pairing at angle phi
ETA = {0: lambda ph: np.ones_like(ph), 1: lambda ph: math.sqrt(2) * np.cos(2 * ph),
       2: lambda ph: math.sqrt(2) * np.sin(2 * ph), 3: lambda ph: math.sqrt(2) * np.sin(4 * ph)}


def _uniform(p, values):
    return np.stack([np.full((p["ny"], p["nx"]), v, complex) for v in values])


@pytest.mark.parametrize("comps,values", [
    ([(2, 1.0), (1, 1.0)], [0.22, 0.22j]),                 # chiral d_xy + i d_x2-y2
    ([(1, 1.0), (0, 0.6)], [0.2, 0.07j]),                  # d + i s, s with T_c^s = 0.6 T_c
    ([(2, 1.0), (0, 0.8)], [0.15 + 0.05j, -0.04]),         # d_xy + s
])
def test_uniform_state_first_sweep_closed_form(comps, values):
    """Uniform Delta_Gamma, A = 0, first sweep from homogeneous entry values:
    gamma is the homogeneous solution on every segment, so at every grain point
    Delta_new_Gamma = t sum_k w_k eta_Gamma(k) Delta(k) sum_n 1/sqrt(eps_n^2 + |Delta(k)|^2) / D_Gamma
    and F is the bulk Eilenberger form of |Delta(k)| (Eq. FEbulk) plus
    sum_Gamma |Delta_Gamma|^2 ln(T_c / T_c^Gamma)."""
    t, ne, N = 0.5, 10, 32
    p = W.disc(6.0, 40, pairing=comps[0][0], t=t, n_angles=N, n_energies=ne)
    p["components"] = comps
    g = oracle.OracleGeom(p)
    delta = _uniform(p, values)
    out = g.full_sweep(delta)
    w, vh, _ = g.quadrature()
    ph = np.arctan2(vh[:, 1], vh[:, 0])
    eps = t * (np.arange(ne) + 0.5)
    eta = np.stack([ETA[pc](ph) for pc, _ in comps])
    dk = np.einsum("ck,c->k", eta, np.array(values))          # Delta(k)
    ad2 = np.abs(dk) ** 2
    s1 = np.sum(1.0 / np.sqrt(eps[None, :] ** 2 + ad2[:, None]), axis=1)
    D = math.log(t) + 2 * np.sum(1.0 / (2 * np.arange(ne) + 1))
    m = g.mask().astype(bool)
    for c, (pc, tcr) in enumerate(comps):
        Dc = D - math.log(tcr)
        ref = t * np.sum(w * eta[c] * dk * s1) / Dc
        np.testing.assert_allclose(out["delta_new"][c][m], ref, rtol=0, atol=1e-13)
    # free energy: bulk Eilenberger form, with the per-component normalisations
    Om = np.sqrt(ad2[:, None] + eps[None, :] ** 2)
    feb = np.sum(w * (ad2 * math.log(t) + t * np.sum(ad2[:, None] ** 2 / (eps * (Om + eps) ** 2), axis=1)))
    feb -= sum(abs(v) ** 2 * math.log(tcr) for v, (_, tcr) in zip(values, comps))
    np.testing.assert_allclose(out["F"][m], feb, rtol=0, atol=1e-13)


def test_single_component_list_equals_plain_parameters():
    p = W.diamond(8.0, 32, pairing=1, t=0.4, n_angles=16, n_energies=6, flux_quanta=0.6)
    d = W.noisy_delta(p, 0.22, 0.1, seed=3)
    a = oracle.OracleGeom(p).full_sweep(d)
    q = dict(p, components=[(1, 1.0)])
    b = oracle.OracleGeom(q).full_sweep(d)
    np.testing.assert_array_equal(a["delta_new"], b["delta_new"])
    np.testing.assert_array_equal(a["F"], b["F"])


def test_second_component_zero_reduces_to_one_component():
    """Delta_2 = 0: the sweep sees only Delta_1 eta_1, so component 1's update,
    j and F equal the single-component oracle's (to rounding of the combined
    field); component 2's update is the induced projection <eta_2 S_f>."""
    p = W.disc(5.0, 32, pairing=1, t=0.3, n_angles=16, n_energies=8, flux_quanta=0.8)
    d1 = W.vortex_delta(p, 0.22, [(1.0, 0.5)], [-1], seed=5, rel_noise=0.05)
    single = oracle.OracleGeom(p).full_sweep(d1)
    q = dict(p, components=[(1, 1.0), (0, 0.5)])
    two = oracle.OracleGeom(q).full_sweep(np.stack([d1, np.zeros_like(d1)]))
    m = oracle.OracleGeom(p).mask().astype(bool)
    np.testing.assert_allclose(two["delta_new"][0][m], single["delta_new"][m], rtol=0, atol=1e-14)
    np.testing.assert_allclose(two["j"], single["j"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(two["F"], single["F"], rtol=0, atol=1e-14)
    assert np.max(np.abs(two["delta_new"][1][m])) > 1e-4  # an s component is induced
