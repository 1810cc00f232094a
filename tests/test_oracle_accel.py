"""Pins of the oracle's self-consistency accelerators (App. E) against facts
that do not come from the oracle: reductions to the Picard step, the exact
secant step of Barzilai-Borwein on linear problems, the classical BB formulas
in terms of s = x_i - x_{i-1} and y = d_{i-1} - d_i, the similarity weight of
CongAcc, and the Picard loop of Algorithm 1."""
import math

import numpy as np
import pytest

import oracle
from oracle import accel
from paper_2205_15000_b300 import workloads as W


def _linear_problem(n, seed, lo=-0.9, hi=0.9):
    """g(x) = A x + b with a symmetric contraction A (eigenvalues in (lo, hi))."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(lo, hi, n)
    A = (q * lam) @ q.T
    b = rng.standard_normal(n)
    xs = np.linalg.solve(np.eye(n) - A, b)
    return A, b, xs


def _run(params, A, b, x0, n_iter, split=(2,)):
    acc = accel.Accelerator(params)
    x = x0.copy()
    xs = [x.copy()]
    for _ in range(n_iter):
        parts = np.split(x, split)
        g = A @ x + b
        x = np.concatenate(acc.step(parts, np.split(g, split)))
        xs.append(x.copy())
    return xs, acc


def test_polyak_without_drag_memory_is_picard():
    """beta = 1: v_{i+1} = alpha d_i, so Polyak is Picard with step alpha."""
    A, b, _ = _linear_problem(6, 1)
    x0 = np.zeros(6)
    pol = dict(accel.default_params("polyak"), drag=1.0, step_size=0.7)
    pic = dict(accel.default_params("picard"), step_size=0.7)
    xa, _ = _run(pol, A, b, x0, 12)
    xb, _ = _run(pic, A, b, x0, 12)
    np.testing.assert_allclose(xa[-1], xb[-1], rtol=0, atol=1e-14)


def test_polyak_recurrence_closed_form():
    """x_{i+1} = x_i + (1 - beta)(x_i - x_{i-1}) + alpha d_i (the heavy-ball form)."""
    A, b, _ = _linear_problem(5, 2)
    p = accel.default_params("polyak")
    xs, _ = _run(p, A, b, np.zeros(5), 8)
    for i in range(1, 8):
        d = A @ xs[i] + b - xs[i]
        ref = xs[i] + (1 - p["drag"]) * (xs[i] - xs[i - 1]) + p["step_size"] * d
        np.testing.assert_allclose(xs[i + 1], ref, rtol=0, atol=1e-13)


def test_congacc_without_adaptation_is_picard():
    """k = 1 and s_min = -1: alpha_c never changes and w_c stays 0, so m = d."""
    A, b, _ = _linear_problem(6, 3)
    p = dict(accel.default_params("congacc"), step_size_factor=1.0, cos_similarity_min=-1.0)
    xa, _ = _run(p, A, b, np.zeros(6), 10)
    xb, _ = _run(dict(accel.default_params("picard"), step_size=p["step_size"]), A, b, np.zeros(6), 10)
    np.testing.assert_allclose(xa[-1], xb[-1], rtol=0, atol=1e-14)


def test_bb_exact_on_scalar_linear_problem():
    """g(x) = a x + b in one dimension: the BB1 step of the second iteration is
    the secant step alpha = 1/(1 - a), which lands on the fixed point."""
    for a, bb in ((0.5, 1.0), (-0.7, 0.3), (0.95, -2.0)):
        p = accel.default_params("barzilai-borwein")
        xs, acc = _run(p, np.array([[a]]), np.array([bb]), np.array([0.0]), 2, split=())
        assert abs(xs[2][0] - bb / (1 - a)) < 1e-12 * max(1.0, abs(bb / (1 - a)))


def test_bb_steps_are_the_classical_formulas():
    """alpha_{i+1} = s.s/s.y (BB1, i odd) or s.y/y.y (BB2, i even) with
    s = x_i - x_{i-1}, y = d_{i-1} - d_i (positive on a contraction)."""
    A, b, _ = _linear_problem(7, 4)
    p = dict(accel.default_params("barzilai-borwein"), step_size_max=1e9, step_size_min=1e-9)
    xs, _ = _run(p, A, b, np.zeros(7), 6)
    for i in range(1, 6):
        d_im1 = A @ xs[i - 1] + b - xs[i - 1]
        d_i = A @ xs[i] + b - xs[i]
        s = xs[i] - xs[i - 1]
        y = d_im1 - d_i
        alpha = abs(s @ s / (s @ y)) if i % 2 == 1 else abs(s @ y / (y @ y))
        np.testing.assert_allclose(xs[i + 1], xs[i] + alpha * d_i, rtol=0, atol=1e-11)


def test_congacc_similarity_weight_solves_its_equation():
    rng = np.random.default_rng(5)
    for _ in range(20):
        m = rng.standard_normal(9)
        d = -m + 0.3 * rng.standard_normal(9)  # nearly opposite: cos < s_min
        s_min = 0.7
        w = accel.Accelerator._similarity_weight(m, d, s_min)
        v = w * m + (1 - w) * d
        assert abs(v @ d / (np.linalg.norm(v) * np.linalg.norm(d)) - s_min) < 1e-12
        assert 0.0 < w < 1.0


def test_congacc_step_size_follows_similarity():
    """A persistent direction multiplies alpha by k per iteration (cos = 1); a
    direction that flips sign divides it by k (cos = -1)."""
    p = accel.default_params("congacc")
    k = p["step_size_factor"]
    acc = accel.Accelerator(p)
    x = [np.zeros(3)]
    for i in range(4):
        x = acc.step(x, [x[0] + np.array([1.0, 2.0, 3.0])])
    assert abs(acc.alpha_c[0] - p["step_size"] * k ** 3) < 1e-12
    acc = accel.Accelerator(dict(p, cos_similarity_min=-1.0))
    x = [np.zeros(3)]
    for i in range(4):
        sign = 1.0 if i % 2 == 0 else -1.0
        x = acc.step(x, [x[0] + sign * np.array([1.0, 2.0, 3.0])])
    assert abs(acc.alpha_c[0] - p["step_size"] * k ** -3) < 1e-12


@pytest.mark.parametrize("kind", ["picard", "polyak", "barzilai-borwein", "congacc"])
def test_accelerators_solve_a_linear_fixed_point(kind):
    """A slow contraction like the gap equation's (Jacobian eigenvalues in
    (0.05, 0.95)): every accelerator with its default parameters converges."""
    A, b, xs_true = _linear_problem(12, 6, 0.05, 0.95)
    xs, _ = _run(accel.default_params(kind), A, b, np.zeros(12), 400, split=(4, 8))
    assert np.linalg.norm(xs[-1] - xs_true) < 1e-8 * np.linalg.norm(xs_true)


def test_picard_loop_equals_algorithm_1_picard():
    """The accelerated loop with Picard, alpha = 1, is the plain fixed-point
    iteration of Algorithm 1 (Delta <- Delta_new, A_ind <- from j)."""
    p = W.disc(4.0, 24, pairing=0, t=0.5, n_angles=12, n_energies=5, flux_quanta=1.2, kappa=3.0)
    d0 = W.vortex_delta(p, 0.25, [(0.5, 0.0)], [-1])
    g = oracle.OracleGeom(p)
    ref = g.picard(d0, 4)
    out = g.self_consistency(d0, 4, accel.default_params("picard"))
    m = g.mask().astype(bool)
    np.testing.assert_allclose(out["delta"][m], ref["delta"][m], rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["aind"], ref["aind"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["history"], ref["history"], rtol=0, atol=1e-14)
