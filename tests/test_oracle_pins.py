"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, textbook limits, exactness properties of the quadrature,
an independent integrator, brute force on tiny inputs and invariances.

Each test names the passage of the paper that fixes the checked fact.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2205_15000_b300 import workloads as W

EULER_GAMMA = 0.5772156649015329


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    """Rows of a fixture under tests/golden ('|'-separated, '#' comments)."""
    with open(os.path.join(GOLDEN, name)) as f:
        return [[c.strip() for c in ln.split("|")] for ln in f if ln.strip() and not ln.startswith("#")]


def _printed_eta(expr, phi):
    """Evaluate a basis function as printed in the paper's table: 1, or
    sqrt(2)*sin(m*phi) / sqrt(2)*cos(m*phi)."""
    import re
    if expr == "1":
        return np.ones_like(phi)
    m = re.fullmatch(r"sqrt\(2\)\*(sin|cos)\((\d+)\*phi\)", expr)
    assert m, expr
    f = np.sin if m.group(1) == "sin" else np.cos
    return math.sqrt(2.0) * f(int(m.group(2)) * phi)


@pytest.mark.parametrize("row", _golden_rows("basis_functions.txt"), ids=lambda r: r[1])
def test_basis_functions_match_printed_table(row):
    """eta(phi) of every pairing symmetry at the Fermi angles phi_k = 2 pi k / N
    equals the printed table of basis functions (Table basis_functions;
    fixture tests/golden/basis_functions.txt)."""
    pairing, _, expr = int(row[0]), row[1], row[2]
    p = W.disc(5.0, 24, pairing=pairing, n_angles=64, n_energies=4, t=0.5)
    _, _, eta = oracle.OracleGeom(p).quadrature()
    phi = 2.0 * np.pi * np.arange(64) / 64
    np.testing.assert_allclose(eta, _printed_eta(expr, phi), rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# Fermi-surface quadrature (Sec. 3.1): rule by divisibility of N by 4, 3, 2.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,rule_order", [(32, 4), (24, 4), (18, 3), (10, 2), (64, 4), (12, 4),
                                          (6, 3)])
def test_quadrature_exact_for_trig_polynomials(N, rule_order):
    w = np.array([oracle.quad_weight(k, N) for k in range(N)])
    assert abs(w.sum() - 1.0) < 1e-14
    phi = 2 * np.pi * np.arange(N) / N
    # A periodic rule whose weights repeat with period P integrates e^{i m phi}
    # exactly unless (N/P) divides m.
    P = {4: 4, 3: 3, 2: 2}[rule_order]
    for m in range(1, N):
        if m % (N // P) == 0:
            continue
        assert abs(np.sum(w * np.exp(1j * m * phi))) < 1e-14, m


def test_quadrature_composite_weights():
    # Boole's rule on [0, 4h]: (2h/45)(7, 32, 12, 32, 7); closed periodically the
    # end weights add up.  Check against scipy's Newton-Cotes coefficients.
    for n_pts, N in ((4, 32), (3, 18), (2, 10)):
        an, _ = integrate.newton_cotes(n_pts, 1)
        period = np.zeros(n_pts)
        period[:] = an[:n_pts]
        period[0] += an[n_pts]
        period = period / period.sum() / (N / n_pts)
        w = np.array([oracle.quad_weight(k, N) for k in range(n_pts)])
        np.testing.assert_allclose(w, period, rtol=1e-14)


# ---------------------------------------------------------------------------
# Gap-equation normalisation (Eq. gapeq_fixpoint): ln t + pi T sum 1/|eps_n|
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("t,ne", [(0.5, 16), (0.1, 80), (0.05, 160), (1.0, 3)])
def test_norm_D_digamma(t, ne):
    # sum_{n<N} 1/(2n+1) = (psi(N+1/2) - psi(1/2)) / 2
    ref = math.log(t) + (special.digamma(ne + 0.5) - special.digamma(0.5))
    assert abs(oracle.norm_D(t, ne) - ref) < 1e-12


# ---------------------------------------------------------------------------
# Bulk gap: BCS limits of the regularised gap equation (Eq. gapeq_regularized)
# ---------------------------------------------------------------------------
def test_bulk_gap_bcs_zero_temperature_s():
    # Delta(0) = pi e^{-gamma_E} kB Tc  ->  e^{-gamma_E}/2 in units of 2 pi kB Tc
    t = 0.01
    ne = W.n_energies_for_cutoff(t, 200.0)
    d = oracle.bulk_gap(0, t, ne, 32)
    assert abs(d - math.exp(-EULER_GAMMA) / 2) < 2e-6


def test_bulk_gap_bcs_zero_temperature_d():
    # eta = sqrt2 cos 2phi: ln(Delta0 / Delta_s(0)) = -<eta^2 ln|eta|> = -(1 - ln 2)/2
    t = 0.01
    ne = W.n_energies_for_cutoff(t, 200.0)
    # the nodal integrand is sharp at low energy: resolve it with 1024 angles
    d = oracle.bulk_gap(1, t, ne, 1024)
    ref = math.exp(-EULER_GAMMA) / 2 * math.exp(-(1 - math.log(2)) / 2)
    assert abs(d - ref) / ref < 2e-6


def test_bulk_gap_near_tc_ginzburg_landau():
    # Delta^2 = 8 pi^2 Tc^2 (1-t) / (7 zeta(3)) -> Delta/(2 pi Tc) = sqrt(2(1-t)/(7 zeta3))
    zeta3 = special.zeta(3)
    for one_minus_t in (1e-3, 4e-3):
        t = 1 - one_minus_t
        ne = W.n_energies_for_cutoff(t, 400.0)
        d = oracle.bulk_gap(0, t, ne, 8)
        ref = math.sqrt(2 * one_minus_t / (7 * zeta3))
        assert abs(d / ref - 1) < 3 * one_minus_t + 2e-3


@pytest.mark.parametrize("pairing,t,ne,anchor", [(0, 0.5, 16, 0.268717), (1, 0.1, 80, 0.240792),
                                                 (1, 0.2, 40, 0.240128), (1, 0.05, 160, 0.240871)])
def test_bulk_gap_anchor_values(pairing, t, ne, anchor):
    """The truncated bulk gap equation (Eq. gapeq_fixpoint with the regularised
    normalisation of Eq. gapeq_regularized, energies below the cutoff) solved
    independently to six decimals for the workloads' temperatures and energy
    counts (units 2 pi kB Tc; the d-wave value is the amplitude of
    Delta(phi) = Delta sqrt(2) cos 2 phi).  1024 angles stand in for the
    continuum angle average."""
    assert abs(oracle.bulk_gap(pairing, t, ne, 1024) - anchor) < 6e-7


def test_bulk_gap_vanishes_at_tc():
    # at t = 1 the right-hand side at Delta = 0 equals D exactly (the
    # regularisation puts Tc where the cutoff sum starts); only rounding is left
    assert oracle.bulk_gap(0, 1.0, 400, 8) < 1e-6
    assert oracle.bulk_gap(1, 1.0, 400, 32) < 1e-6


# ---------------------------------------------------------------------------
# Closed-form step (stepping method of App. C) vs an independent RK4 on
# d gamma/ds = i (P g^2 + 2 Q g + R)  (Eq. riccati_standard_form).
# ---------------------------------------------------------------------------
def _rk4(P, Q, R, ell, g, n=20000):
    f = lambda x: 1j * (P * x * x + 2 * Q * x + R)  # noqa: E731
    hh = ell / n
    for _ in range(n):
        k1 = f(g)
        k2 = f(g + 0.5 * hh * k1)
        k3 = f(g + 0.5 * hh * k2)
        k4 = f(g + hh * k3)
        g = g + hh / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return g


def test_step_matches_rk4():
    rng = np.random.default_rng(7)
    for _ in range(12):
        D = complex(*rng.normal(0, 0.3, 2))
        z = complex(rng.normal(0, 0.3), rng.uniform(0.02, 1.0))
        ell = rng.uniform(1e-4, 0.6)
        g0 = complex(*rng.normal(0, 0.4, 2))
        # gamma: P = Delta*, Q = z, R = Delta
        ref = _rk4(D.conjugate(), z, D, ell, g0)
        assert abs(oracle.step(D.conjugate(), z, D, ell, g0) - ref) < 1e-11
        # gamma~ stepped against v_F: P = -Delta, Q = z, R = -Delta*
        ref = _rk4(-D, z, -D.conjugate(), ell, g0)
        assert abs(oracle.step(-D, z, -D.conjugate(), ell, g0) - ref) < 1e-11


def test_step_bulk_fixed_point_closed_form():
    # homogeneous solution gamma = i Delta / (eps + sqrt(eps^2 + |Delta|^2))
    for D in (0.27, 0.2 + 0.1j, -0.05j):
        for eps in (0.05, 0.3, 2.0):
            gh = 1j * D / (eps + math.sqrt(eps ** 2 + abs(D) ** 2))
            assert abs(oracle.step(D.conjugate() if isinstance(D, complex) else D, 1j * eps, D, 0.37, gh) - gh) < 1e-15
            # far from the fixed point the step contracts toward it
            g1 = oracle.step(complex(D).conjugate(), 1j * eps, D, 400.0, 0.9 + 0.1j)
            assert abs(g1 - gh) < 1e-12


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------
def test_mask_area_and_chords_approach_shape_area():
    for p in (W.disc(8.0, 64, n_angles=8, n_energies=2), W.diamond(12.0, 64, n_angles=8, n_energies=2)):
        g = oracle.OracleGeom(p)
        m = g.mask()
        # grid points on an edge count as inside: O(perimeter h / area) excess
        assert abs(m.sum() * p["h"] ** 2 / g.area - 1) < 0.04
        L = g.lines()
        off = 0
        for q in range(g.n_pairs):
            nl = L["l_hi"][q] - L["l_lo"][q] + 1
            chords = (L["smax"] - L["smin"])[off:off + nl]
            off += nl
            assert abs(chords.sum() * p["h"] / g.area - 1) < 0.01


def test_chord_endpoints_on_boundary():
    p = W.polygon([0.0, 7.0, 9.0, 2.0], [0.0, -1.0, 6.0, 8.0], 0.25, n_angles=12, n_energies=2)
    g = oracle.OracleGeom(p)
    L = g.lines()
    w, vh, _ = g.quadrature()
    Ox = p["x0"] + 0.5 * p["nx"] * p["h"] + p["lattice_ox"] * p["h"]
    Oy = p["y0"] + 0.5 * p["ny"] * p["h"] + p["lattice_oy"] * p["h"]
    vx, vy = np.array(p["vx"]), np.array(p["vy"])
    ex_, ey_ = np.roll(vx, -1) - vx, np.roll(vy, -1) - vy
    ln = np.hypot(ex_, ey_)
    nx_, ny_ = ey_ / ln, -ex_ / ln
    off = 0
    for q in range(g.n_pairs):
        e = vh[q]
        for l in range(L["l_lo"][q], L["l_hi"][q] + 1):
            i = off + l - L["l_lo"][q]
            for s in (L["smin"][i], L["smax"][i]):
                x = Ox - l * p["h"] * e[1] + s * e[0]
                y = Oy + l * p["h"] * e[0] + s * e[1]
                sd = np.max((x - vx) * nx_ + (y - vy) * ny_)
                assert abs(sd) < 1e-10
        off += L["l_hi"][q] - L["l_lo"][q] + 1


def test_ghost_map_brute_force():
    p = W.disc(3.3, 20, margin=0.6, n_angles=4, n_energies=1)
    g = oracle.OracleGeom(p)
    m = g.mask()
    gh = g.ghost()
    inside = [(j, i) for j in range(p["ny"]) for i in range(p["nx"]) if m[j, i]]
    for jj in range(p["ny"] + 2):
        for ii in range(p["nx"] + 2):
            v = gh[jj, ii]
            if v < 0:
                continue
            i, j = ii - 1, jj - 1
            best = min(inside, key=lambda q: ((q[1] - i) ** 2 + (q[0] - j) ** 2, q[0] * p["nx"] + q[1]))
            assert v == best[0] * p["nx"] + best[1]


def test_links_reflect_exactly_on_square():
    # On an axis-aligned square with N divisible by 4 the specular partner of
    # phi_k is again on the grid (-phi or pi - phi): every link has a single
    # non-zero angle weight, on that partner.
    p = W.square(10.0, 40, n_angles=16, n_energies=1)
    g = oracle.OracleGeom(p)
    lk = g.links()
    w, vh, _ = g.quadrature()
    N = p["n_angles"]
    angle_of_line = np.repeat(np.arange(N), [0] * 0 + [int(x) for x in np.diff(_ang_line_off(g))])
    for A in range(lk["w"].shape[0]):
        k = angle_of_line[A]
        ws = {}
        for q in range(4):
            ws[lk["angle"][A, q]] = ws.get(lk["angle"][A, q], 0.0) + lk["w"][A, q]
        big = [a for a, v in ws.items() if v > 1e-9]
        assert len(big) == 1
        a = big[0]
        # reflected direction is a mirror image of v_k in x or y
        v, u = vh[k], vh[a]
        assert (abs(u[0] + v[0]) < 1e-12 and abs(u[1] - v[1]) < 1e-12) or \
               (abs(u[0] - v[0]) < 1e-12 and abs(u[1] + v[1]) < 1e-12)
        assert abs(lk["w"][A].sum() - 1) < 1e-12


def _ang_line_off(g):
    L = g.lines()
    nl = L["l_hi"] - L["l_lo"] + 1
    N = g.N
    return np.concatenate([[0], np.cumsum([nl[k % g.n_pairs] for k in range(N)])])


def _link_shape(kind):
    """Grain, and the outward normal of the grain at a boundary point P with
    the part it lies on (None where the normal is ambiguous: polygon vertices)."""
    if kind == "disc":
        p = W.disc(12.0, 96, n_angles=64, n_energies=1)

        def normal(P):
            d = P - np.array([p["disc_cx"], p["disc_cy"]])
            return d / np.hypot(*d), 0
        return p, normal
    if kind == "polygon":
        rng = np.random.default_rng(11)
        while True:  # a seeded strictly convex heptagon
            vx, vy = W.random_convex_polygon(rng, 11.0, 7)
            e = np.diff(np.stack([vx, vy], axis=1), axis=0, append=[[vx[0], vy[0]]])
            if np.min(e[:, 0] * np.roll(e[:, 1], -1) - e[:, 1] * np.roll(e[:, 0], -1)) > 1.0:
                break
        p = W.polygon(vx, vy, 0.25, n_angles=48, n_energies=1)
        V = np.stack([vx, vy], axis=1)

        def normal(P):
            if np.min(np.hypot(*(V - P).T)) < 1e-6:
                return None, None
            best, nrm = np.inf, None
            for i in range(len(V)):
                a, b = V[i], V[(i + 1) % len(V)]
                e = b - a
                s = np.clip(np.dot(P - a, e) / np.dot(e, e), 0.0, 1.0)
                d = np.hypot(*(a + s * e - P))
                if d < best:  # counter-clockwise vertices: the outward normal is (e_y, -e_x)
                    best, nrm = d, np.array([e[1], -e[0]]) / np.hypot(*e)
            return nrm, 0
        return p, normal
    r_out, r_in = 12.0, 5.0
    p = W.annulus(r_out, r_in, 96, n_angles=64, n_energies=1)

    def normal(P):
        d = P / np.hypot(*P)
        # on the hole the grain's outward normal points into the hole
        return (d, 0) if np.hypot(*P) > 0.5 * (r_out + r_in) else (-d, 1)
    return p, normal


@pytest.mark.parametrize("kind", ["disc", "polygon", "annulus"])
def test_link_weights_interpolate_affine_exits(kind):
    """Sec. 3.1 and Fig. riccati_fig_A: the entry value of gamma is the exit
    value along the specularly reflected incoming direction, interpolated
    linearly in the Fermi angle and in the lattice-line coordinate.  With exit
    values affine in (angle index j, lattice line l), f = B j + C l, the 4-tap
    gather must return B u + C sum_a w_a c_a exactly, where the reflection
    point, the normal, u = psi N / 2 pi and c_a = (P - O).e_perp(phi_a) / h are
    recomputed here from circle and edge geometry.  Exchanging the two angle
    weights or the two line weights of a link breaks the identity (checked
    below on the same links)."""
    p, normal = _link_shape(kind)
    g = oracle.OracleGeom(p)
    N, npair, h = p["n_angles"], g.n_pairs, p["h"]
    O = np.array([p["x0"] + 0.5 * p["nx"] * h + p["lattice_ox"] * h,
                  p["y0"] + 0.5 * p["ny"] * h + p["lattice_oy"] * h])
    phi = 2 * np.pi * np.arange(N) / N
    vh = np.stack([np.cos(phi), np.sin(phi)], axis=1)
    L = g.lines()
    lk = g.links()
    chorded = set(zip(L["pair"].tolist(), L["l"].tolist()))
    line_off = np.concatenate([[0], np.cumsum(np.bincount(L["pair"], minlength=npair))])
    B, C = 0.731, -1.377

    def lattice_line_ok(pa, l, part):
        """Lattice line l of pair pa carries a chord whose end (in either
        direction of travel) lies on `part`."""
        if (pa, l) not in chorded:
            return False
        if kind != "annulus":
            return True
        d = abs(np.dot(O + l * h * np.array([-vh[pa, 1], vh[pa, 0]]), np.array([-vh[pa, 1], vh[pa, 0]])))
        return d < 5.0 - 1e-9 if part == 1 else d < 12.0 - 1e-9

    checked, swap_a_fail, swap_l_fail, A = 0, 0, 0, 0
    for k in range(N):
        pk = k % npair
        epar, eperp = vh[pk], np.array([-vh[pk, 1], vh[pk, 0]])
        for Lc in range(line_off[pk], line_off[pk + 1]):
            row = A
            A += 1
            s_in = L["smin"][Lc] if k < npair else L["smax"][Lc]
            P = O + L["l"][Lc] * h * eperp + s_in * epar
            n, part = normal(P)
            if n is None:
                continue
            v = vh[k]
            vin = v - 2.0 * np.dot(v, n) * n
            u = (math.atan2(vin[1], vin[0]) % (2 * np.pi)) * N / (2 * np.pi)
            j0 = math.floor(u)
            wa = u - j0
            cs, ok = [], True
            for j in (j0, j0 + 1):
                pa = j % N % npair
                c = float(np.dot(P - O, np.array([-vh[pa, 1], vh[pa, 0]]))) / h
                cs.append(c)
                ok &= all(lattice_line_ok(pa, math.floor(c) + b, part) for b in (0, 1))
            if not ok:
                continue
            want = B * u + C * ((1 - wa) * cs[0] + wa * cs[1])
            ta, tl, tw = lk["angle"][row], lk["line"][row], lk["w"][row]
            jj = ta + N * np.round((u - ta) / N)  # unwrapped next to u
            assert np.all(np.abs(jj - u)[tw > 1e-12] <= 1 + 1e-9)
            got = float(np.sum(tw * (B * jj + C * tl)))
            assert abs(got - want) < 1e-10, (kind, k, Lc, got, want)
            checked += 1
            # the same gather with the angle weights, or the line weights, exchanged
            lo_a = jj < u
            w_a = np.where(lo_a, 1 - wa, wa)
            sw_a = tw / w_a * np.where(lo_a, wa, 1 - wa)
            if abs(float(np.sum(sw_a * (B * jj + C * tl))) - want) > 1e-6:
                swap_a_fail += 1
            sw_l = tw.copy()
            for q in (0, 2):  # taps (2a, 2a+1) are the lower and upper line of angle a
                c = cs[0] if jj[q] < u else cs[1]
                wl = c - math.floor(c)
                if 1e-3 < abs(wl - 0.5) < 0.5 - 1e-3 and tw[q] > 0:
                    sw_l[q], sw_l[q + 1] = tw[q] / (1 - wl) * wl, tw[q + 1] / wl * (1 - wl)
            if abs(float(np.sum(sw_l * (B * jj + C * tl))) - want) > 1e-6:
                swap_l_fail += 1
    assert A == lk["w"].shape[0]
    assert checked > 0.5 * A, (checked, A)
    assert swap_a_fail > 0.9 * checked and swap_l_fail > 0.9 * checked, (swap_a_fail, swap_l_fail, checked)


# ---------------------------------------------------------------------------
# Sweep pins
# ---------------------------------------------------------------------------
def _bulk_gamma(D, eps):
    return 1j * D / (eps + np.sqrt(eps ** 2 + abs(D) ** 2))


@pytest.mark.parametrize("shape", ["square", "disc", "polygon"])
def test_bulk_s_wave_maps_to_itself(shape):
    """P1: uniform real s-wave Delta at its bulk value, A = 0: specular
    reflection maps bulk to bulk, so gamma is the homogeneous solution at every
    sample and the gap equation returns Delta (Eq. gapeq_fixpoint)."""
    t, ne, N = 0.5, 16, 32
    kw = dict(pairing=0, t=t, n_angles=N, n_energies=ne)
    p = {"square": lambda: W.square(12.0, 48, **kw),
         "disc": lambda: W.disc(7.0, 48, **kw),
         "polygon": lambda: W.polygon([0.0, 7.0, 9.0, 2.0], [0.0, -1.0, 6.0, 8.0], 0.3, **kw)}[shape]()
    d0 = oracle.bulk_gap(0, t, ne, N)
    g = oracle.OracleGeom(p)
    delta = np.full((p["ny"], p["nx"]), d0, complex)
    m = g.mask().astype(bool)
    ex = None
    for it in range(3):
        im, ex2, gam = g.sweep(delta, None, g.matsubara(), 0, ex, want_gammas=True)
        eps = t * (np.arange(ne) + 0.5)
        np.testing.assert_allclose(gam[0], np.broadcast_to(_bulk_gamma(d0, eps), gam[0].shape), atol=1e-13)
        np.testing.assert_allclose(gam[1], np.broadcast_to(np.conj(_bulk_gamma(d0, eps)), gam[1].shape), atol=1e-13)
        ex = ex2
        out = g.outputs(g.rotate_back(im), delta, None)
        assert np.max(np.abs(out["delta_new"][m] - d0)) < 1e-12
        assert np.max(np.abs(out["j"])) < 1e-12


def test_bulk_d_wave_axis_square_no_pair_breaking():
    """d_{x2-y2} in an axis-aligned square: the [100] edges map eta to itself,
    so the bulk state survives repeated sweeps through the boundary links."""
    t, ne, N = 0.3, 20, 32
    p = W.square(10.0, 40, pairing=1, t=t, n_angles=N, n_energies=ne)
    d0 = oracle.bulk_gap(1, t, ne, N)
    g = oracle.OracleGeom(p)
    delta = np.full((p["ny"], p["nx"]), d0, complex)
    m = g.mask().astype(bool)
    ex = None
    for it in range(3):
        out = g.full_sweep(delta, None, ex)
        ex = out["exit"]
        assert np.max(np.abs(out["delta_new"][m] - d0)) < 1e-12


def test_bulk_free_energy_matches_FEbulk():
    """P5: uniform Delta: F(R) equals the bulk free energy (Eq. FEbulk) at
    every grain point, s- and d-wave."""
    for pairing, t, ne, N in ((0, 0.5, 16, 32), (1, 0.2, 40, 32)):
        p = W.disc(6.0, 40, pairing=pairing, t=t, n_angles=N, n_energies=ne)
        g = oracle.OracleGeom(p)
        d0 = 0.9 * oracle.bulk_gap(pairing, t, ne, N)
        delta = np.full((p["ny"], p["nx"]), d0, complex)
        out = g.full_sweep(delta)
        w, vh, eta = g.quadrature()
        eps = t * (np.arange(ne) + 0.5)
        dk = np.abs(d0 * eta)[:, None]
        Om = np.sqrt(dk ** 2 + eps[None, :] ** 2)
        feb = np.sum(w * (dk[:, 0] ** 2 * math.log(t) + t * np.sum(dk ** 4 / (eps * (Om + eps) ** 2), axis=1)))
        m = g.mask().astype(bool)
        assert np.max(np.abs(out["F"][m] - feb)) < 1e-12
        assert abs(out["F_total"] - feb) < 1e-12


def test_uniform_superflow_current_closed_form():
    """P4: uniform Delta and uniform A after one sweep from fresh boundary
    values: g = -pi z / Omega with z = i eps_n + sigma v.A (Eilenberger bulk
    solution), so j = sigma (t/pi) sum_k w_k v_k sum_n 2 Re g (Eq. current_density)."""
    t, ne, N = 0.4, 12, 16
    for sigma in (-1, 1):
        p = W.disc(5.0, 32, pairing=0, t=t, n_angles=N, n_energies=ne, charge_sign=sigma)
        g = oracle.OracleGeom(p)
        d0 = 0.2
        A = np.array([0.03, -0.02])
        delta = np.full((p["ny"], p["nx"]), d0, complex)
        out = g.full_sweep(delta, W.uniform_field(p, *A))
        w, vh, eta = g.quadrature()
        eps = t * (np.arange(ne) + 0.5)
        a = sigma * (vh @ A)
        z = 1j * eps[None, :] + a[:, None]
        Om = np.sqrt(d0 ** 2 - z ** 2)
        gg = -np.pi * z / Om
        Sg = np.sum(2 * gg.real, axis=1)
        jref = sigma * t / np.pi * (w * Sg) @ vh
        m = g.mask().astype(bool)
        assert np.max(np.abs(out["j"][m] - jref)) < 1e-12


def test_linear_response_yoshida():
    """Small A: j = -2 <v (v.A) Y>, Y = t sum_n |Delta|^2/Omega^3 (linear
    response, Eqs. linearcurrent with the Yoshida function), error O(A^3)."""
    t, ne, N = 0.4, 40, 32
    p = W.disc(5.0, 24, pairing=1, t=t, n_angles=N, n_energies=ne)
    g = oracle.OracleGeom(p)
    w, vh, eta = g.quadrature()
    d0 = 0.22
    eps = t * (np.arange(ne) + 0.5)
    Y = t * np.sum((d0 * eta[:, None]) ** 2 / ((d0 * eta[:, None]) ** 2 + eps ** 2) ** 1.5, axis=1)
    errs = []
    m = g.mask().astype(bool)
    for s in (1e-2, 5e-3):
        A = s * np.array([1.0, 0.4])
        out = g.full_sweep(np.full((p["ny"], p["nx"]), d0, complex), W.uniform_field(p, *A))
        jlin = -2 * (w * Y * (vh @ A)) @ vh
        errs.append(np.max(np.abs(out["j"][m] - jlin)) / np.linalg.norm(jlin))
    assert errs[0] < 1e-3
    # absolute error O(A^3) -> relative error O(A^2): halving A quarters it
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_propagator_normalisation_and_tilde_symmetry():
    """P8: g^2 - f f~ = -pi^2 (Eq. norm) and gamma~(phi) = conj gamma(phi+pi)
    (Eq. symmetries) for an inhomogeneous Delta with a vector potential,
    across sweeps that use the boundary links."""
    t, ne, N = 0.3, 6, 16
    p = W.polygon([0.0, 6.0, 7.0, 1.0], [0.0, -1.0, 5.0, 6.0], 0.3, pairing=1, t=t,
                  n_angles=N, n_energies=ne, flux_quanta=1.0)
    g = oracle.OracleGeom(p)
    delta = W.vortex_delta(p, 0.2, [(3.0, 2.0)], [-1], seed=3, rel_noise=0.1)
    aind = W.uniform_field(p, 0.01, 0.02)
    ex = None
    for it in range(3):
        im, ex, gam = g.sweep(delta, aind, g.matsubara(), 0, ex, want_gammas=True)
    ga, gt = gam[0], gam[1]
    den = 1 + ga * gt
    gg = -1j * np.pi * (1 - ga * gt) / den
    ff = -2j * np.pi * ga / den
    fft = 2j * np.pi * gt / den
    assert np.max(np.abs(gg * gg - ff * fft + np.pi ** 2)) < 1e-10
    # angle k sample s and angle k+N/2 share the lattice points
    off = np.concatenate([[0], np.cumsum([g.n_samples_all // N] * N)]) if False else None
    half = g.n_samples_all // 2
    np.testing.assert_allclose(gt[:half], np.conj(ga[half:]), atol=1e-12)
    np.testing.assert_allclose(gt[half:], np.conj(ga[:half]), atol=1e-12)


def test_segments_against_rk4_brute_force():
    """P9: on a tiny grain, gamma at every sample equals an RK4 integration
    (2000 substeps per segment) of Eq. riccati with the half-step
    coefficients of App. C (linear interpolation between samples,
    nearest-sample values on the end segments), entry = homogeneous solution."""
    t, ne, N = 0.5, 2, 4
    p = W.disc(1.6, 8, pairing=0, t=t, n_angles=N, n_energies=ne, flux_quanta=0.7)
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
                gm = _rk4(np.conj(Dc), z0 + ac, Dc, ell, gm, n=2000)
                assert abs(gm - gam[0][off + q, n]) < 1e-10
        off += ns


# ---------------------------------------------------------------------------
# Rotate back (Sec. 3.1)
# ---------------------------------------------------------------------------
def test_rotate_back_reproduces_linear_images():
    p = W.disc(6.0, 40, n_angles=8, n_energies=1)
    g = oracle.OracleGeom(p)
    L = g.lines()
    w, vh, eta = g.quadrature()
    N = p["n_angles"]
    h = p["h"]
    Ox = p["x0"] + 0.5 * p["nx"] * h + p["lattice_ox"] * h
    Oy = p["y0"] + 0.5 * p["ny"] * h + p["lattice_oy"] * h
    # image = x-coordinate of each sample for every angle (SF slot)
    imgs = []
    for k in range(N):
        q = k % g.n_pairs
        e = vh[q]
        off = int(sum(L["l_hi"][:q] - L["l_lo"][:q] + 1))
        for l in range(L["l_lo"][q], L["l_hi"][q] + 1):
            i = off + l - L["l_lo"][q]
            for mm in range(L["m0"][i], L["m1"][i] + 1):
                x = Ox - l * h * e[1] + mm * h * e[0]
                imgs.append([0, 0, 0, x])
    acc = g.rotate_back(np.array(imgs))
    X, Y = W.grid_xy(p)
    m = g.mask().astype(bool)
    r = np.hypot(X, Y)
    interior = m & (r < 6.0 - 2 * h)
    np.testing.assert_allclose(acc[4][interior], X[interior], atol=1e-12)


# ---------------------------------------------------------------------------
# Vector potential (App. D)
# ---------------------------------------------------------------------------
def _G_quadrature(m, n, h):
    f = lambda y, x: math.log(((x + h * m) ** 2 + (y + h * n) ** 2))  # noqa: E731
    if m == 0 and n == 0:
        # log singularity at the origin: integrate in polar pieces over the square
        tot = 0.0
        for k in range(4):
            a0 = k * math.pi / 2
            for (lo, hi) in ((a0, a0 + math.pi / 4), (a0 + math.pi / 4, a0 + math.pi / 2)):
                def rmax(th):
                    return (h / 2) / max(abs(math.cos(th)), abs(math.sin(th)))
                val, _ = integrate.dblquad(lambda r, th: math.log(r * r) * r, lo, hi, 0, rmax,
                                           epsabs=1e-14, epsrel=1e-13)
                tot += val
        return tot / (4 * math.pi)
    val, _ = integrate.dblquad(f, -h / 2, h / 2, -h / 2, h / 2, epsabs=1e-14, epsrel=1e-13)
    return val / (4 * math.pi)


@pytest.mark.parametrize("m,n,h", [(0, 0, 0.3), (1, 0, 0.3), (2, 3, 0.25), (7, 1, 0.5), (0, 5, 0.2)])
def test_greens_closed_form_vs_quadrature(m, n, h):
    assert abs(oracle.greens(m, n, h) - _G_quadrature(m, n, h)) < 1e-10 * max(1.0, h * h)


def test_vector_potential_direct_vs_fft():
    p = W.disc(4.0, 20, n_angles=4, n_energies=1, kappa=3.0)
    g = oracle.OracleGeom(p)
    rng = np.random.default_rng(5)
    j = rng.standard_normal((p["ny"], p["nx"], 2))
    m = g.mask().astype(bool)
    j[~m] = 0
    a = g.vector_potential(j)
    jc = j - j[m].mean(axis=0)
    jc[~m] = 0
    n = p["nx"]
    G = np.array([[oracle.greens(abs(u), abs(v), p["h"]) for u in range(-n + 1, n)] for v in range(-n + 1, n)])
    ref = np.zeros_like(a)
    for c in range(2):
        full = np.real(np.fft.ifft2(np.fft.fft2(G, (3 * n, 3 * n)) * np.fft.fft2(jc[..., c], (3 * n, 3 * n))))
        ref[..., c] = -full[n - 1:2 * n - 1, n - 1:2 * n - 1] / 9.0
    np.testing.assert_allclose(a, ref, atol=1e-12)


# ---------------------------------------------------------------------------
# LDOS (Sec. 2): interior of a homogeneous s-wave grain is Dynes-BCS.
# ---------------------------------------------------------------------------
def test_ldos_homogeneous_dynes():
    p = W.disc(6.0, 32, pairing=0, t=0.5, n_angles=16, n_energies=1)
    g = oracle.OracleGeom(p)
    d0 = 0.25
    e = np.linspace(-0.5, 0.5, 9)
    dl = 0.02
    z = e + 1j * dl
    im, ex = g.sweep(np.full((p["ny"], p["nx"]), d0, complex), None, z, 1, None)
    acc = g.rotate_back(im, 1, len(e))
    ref = np.real(z / np.sqrt(z * z - d0 ** 2 + 0j) * np.sign(np.real(z) + 1e-300))
    ref = np.real(-1j * z / np.sqrt(d0 ** 2 - z ** 2))
    m = g.mask().astype(bool)
    for c in range(len(e)):
        assert np.max(np.abs(acc[c][m] - ref[c])) < 1e-12


def test_zero_bias_state_at_110_edge_scales_inverse_broadening():
    """P7: d_{x2-y2} grain with [110] edges (square rotated by 45 deg): every
    trajectory sees eta change sign on reflection, so the zero-energy LDOS at
    the edge is far above the normal state and grows as the broadening delta
    shrinks (a bound state); a [100] edge (unrotated square) keeps the
    d-wave bulk value (no peak)."""
    kw = dict(pairing=1, t=0.5, n_angles=32, n_energies=1)
    side = 24.0
    res = {}
    for name in ("110", "100"):
        p = W.diamond(side, 96, **kw) if name == "110" else W.square(side, 68, **kw)
        g = oracle.OracleGeom(p)
        d = np.full((p["ny"], p["nx"]), 0.22, complex)
        X, Y = W.grid_xy(p)
        h = p["h"]
        if name == "110":
            r = side / math.sqrt(2)
            u = np.abs(X) + np.abs(Y)
            sel = (u <= r + 1e-9) & (u > r - 1.2 * h) & (np.abs(X) > r / 4) & (np.abs(Y) > r / 4)
        else:
            mx = np.maximum(np.abs(X), np.abs(Y))
            sel = (mx > side / 2 - h) & (np.minimum(np.abs(X), np.abs(Y)) < side / 4)
        res[name] = [np.median(g.ldos(d, None, [0.0], dl, n_burnin=40)[0][0][sel]) for dl in (0.02, 0.01)]
    assert res["110"][0] > 5.0
    assert res["110"][1] / res["110"][0] > 1.4
    assert res["100"][0] < 0.5 and res["100"][1] < res["100"][0]


# ---------------------------------------------------------------------------
# Self-consistency loop (Algorithm 1 with the Picard step, App. E)
# ---------------------------------------------------------------------------
def test_c1_picard_converges_to_bulk():
    """P3: s-wave square from a noisy bulk guess: the global error (Eq.
    global_error) falls and Delta approaches the bulk root of the gap equation."""
    p, d0, _ = W.c1_square_s()
    g = oracle.OracleGeom(p)
    m = g.mask().astype(bool)
    r = g.picard(d0, 50)
    hist = r["history"]
    assert hist[49] < hist[10] < hist[1] < hist[0]
    assert hist[49] < 3e-5
    db = oracle.bulk_gap(0, p["t"], p["n_energies"], p["n_angles"])
    assert np.max(np.abs(r["delta"][m] - db)) < 2e-3


# ---------------------------------------------------------------------------
# Gauge covariance (Eqs. gaugetransformation, phase): A -> A + grad L together
# with Delta -> Delta exp(2 i sigma L) leaves g, j and |Delta_new| unchanged in
# the continuum; the discrete scheme must reproduce this to O(h^2).
# ---------------------------------------------------------------------------
def test_gauge_covariance_second_order():
    errs = []
    for n in (32, 64):
        p = W.disc(4.0, n, margin=0.2, pairing=0, t=0.5, n_angles=16, n_energies=4,
                   charge_sign=-1, flux_quanta=0.3)
        g = oracle.OracleGeom(p)
        X, Y = W.grid_xy(p)
        lam = 0.25 * np.sin(0.5 * X) * np.cos(0.4 * Y)
        grad = np.stack([0.125 * np.cos(0.5 * X) * np.cos(0.4 * Y),
                         -0.1 * np.sin(0.5 * X) * np.sin(0.4 * Y)], axis=-1)
        delta = 0.25 * (1 + 0.2 * np.cos(0.6 * X + 0.3 * Y)) + 0j
        delta2 = delta * np.exp(2j * p["charge_sign"] * lam)
        res = []
        for d, a in ((delta, np.zeros_like(grad)), (delta2, grad)):
            ex = None
            for it in range(12):
                out = g.full_sweep(d, a, ex)
                ex = out["exit"]
            res.append(out)
        # interior points: the end segments (nearest-sample values) and the
        # ghost-filled stencils make the boundary layer only first order
        sel = g.mask().astype(bool) & (np.hypot(X, Y) < 3.0)
        dj = np.max(np.abs(res[0]["j"][sel] - res[1]["j"][sel]))
        dd = np.max(np.abs(np.abs(res[0]["delta_new"][sel]) - np.abs(res[1]["delta_new"][sel])))
        dF = np.max(np.abs(res[0]["F"][sel] - res[1]["F"][sel]))
        errs.append((dj, dd, dF))
    for c in range(3):
        assert 3.0 < errs[0][c] / errs[1][c] < 5.5
    assert errs[1][0] < 3e-4 and errs[1][1] < 1e-4


# ---------------------------------------------------------------------------
# P11: charge conservation at self-consistency.  The Eilenberger equation
# conserves the current only when Delta solves the gap equation (Sec. 2):
# after Picard convergence the divergence of j in the interior is orders of
# magnitude below that of a non-self-consistent field, and what remains is set
# by the Fermi-surface quadrature (it falls with the angle count, not with h).
# ---------------------------------------------------------------------------
def _rms_divergence(p, j, sel):
    h = p["h"]
    dv = np.zeros(j.shape[:2])
    dv[1:-1, 1:-1] = (j[1:-1, 2:, 0] - j[1:-1, :-2, 0] + j[2:, 1:-1, 1] - j[:-2, 1:-1, 1]) / (2 * h)
    return float(np.sqrt(np.mean(dv[sel] ** 2)))


def test_current_is_conserved_at_self_consistency():
    out = {}
    for n, N in ((24, 16), (24, 32), (48, 32)):
        p = W.disc(4.0, n, margin=0.2, pairing=0, t=0.5, n_angles=N, n_energies=6, flux_quanta=1.0,
                   charge_sign=-1)
        g = oracle.OracleGeom(p)
        X, Y = W.grid_xy(p)
        sel = g.mask().astype(bool) & (np.hypot(X, Y) < 2.5)
        d0 = W.noisy_delta(p, 0.26, 0.2, seed=5)
        res = g.picard(d0, 150, update_a=False)
        assert res["history"][-1] < 1e-6
        j = res["last"]["j"]
        scale = float(np.max(np.hypot(j[..., 0], j[..., 1])))
        out[(n, N)] = (_rms_divergence(p, j, sel) / scale, _rms_divergence(p, g.full_sweep(d0)["j"], sel) / scale)
    for conv, noisy in out.values():
        assert conv < 3e-3 * noisy
    assert out[(24, 32)][0] < out[(24, 16)][0] / 3           # set by the angular quadrature
    assert 0.5 < out[(48, 32)][0] / out[(24, 32)][0] < 2.0    # not by the grid spacing
