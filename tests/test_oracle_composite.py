"""Pins of the oracle's composite grains (Sec. 4 and App. B: discs and convex
polygons added and removed in order) and of its three gauges (App. B;
Eq. solenoid_gauge; Sec. 5.1.2), against closed forms written here from
elementary geometry and from the paper's superflow equations (Eqs.
gaugetransformation, phase, linearcurrent, lFEkin), not from the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W


def _lens(r1, r2, d):
    """Area of the intersection of two discs at centre distance d."""
    a1 = r1 * r1 * math.acos((d * d + r1 * r1 - r2 * r2) / (2 * d * r1))
    a2 = r2 * r2 * math.acos((d * d + r2 * r2 - r1 * r1) / (2 * d * r2))
    return a1 + a2 - 0.5 * math.sqrt((-d + r1 + r2) * (d + r1 - r2) * (d - r1 + r2) * (d + r1 + r2))


def _area(parts, h=0.25):
    p = W.composite(parts, h, n_angles=4, n_energies=1)
    return oracle.OracleGeom(p).area


# ---------------------------------------------------------------------------
# areas (the flux-to-field conversion B = pi alpha / area uses them)
# ---------------------------------------------------------------------------
def test_area_annulus_and_square_hole():
    a = _area([W.disc_part((0, 0), 7.0), W.disc_part((0, 0), 3.0, add=False)])
    assert abs(a - math.pi * (49 - 9)) < 1e-11
    # the compound geometry of App. B: disc of radius 15 with a square hole of
    # side 5 centred 10 to the right of the disc centre
    vx, vy = W.regular_polygon((10.0, 0.0), 4, 5.0)
    a = _area([W.disc_part((0, 0), 15.0), W.polygon_part(vx, vy, add=False)])
    assert abs(a - (math.pi * 225 - 25)) < 1e-10


def test_area_overlapping_discs_and_l_shape():
    r1, r2, d = 4.0, 3.0, 5.0
    a = _area([W.disc_part((0, 0), r1), W.disc_part((d, 0), r2)])
    assert abs(a - (math.pi * (r1 * r1 + r2 * r2) - _lens(r1, r2, d))) < 1e-10
    # difference: the first disc minus the second
    a = _area([W.disc_part((0, 0), r1), W.disc_part((d, 0), r2, add=False)])
    assert abs(a - (math.pi * r1 * r1 - _lens(r1, r2, d))) < 1e-10
    # L-shape from two rectangles sharing part of an edge, and a part that
    # misses the grain leaves it unchanged
    parts = [W.polygon_part([0, 6, 6, 0], [0, 0, 2, 2]), W.polygon_part([0, 2, 2, 0], [2, 2, 7, 7]),
             W.disc_part((20, 20), 1.0, add=False)]
    assert abs(_area(parts) - 22.0) < 1e-12


def test_area_squid_geometry():
    """The SQUID-like grain of Sec. 4: a 100 x 10 bar, a regular octagon of
    side 15 centred on it, and a disc of radius 8 removed from the centre.
    The bar crosses the octagon between its two vertical edges (|y| < s/2)."""
    s = 15.0
    ox, oy = W.regular_polygon((50.0, 0.0), 8, s)
    parts = [W.polygon_part([0, 100, 100, 0], [-5, -5, 5, 5]), W.polygon_part(ox, oy),
             W.disc_part((50.0, 0.0), 8.0, add=False)]
    inr = s / (2 * math.tan(math.pi / 8))
    expect = 1000.0 + 2 * (1 + math.sqrt(2)) * s * s - 10.0 * 2 * inr - math.pi * 64
    assert abs(_area(parts, h=1.0) - expect) < 1e-9


# ---------------------------------------------------------------------------
# mask, chords and links of an annulus
# ---------------------------------------------------------------------------
R_OUT, R_IN = 6.0, 2.5


def _annulus(n=48, **kw):
    kw.setdefault("n_angles", 16)
    kw.setdefault("n_energies", 4)
    return W.annulus(R_OUT, R_IN, n, margin=0.3, **kw)


def test_annulus_mask_and_chords():
    p = _annulus()
    g = oracle.OracleGeom(p)
    X, Y = W.grid_xy(p)
    r = np.hypot(X, Y)
    np.testing.assert_array_equal(g.mask().astype(bool), (r <= R_OUT) & (r >= R_IN))
    L = g.lines()
    _, vh, _ = g.quadrature()
    h = p["h"]
    ox = p["x0"] + 0.5 * p["nx"] * h + p["lattice_ox"] * h
    oy = p["y0"] + 0.5 * p["ny"] * h + p["lattice_oy"] * h
    n_two = 0
    for q in range(g.n_pairs):
        ex, ey = vh[q]
        for l in range(L["l_lo"][q], L["l_hi"][q] + 1):
            sel = np.nonzero((L["pair"] == q) & (L["l"] == l))[0]
            bx, by = ox - l * h * ey, oy + l * h * ex
            s0 = -(bx * ex + by * ey)              # foot of the centre on the line
            b2 = bx * bx + by * by - s0 * s0       # squared distance of the line from the centre
            wo = math.sqrt(R_OUT ** 2 - b2)
            if b2 < R_IN ** 2:
                wi = math.sqrt(R_IN ** 2 - b2)
                expect = [(s0 - wo, s0 - wi), (s0 + wi, s0 + wo)]
                n_two += 1
            else:
                expect = [(s0 - wo, s0 + wo)]
            assert len(sel) == len(expect), (q, l)
            for c, (a, b) in zip(sel, expect):
                assert abs(L["smin"][c] - a) < 1e-12 and abs(L["smax"][c] - b) < 1e-12
    assert n_two > 0


def test_annulus_links_reflect_on_the_hole():
    """A chord that starts on the hole takes, as entry value, exits of chords
    that end on the hole next to its entry point, in the directions that
    reflect into it about the hole's normal (pointing into the hole), also
    where one of the two bracketing lattice lines passes beside the hole."""
    p = _annulus(n_angles=24)
    g = oracle.OracleGeom(p)
    L = g.lines()
    lk = g.links()
    _, vh, _ = g.quadrature()
    N, P, h = p["n_angles"], g.n_pairs, p["h"]
    ox = p["x0"] + 0.5 * p["nx"] * h + p["lattice_ox"] * h
    oy = p["y0"] + 0.5 * p["ny"] * h + p["lattice_oy"] * h
    first = np.searchsorted(L["pair"], np.arange(P))
    checked = 0
    row = 0
    for k in range(N):
        q = k % P
        chords = np.nonzero(L["pair"] == q)[0]
        for c in chords:
            s_in = L["smin"][c] if k < P else L["smax"][c]
            ex, ey = vh[q]
            l = L["l"][c]
            px, py = ox - l * h * ey + s_in * ex, oy + l * h * ex + s_in * ey
            r = math.hypot(px, py)
            if abs(r - R_IN) < 1e-9:
                nx_, ny_ = -px / r, -py / r          # the grain's outward normal
                vx, vy = vh[k]
                vn = vx * nx_ + vy * ny_
                ux, uy = vx - 2 * vn * nx_, vy - 2 * vn * ny_
                u = (math.atan2(uy, ux) % (2 * math.pi)) * N / (2 * math.pi)
                a0 = int(math.floor(u)) % N
                assert set(lk["angle"][row]) <= {a0, (a0 + 1) % N}
                for t in range(4):
                    if lk["w"][row, t] < 1e-12:
                        continue
                    j = lk["angle"][row, t]
                    cc = first[j % P] + lk["chord"][row, t]
                    assert L["l"][cc] == lk["line"][row, t]
                    jx, jy = vh[j % P]
                    s_out = L["smax"][cc] if j < P else L["smin"][cc]
                    qx = ox - L["l"][cc] * h * jy + s_out * jx
                    qy = oy + L["l"][cc] * h * jx + s_out * jy
                    # next to the entry: a line within h of it meets the circle within
                    # sqrt(2 r h) of it along the boundary, even at grazing incidence
                    assert math.hypot(qx - px, qy - py) < 1.5 * math.sqrt(2 * R_IN * h) + h
                    assert abs(math.hypot(qx, qy) - R_IN) < 1e-9      # on the hole
                checked += 1
            row += 1
    assert checked > 20


# ---------------------------------------------------------------------------
# gauges: circulation of the external vector potential (units A0 = Phi0/(pi xi0):
# the circulation around a flux Phi is pi Phi / Phi0)
# ---------------------------------------------------------------------------
def _circulation(g, cx, cy, rad, n=4000):
    th = (np.arange(n) + 0.5) * 2 * math.pi / n
    x, y = cx + rad * np.cos(th), cy + rad * np.sin(th)
    A = g.external_a(x, y)
    return float(np.sum(A[:, 0] * (-np.sin(th)) + A[:, 1] * np.cos(th)) * rad * 2 * math.pi / n)


@pytest.mark.parametrize("gauge", ["symmetric", "landau"])
def test_uniform_field_gauges(gauge):
    """Uniform field B = pi alpha / area: the circulation around any circle is
    B times its area, whatever the centre."""
    alpha = 1.7
    p = _annulus(flux_quanta=alpha, gauge=gauge)
    g = oracle.OracleGeom(p)
    B = math.pi * alpha / (math.pi * (R_OUT ** 2 - R_IN ** 2))
    for cx, cy, rad in ((0.0, 0.0, 3.0), (1.0, -2.0, 1.5), (-3.0, 2.5, 0.7)):
        assert abs(_circulation(g, cx, cy, rad) - B * math.pi * rad * rad) < 1e-9


def test_solenoid_gauge():
    """Eq. solenoid_gauge: the flux alpha Phi0 threads the hole only: the
    circulation around the hole is pi alpha at every radius, zero around a loop
    that does not enclose the flux line, and |A| = alpha / (2 r)."""
    alpha = -1.3
    p = _annulus(flux_quanta=alpha, gauge="solenoid")
    g = oracle.OracleGeom(p)
    for rad in (2.6, 4.0, 5.9):
        assert abs(_circulation(g, 0.0, 0.0, rad) - math.pi * alpha) < 1e-9
    assert abs(_circulation(g, 4.0, 1.0, 1.0)) < 1e-9
    A = g.external_a(np.array([3.0, 0.0]), np.array([0.0, -5.0]))
    np.testing.assert_allclose(np.hypot(A[:, 0], A[:, 1]), [abs(alpha) / 6.0, abs(alpha) / 10.0], rtol=1e-14)
    with pytest.raises(ValueError):   # the flux line inside the grain is refused
        oracle.OracleGeom(W.disc(4.0, 32, n_angles=4, n_energies=1, gauge="solenoid", flux_quanta=0.5))


# ---------------------------------------------------------------------------
# physics through the whole sweep
# ---------------------------------------------------------------------------
def _burnt_in(g, delta, aind, n=12):
    ex = None
    for _ in range(n):
        out = g.full_sweep(delta, aind, ex)
        ex = out["exit"]
    return out


def test_bulk_survives_holes_and_composites():
    """A uniform s-wave Delta at the bulk gap, A = 0, is a fixed point of
    repeated sweeps in an annulus and in a grain with a polygonal hole and a
    second added disc: every reflection, on an outer or an inner boundary,
    keeps the bulk solution."""
    t, ne, N = 0.5, 6, 16
    db = oracle.bulk_gap(0, t, ne, N)
    vx, vy = W.regular_polygon((1.0, 0.5), 5, 2.0, rotation=0.1)
    geoms = [_annulus(pairing=0, t=t, n_angles=N, n_energies=ne),
             W.composite([W.disc_part((0, 0), 5.0), W.disc_part((5.5, 1.0), 2.5),
                          W.polygon_part(vx, vy, add=False)], 0.25, pairing=0, t=t, n_angles=N,
                         n_energies=ne)]
    for p in geoms:
        g = oracle.OracleGeom(p)
        m = g.mask().astype(bool)
        ex = None
        for _ in range(2):
            out = g.full_sweep(np.full((p["ny"], p["nx"]), db, complex), None, ex)
            ex = out["exit"]
            assert np.max(np.abs(out["delta_new"][m] - db)) < 1e-12
            assert np.max(np.abs(out["j"])) < 1e-12


def _yosida(t, ne, d):
    """Y = pi T sum_n |Delta|^2 / Lambda_n^3 over all Matsubara energies below
    the cutoff (Eq. linearcurrent, both signs of eps_n)."""
    eps = t * (np.arange(ne) + 0.5)
    return t * float(np.sum(d * d / (eps * eps + d * d) ** 1.5))


def test_solenoid_annulus_linear_response():
    """s-wave annulus in the solenoid gauge with flux alpha and phase winding
    n: p_s = (n + alpha)/(2R) phi^ (units 2 pi kB Tc / v_F; Sec. 5.1.1 with
    e = sigma |e|, sigma = -1), so linear response gives the charge current
    j = sigma Y p_s (Eq. linearcurrent, units j0) and the kinetic free-energy
    density Y p_s^2 / 2 (Eq. lFEkin), Y the Yosida function at the bulk gap.
    The local forms hold up to nonlocal corrections of order (xi0/R)^2, a few
    per cent point by point at these radii, less on average.  The free energy
    of a wound state is measured from the matched state of the same winding,
    which cancels the offset of sampling the winding phase on the grid."""
    t, ne, N = 0.5, 6, 16
    db = oracle.bulk_gap(0, t, ne, N)
    Y = _yosida(t, ne, db)
    res = {}
    for wind, alpha in ((0, 0.0), (0, 0.2), (1, -1.0), (1, -0.8)):
        p = _annulus(n=64, pairing=0, t=t, n_angles=N, n_energies=ne, gauge="solenoid",
                     flux_quanta=alpha, charge_sign=-1)
        g = oracle.OracleGeom(p)
        X, Yg = W.grid_xy(p)
        delta = db * np.exp(1j * wind * np.arctan2(Yg, X))
        res[(wind, alpha)] = _burnt_in(g, delta, None, 10)
    r = np.hypot(X, Yg)
    m = g.mask().astype(bool)
    sel = m & (r > R_IN + 0.8) & (r < R_OUT - 0.8)
    phx, phy = -Yg / r, X / r
    for key, ref in (((0, 0.2), (0, 0.0)), ((1, -0.8), (1, -1.0))):
        wind, alpha = key
        ps = (wind + alpha) / (2 * r)
        out = res[key]
        jphi = out["j"][..., 0] * phx + out["j"][..., 1] * phy
        jrad = out["j"][..., 0] * X / r + out["j"][..., 1] * Yg / r
        ratio = jphi[sel] / (-Y * ps[sel])
        assert abs(np.mean(ratio) - 1.0) < 0.03 and np.all(np.abs(ratio - 1.0) < 0.12), ratio
        assert np.max(np.abs(jrad[sel])) < 0.05 * np.max(np.abs(Y * ps[sel]))
        dF = out["F"] - res[ref]["F"]
        assert abs(np.sum(dF[sel]) / np.sum(0.5 * Y * ps[sel] ** 2) - 1.0) < 0.05


def test_solenoid_matching_flux_is_a_gauge_transformation():
    """At alpha = sigma n the solenoid vector potential is grad(alpha phi / 2)
    and Delta exp(i n phi) is its gauge transform (Eq. gaugetransformation), so
    p_s = 0: the current and the free energy are those of the field-free state
    with real Delta, up to the discretisation (a few per cent of what one
    unmatched flux quantum drives), while the opposite flux drives p_s = 1/R."""
    t, ne, N = 0.5, 4, 16
    db = oracle.bulk_gap(0, t, ne, N)
    Y = _yosida(t, ne, db)
    p0 = _annulus(n=64, pairing=0, t=t, n_angles=N, n_energies=ne, charge_sign=-1)
    p1 = dict(p0, gauge="solenoid", flux_quanta=-1.0)
    X, Yg = W.grid_xy(p0)
    prof = db * (1 + 0.15 * np.cos(0.7 * X - 0.4 * Yg))
    wound = prof * np.exp(1j * np.arctan2(Yg, X))
    a = _burnt_in(oracle.OracleGeom(p0), prof + 0j, None, 10)
    b = _burnt_in(oracle.OracleGeom(p1), wound, None, 10)
    c = _burnt_in(oracle.OracleGeom(dict(p1, flux_quanta=1.0)), wound, None, 10)
    m = oracle.OracleGeom(p0).mask().astype(bool)
    r = np.hypot(X, Yg)
    sel = m & (r > R_IN + 0.7) & (r < R_OUT - 0.7)   # off the first-order boundary layer
    j_unit = Y / (2 * R_OUT)                 # |j| of p_s = 1/(2R) at the outer radius
    F_unit = 0.5 * Y / (2 * R_OUT) ** 2      # its kinetic free-energy density
    assert np.max(np.abs(b["j"][sel] - a["j"][sel])) < 0.05 * j_unit
    assert np.max(np.abs(b["j"][m] - a["j"][m])) < 0.15 * j_unit
    assert np.max(np.abs(np.abs(b["delta_new"][sel]) - np.abs(a["delta_new"][sel]))) < 0.02 * db
    assert abs(np.sum(b["F"][m] - a["F"][m])) < 0.05 * F_unit * m.sum()
    assert np.min(np.hypot(c["j"][m][:, 0], c["j"][m][:, 1])) > 0.5 * j_unit


def test_landau_equals_symmetric_after_gauge_transformation():
    """A_landau - A_symmetric = grad L with L = -B/2 (x - xg)(y - yg), so the
    landau gauge with Delta exp(2 i sigma L) reproduces the symmetric gauge's
    j, |Delta_new| and F to second order in h (Eqs. gaugetransformation, phase)."""
    errs = []
    for n in (32, 64):
        p = W.disc(4.0, n, margin=0.2, pairing=0, t=0.5, n_angles=16, n_energies=4, charge_sign=-1,
                   flux_quanta=1.2)
        q = dict(p, gauge="landau")
        X, Y = W.grid_xy(p)
        B = math.pi * 1.2 / (math.pi * 16.0)
        lam = -0.5 * B * X * Y
        delta = 0.25 * (1 + 0.2 * np.cos(0.6 * X + 0.3 * Y)) + 0j
        a = _burnt_in(oracle.OracleGeom(p), delta, None, 10)
        b = _burnt_in(oracle.OracleGeom(q), delta * np.exp(2j * p["charge_sign"] * lam), None, 10)
        # interior: the boundary layer is only first order
        sel = oracle.OracleGeom(p).mask().astype(bool) & (np.hypot(X, Y) < 2.0)
        errs.append((np.max(np.abs(a["j"][sel] - b["j"][sel])),
                     np.max(np.abs(np.abs(a["delta_new"][sel]) - np.abs(b["delta_new"][sel]))),
                     np.max(np.abs(a["F"][sel] - b["F"][sel]))))
    for c in range(3):
        assert 3.0 < errs[0][c] / errs[1][c] < 5.5, errs
    assert errs[1][0] < 1e-4
