"""C-ABI checks that need no GPU: the library loads, exports every symbol of
include/sc.h, validates parameters, and its host-side discretisation (mask,
nearest-grain-point map, rotated lattices, chords, specular links) equals the
oracle's, decision for decision."""
import os
import re

import math

import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import sc
from paper_2205_15000_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sc_[a-z0-9_]+)\s*\(", txt)))


def test_header_symbols_exported():
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(sc.lib, n), n
    assert sorted(sc.EXPORTED) == names


def test_version_and_defaults():
    assert "sm_103a" in sc.sc_version()
    p = sc.sc_params_default()
    assert p.n_angles == 32 and p.charge_sign == -1 and p.precision == sc.SC_PREC_FP32
    assert abs(p.lattice_ox - 0.1) < 1e-15 and abs(p.lattice_oy - 0.2) < 1e-15


@pytest.mark.parametrize("bad", [dict(n_angles=31), dict(t=0.0), dict(t=1.5), dict(n_energies=0),
                                 dict(charge_sign=2), dict(disc_r=-1.0), dict(disc_r=40.0),
                                 dict(h=-0.1)])
def test_invalid_params_rejected(bad):
    p = W.disc(5.0, 32, n_angles=8, n_energies=2)
    p.update(bad)
    with pytest.raises(sc.ScError) as ei:
        sc.Context(p, host_only=True)
    assert ei.value.status == sc.SC_EINVAL


def test_stepper_validated_and_default_closed():
    """sc_params.stepper: 0 (closed form, the default) or 1 (implicit midpoint);
    anything else is SC_EINVAL."""
    assert sc.sc_params_default().stepper == sc.SC_STEP_CLOSED
    p = W.disc(5.0, 32, n_angles=8, n_energies=2)
    q = sc.make_params(dict(p, stepper="midpoint"), host_only=True)
    assert q.stepper == sc.SC_STEP_MIDPOINT
    h = sc.sc_create(q)
    sc.sc_destroy(h)
    q.stepper = 2
    with pytest.raises(sc.ScError) as ei:
        sc.sc_create(q)
    assert ei.value.status == sc.SC_EINVAL


@pytest.mark.parametrize("n", [1, 4, 16, 100, 512])
def test_ozaki_poles_match_the_oracle(n):
    """The library's poles (bisection + inverse iteration) against the oracle's
    (LAPACK eigen-decomposition of the same matrix)."""
    z, R = sc.sc_ozaki_poles(n)
    zo, Ro = oracle.ozaki_poles(n)
    np.testing.assert_allclose(z, zo, rtol=1e-12)
    np.testing.assert_allclose(R, Ro, rtol=1e-9)


def test_ozaki_energy_grid_and_normalisation():
    p = W.disc(5.0, 32, n_angles=8, n_energies=12, t=0.3)
    p["energy_sum"] = "ozaki"
    ctx = sc.Context(p, host_only=True)
    eps, w = sc.sc_energy_grid(ctx.h, 12)
    eo, wo = oracle.ozaki_energies(0.3, 12)
    np.testing.assert_allclose(eps, eo, rtol=1e-12)
    np.testing.assert_allclose(w, wo, rtol=1e-9)
    g = oracle.OracleGeom(p)
    assert abs(ctx.info.norm_D - g.normD) < 1e-10
    q = dict(p, energy_sum="matsubara")
    ctx2 = sc.Context(q, host_only=True)
    eps2, w2 = sc.sc_energy_grid(ctx2.h, 12)
    np.testing.assert_allclose(eps2, 0.3 * (np.arange(12) + 0.5), rtol=1e-15)
    assert np.all(w2 == 1.0)
    assert abs(ctx2.info.norm_D - oracle.norm_D(0.3, 12)) < 1e-13
    with pytest.raises(sc.ScError) as ei:
        sc.Context(dict(p, n_energies=2000), host_only=True)
    assert ei.value.status == sc.SC_EINVAL


def test_nonconvex_polygon_rejected():
    p = W.polygon([0.0, 4.0, 2.0, 4.0, 0.0], [0.0, 0.0, 1.0, 4.0, 4.0], 0.25, n_angles=8, n_energies=2)
    with pytest.raises(sc.ScError) as ei:
        sc.Context(p, host_only=True)
    assert ei.value.status == sc.SC_EINVAL


def test_clockwise_polygon_rejected():
    p = W.polygon([0.0, 0.0, 4.0, 4.0], [0.0, 4.0, 4.0, 0.0], 0.25, n_angles=8, n_energies=2)
    with pytest.raises(sc.ScError):
        sc.Context(p, host_only=True)


def test_gauges_validated():
    """The solenoid gauge needs its flux line outside the grain (Eq.
    solenoid_gauge holds on the annulus R< <= r <= R>); unknown gauges and
    empty composites are refused."""
    with pytest.raises(sc.ScError):
        sc.Context(W.disc(4.0, 32, n_angles=8, n_energies=2, gauge="solenoid", flux_quanta=0.5), host_only=True)
    sc.Context(W.annulus(4.0, 1.5, 32, n_angles=8, n_energies=2, gauge="solenoid", flux_quanta=0.5), host_only=True)
    p = sc.make_params(W.disc(4.0, 32, n_angles=8, n_energies=2), host_only=True)
    p.gauge = 3
    with pytest.raises(sc.ScError):
        sc.sc_create(p)
    p = sc.make_params(W.annulus(4.0, 1.5, 32, n_angles=8, n_energies=2), host_only=True)
    p.n_parts = 0
    with pytest.raises(sc.ScError):
        sc.sc_create(p)


def test_compute_on_host_only_context_is_state_error():
    c = sc.Context(W.disc(5.0, 32, n_angles=8, n_energies=2), host_only=True)
    with pytest.raises(sc.ScError) as ei:
        sc.sc_riccati_sweep(c.h)
    assert ei.value.status == sc.SC_ESTATE


GEOMS = {
    "c1_square": lambda: W.c1_square_s()[0],
    "c2_diamond": lambda: W.c2_diamond_d()[0],
    "c4_disc": lambda: W.c4_disc_d()[0],
    "disc_small": lambda: W.disc(1.6, 8, n_angles=4, n_energies=2),
    "polygon": lambda: W.polygon([0.0, 7.0, 9.0, 2.0], [0.0, -1.0, 6.0, 8.0], 0.3, n_angles=12, n_energies=3),
    "triangle": lambda: W.polygon([0.0, 5.0, 1.0], [0.0, 1.0, 4.0], 0.2, n_angles=18, n_energies=2),
    "rotated": lambda: W.square(9.0, 50, rotation=0.3, n_angles=10, n_energies=2, crystal_rotation=0.1),
    # composite grains (Sec. 4): holes, unions, a removed polygon crossing the edge
    "annulus": lambda: W.annulus(6.0, 2.5, 48, margin=0.3, n_angles=24, n_energies=2),
    "square_hole": lambda: W.composite([W.disc_part((0, 0), 7.5), W.polygon_part(*W.regular_polygon((4.0, 0.5), 4, 3.0),
                                                                                 add=False)], 0.3, n_angles=16, n_energies=2),
    "two_discs": lambda: W.composite([W.disc_part((0, 0), 4.0), W.disc_part((5.0, 1.0), 3.0)], 0.25, n_angles=20,
                                     n_energies=2),
    "l_shape": lambda: W.composite([W.polygon_part([0, 6, 6, 0], [0, 0, 2, 2]), W.polygon_part([0, 2, 2, 0], [2, 2, 7, 7])],
                                   0.2, n_angles=16, n_energies=2),
    "bite": lambda: W.composite([W.polygon_part([0, 8, 8, 0], [0, 0, 8, 8]), W.disc_part((8.0, 4.0), 2.5, add=False),
                                 W.polygon_part(*W.regular_polygon((2.0, 6.0), 3, 2.5, rotation=0.05), add=False)],
                                0.25, n_angles=12, n_energies=2),
    "squid": lambda: W.composite([W.polygon_part([0, 100, 100, 0], [-5, -5, 5, 5]),
                                  W.polygon_part(*W.regular_polygon((50.0, 0.0), 8, 15.0)),
                                  W.disc_part((50.0, 0.0), 8.0, add=False)], 1.0, n_angles=8, n_energies=2),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_geometry_matches_oracle(name):
    p = GEOMS[name]()
    c = sc.Context(p, host_only=True)
    g = oracle.OracleGeom(p)
    assert c.info.n_pairs == g.n_pairs and c.info.n_lines == g.n_lines
    assert c.info.n_samples == g.n_samples and c.info.n_in == g.n_in
    assert abs(c.info.area - g.area) < 1e-12 * g.area
    np.testing.assert_array_equal(c.mask(), g.mask())
    np.testing.assert_array_equal(c.ghost(), g.ghost())
    a, b = c.lines(), g.lines()
    for k in ("l_lo", "l_hi", "m0", "m1", "pair", "l"):
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_allclose(a["smin"], b["smin"], atol=1e-12, rtol=0)
    np.testing.assert_allclose(a["smax"], b["smax"], atol=1e-12, rtol=0)
    la, lb = c.links(), g.links()
    # taps with vanishing weight may differ by rounding of a floor(); compare weighted maps
    assert la["w"].shape == lb["w"].shape
    for A in range(la["w"].shape[0]):
        da, db = {}, {}
        for q in range(4):
            ka = (la["angle"][A, q], la["line"][A, q], la["chord"][A, q])
            kb = (lb["angle"][A, q], lb["line"][A, q], lb["chord"][A, q])
            da[ka] = da.get(ka, 0.0) + la["w"][A, q]
            db[kb] = db.get(kb, 0.0) + lb["w"][A, q]
        keys = set(da) | set(db)
        for k in keys:
            assert abs(da.get(k, 0.0) - db.get(k, 0.0)) < 1e-12, (A, k)


def test_steps_per_sweep_count():
    p = W.c1_square_s()[0]
    c = sc.Context(p, host_only=True)
    L = c.lines()
    ns = np.maximum(L["m1"] - L["m0"] + 1, 0)
    assert c.info.steps_per_sweep == p["n_energies"] * int(np.sum(2 * (ns + 1)))
    assert c.info.points_per_sweep == 2 * p["n_energies"] * int(ns.sum())


@pytest.mark.parametrize("energy_sum", ["matsubara", "ozaki"])
def test_energy_count_from_cutoff(energy_sum):
    """n_energies = 0 takes the count from eps_cut: the Matsubara energies
    t (n + 1/2) below it, or the fewest Ozaki poles whose largest energy
    t z_max / 2 pi reaches it (counted here from the oracle's poles)."""
    t, cut = 0.1, 8.0
    base = W.disc(5.0, 32, n_angles=8, t=t, energy_sum=energy_sum)
    if energy_sum == "matsubara":
        expect = sum(1 for n in range(10000) if t * (n + 0.5) < cut)
    else:
        expect = next(n for n in range(1, 200) if t * oracle.ozaki_poles(n)[0][-1] / (2 * math.pi) >= cut)
        assert sc.sc_ozaki_poles_for_cutoff(t, cut) == expect
    c = sc.Context(dict(base, n_energies=0, eps_cut=cut), host_only=True)
    r = sc.Context(dict(base, n_energies=expect), host_only=True)
    assert c.info.steps_per_sweep == r.info.steps_per_sweep and c.info.norm_D == r.info.norm_D
    with pytest.raises(sc.ScError):
        sc.Context(dict(base, n_energies=0), host_only=True)


def test_given_mask_must_match_the_shape():
    p = W.annulus(6.0, 2.5, 48, margin=0.3, n_angles=8, n_energies=2)
    m = sc.Context(p, host_only=True).mask()
    sc.Context(dict(p, mask=m), host_only=True)
    bad = m.copy()
    bad[24, 24] ^= 1
    with pytest.raises(sc.ScError):
        sc.Context(dict(p, mask=bad), host_only=True)


@pytest.mark.parametrize("name", ["disc", "diamond", "annulus", "squid"])
def test_table_indices_validate(name):
    """Every index of the host tables lies inside the table it points into, and
    each kind of corruption (an image slot, a boundary tap, a lattice-line
    record) is caught -- on host_only contexts, whose tables never reach a GPU."""
    p = {"disc": lambda: W.disc(5.0, 40, n_angles=18, n_energies=4),
         "diamond": lambda: W.diamond(12.0, 48, n_angles=16, n_energies=4),
         "annulus": lambda: W.annulus(6.0, 2.5, 48, margin=0.3, n_angles=8, n_energies=2),
         "squid": GEOMS["squid"]}[name]()
    c = sc.Context(p, host_only=True)
    assert sc.sc_debug_validate_tables(c.h) == 0
    for which in (0, 1, 2):
        bad = sc.Context(p, host_only=True)
        sc.sc_debug_corrupt_table(bad.h, which)
        assert sc.sc_debug_validate_tables(bad.h) >= 1, which
    with pytest.raises(sc.ScError):
        sc.sc_debug_corrupt_table(c.h, 3)


def test_checked_library_exports_the_same_symbols():
    """The bounds-checked variant of the library (index checks compiled into the
    kernels) loads and exports every symbol of include/sc.h."""
    import ctypes
    from paper_2205_15000_b300 import build
    assert os.path.exists(build.LIB_CHECKED)
    L = ctypes.CDLL(build.LIB_CHECKED)
    for n in _declared():
        assert hasattr(L, n), n


def test_residual_history_arguments():
    """sc_get_history on a context with no residual computed yet: no records;
    a negative capacity, or a positive one without arrays, is refused."""
    import ctypes
    p = W.disc(5.0, 32, n_angles=8, n_energies=6, t=0.4)
    ctx = sc.Context(p, host_only=True)
    sw, eps = sc.sc_get_history(ctx.h)
    assert sw.size == 0 and eps.size == 0
    n = ctypes.c_int32(-1)
    assert sc.lib.sc_get_history(ctx.h, ctypes.byref(n), None, None) == sc.SC_EINVAL
    n = ctypes.c_int32(2)
    assert sc.lib.sc_get_history(ctx.h, ctypes.byref(n), None, None) == sc.SC_EINVAL
    assert sc.lib.sc_get_history(None, ctypes.byref(n), None, None) == sc.SC_EINVAL
    sc.sc_clear_history(ctx.h)
