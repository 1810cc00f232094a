"""Seeded synthetic workloads shaped like the paper's grains.

This module only builds inputs: grids, grain shapes, parameter dicts and
seeded initial order-parameter fields.  It holds none of the method's
arithmetic, so both the CUDA path and the oracle can be fed from it.

Workloads (grain sizes in xi0, energies in 2 pi kB Tc):
  c1_square_s   s-wave square, side 20, 64x64, 32 angles, 16 energies, t=0.5
  c2_diamond_d  d_{x2-y2} square rotated 45 deg (pair-breaking [110] edges),
                side 50, 256x256 over the bounding box, 128 angles, t=0.1,
                Matsubara cutoff 8 (= 16 pi kB Tc) -> 80 energies, 0.5 flux
                quanta, kappa=80
  c3_batch      64 seeded discs / convex polygons, radius 10-40, h=0.2
  c4_disc_d     d-wave disc radius 25, 128x128, 64 angles, t=0.2, one vortex
  c5_square_d   d-wave square side 200, 1024x1024, 256 angles, t=0.05 (160
                energies), 20 vortices, kappa=80
  annulus_d     d_{x2-y2} annulus R> = 25, R< = 10 (Sec. 5.1), 256x256, 128
                angles, t=0.1 (80 energies), solenoid gauge with half a flux
                quantum through the hole, no screening
"""
import math

import numpy as np

# parameter keys shared by the product's sc_params and the oracle's or_params
PARAM_KEYS = ("nx", "ny", "h", "x0", "y0", "shape_kind", "disc_cx", "disc_cy", "disc_r",
              "vx", "vy", "pairing", "crystal_rotation", "t", "flux_quanta", "gauge_cx",
              "gauge_cy", "kappa", "charge_sign", "n_angles", "n_energies", "lattice_ox",
              "lattice_oy")

PAIRING = {"s": 0, "dx2y2": 1, "dxy": 2, "g": 3}

# Bulk gap values used only to scale initial guesses (a wrong digit here
# changes the input, not the check).
BULK_GUESS = {("s", 0.5): 0.268717, ("dx2y2", 0.1): 0.240792, ("dx2y2", 0.2): 0.240128,
              ("dx2y2", 0.05): 0.240871}


def n_energies_for_cutoff(t, eps_cut=8.0):
    """Number of positive Matsubara energies t(n+1/2) below the cutoff."""
    return int(math.ceil(eps_cut / t - 0.5))


def ozaki_poles_for_cutoff(t, eps_cut=8.0):
    """Number of Ozaki poles whose largest energy t z_max/(2 pi) reaches the
    cutoff, z_max ~ 0.84 pi n^2: the Ozaki counterpart of n_energies_for_cutoff
    (at equal cutoff the Ozaki sum is the more accurate of the two)."""
    n = max(1, int(math.ceil(math.sqrt(2.0 * eps_cut / (0.84 * t)))))
    return n


def base_params(**kw):
    p = dict(nx=64, ny=64, h=20.0 / 64, x0=-10.0, y0=-10.0, shape_kind=1, disc_cx=0.0,
             disc_cy=0.0, disc_r=0.0, vx=[], vy=[], pairing=0, crystal_rotation=0.0, t=0.5,
             flux_quanta=0.0, gauge_cx=0.0, gauge_cy=0.0, kappa=0.0, charge_sign=-1,
             n_angles=32, n_energies=16, lattice_ox=0.1, lattice_oy=0.2)
    p.update(kw)
    return p


def square(side, n, center=(0.0, 0.0), rotation=0.0, **kw):
    """Square grain of the given side, rotated by `rotation` (radians), on an
    n x n grid covering its bounding box."""
    cx, cy = center
    half = side / 2.0
    corners = [(-half, -half), (half, -half), (half, half), (-half, half)]
    c, s = math.cos(rotation), math.sin(rotation)
    vx = [cx + c * x - s * y for x, y in corners]
    vy = [cy + s * x + c * y for x, y in corners]
    ext = max(max(vx) - min(vx), max(vy) - min(vy))
    h = ext / n
    return base_params(nx=n, ny=n, h=h, x0=cx - ext / 2, y0=cy - ext / 2, shape_kind=1, vx=vx,
                       vy=vy, gauge_cx=cx, gauge_cy=cy, **kw)


def diamond(side, n, center=(0.0, 0.0), **kw):
    """Square rotated by 45 degrees; its vertices lie on the axes."""
    cx, cy = center
    r = side / math.sqrt(2.0)
    vx = [cx + r, cx, cx - r, cx]
    vy = [cy, cy + r, cy, cy - r]
    ext = 2 * r
    return base_params(nx=n, ny=n, h=ext / n, x0=cx - r, y0=cy - r, shape_kind=1, vx=vx, vy=vy,
                       gauge_cx=cx, gauge_cy=cy, **kw)


def disc(radius, n, center=(0.0, 0.0), margin=0.0, **kw):
    cx, cy = center
    ext = 2 * radius + 2 * margin
    return base_params(nx=n, ny=n, h=ext / n, x0=cx - ext / 2, y0=cy - ext / 2, shape_kind=0,
                       disc_cx=cx, disc_cy=cy, disc_r=radius, gauge_cx=cx, gauge_cy=cy, **kw)


def polygon(vx, vy, h, margin=0.5, **kw):
    """Convex polygon (counter-clockwise) on a grid with spacing ~h covering it."""
    xlo, xhi, ylo, yhi = min(vx), max(vx), min(vy), max(vy)
    ext = max(xhi - xlo, yhi - ylo) + 2 * margin * h
    n = int(math.ceil(ext / h))
    hh = ext / n
    cx, cy = 0.5 * (xlo + xhi), 0.5 * (ylo + yhi)
    return base_params(nx=n, ny=n, h=hh, x0=cx - ext / 2, y0=cy - ext / 2, shape_kind=1,
                       vx=list(vx), vy=list(vy), gauge_cx=float(np.mean(vx)),
                       gauge_cy=float(np.mean(vy)), **kw)


def regular_polygon(center, n_edges, side_length, rotation=0.0):
    """Vertices (counter-clockwise) of a regular polygon: centre, number of
    edges, side length and rotation in units of a full turn (App. B's
    regular_polygon).  Unrotated, the first vertex lies on the -y side so that
    a square (n_edges 4) has edges parallel to the axes."""
    cx, cy = center
    R = side_length / (2.0 * math.sin(math.pi / n_edges))
    a0 = -math.pi / 2 - math.pi / n_edges + 2.0 * math.pi * rotation
    vx = [cx + R * math.cos(a0 + 2.0 * math.pi * k / n_edges) for k in range(n_edges)]
    vy = [cy + R * math.sin(a0 + 2.0 * math.pi * k / n_edges) for k in range(n_edges)]
    return vx, vy


def disc_part(center, radius, add=True):
    return dict(kind="disc", add=add, cx=float(center[0]), cy=float(center[1]), r=float(radius))


def polygon_part(vx, vy, add=True):
    return dict(kind="polygon", add=add, vx=[float(v) for v in vx], vy=[float(v) for v in vy])


def composite(parts, h, margin=1.0, gauge_center=None, **kw):
    """Composite grain (Sec. 4 and App. B): discs and convex polygons added and
    removed in the listed order.  The grid has spacing ~h and covers the added
    parts with `margin` grid points to spare; the gauge origin defaults to the
    centre of that box."""
    xs, ys = [], []
    for q in parts:
        if not q.get("add", True):
            continue
        if q["kind"] == "disc":
            xs += [q["cx"] - q["r"], q["cx"] + q["r"]]
            ys += [q["cy"] - q["r"], q["cy"] + q["r"]]
        else:
            xs += list(q["vx"])
            ys += list(q["vy"])
    xlo, xhi, ylo, yhi = min(xs), max(xs), min(ys), max(ys)
    ext = max(xhi - xlo, yhi - ylo) + 2 * margin * h
    n = int(math.ceil(ext / h))
    hh = ext / n
    cx, cy = 0.5 * (xlo + xhi), 0.5 * (ylo + yhi)
    gx, gy = gauge_center if gauge_center is not None else (cx, cy)
    return base_params(nx=n, ny=n, h=hh, x0=cx - ext / 2, y0=cy - ext / 2, shape_kind=2,
                       parts=[dict(q) for q in parts], gauge_cx=gx, gauge_cy=gy, **kw)


def annulus(r_out, r_in, n, center=(0.0, 0.0), margin=0.0, **kw):
    """Disc of radius r_out with a concentric hole of radius r_in (the annulus
    of Sec. 5.1) on an n x n grid over its bounding box (+ margin)."""
    cx, cy = center
    ext = 2 * r_out + 2 * margin
    return base_params(nx=n, ny=n, h=ext / n, x0=cx - ext / 2, y0=cy - ext / 2, shape_kind=2,
                       parts=[disc_part(center, r_out), disc_part(center, r_in, add=False)],
                       gauge_cx=cx, gauge_cy=cy, **kw)


def grid_xy(p):
    x = p["x0"] + (np.arange(p["nx"]) + 0.5) * p["h"]
    y = p["y0"] + (np.arange(p["ny"]) + 0.5) * p["h"]
    return np.meshgrid(x, y)


def noisy_delta(p, amplitude, rel_noise=0.05, seed=0):
    """amplitude * (1 + rel_noise * Z), Z complex standard normal (seeded)."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((p["ny"], p["nx"])) + 1j * rng.standard_normal((p["ny"], p["nx"]))) / math.sqrt(2)
    return amplitude * (1.0 + rel_noise * z)


def vortex_delta(p, amplitude, centers, windings, seed=None, rel_noise=0.0):
    """amplitude * exp(i sum_v w_v atan2(R - C_v)) (+ noise): the initial order
    parameter of the paper's configuration appendix."""
    X, Y = grid_xy(p)
    chi = np.zeros_like(X)
    for (cx, cy), w in zip(centers, windings):
        chi += w * np.arctan2(Y - cy, X - cx)
    d = amplitude * np.exp(1j * chi)
    if rel_noise and seed is not None:
        rng = np.random.default_rng(seed)
        d = d + amplitude * rel_noise * (rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)) / math.sqrt(2)
    return d


def uniform_field(p, ax, ay):
    a = np.zeros((p["ny"], p["nx"], 2))
    a[..., 0] = ax
    a[..., 1] = ay
    return a


# ---------------------------------------------------------------------------
# named configurations
# ---------------------------------------------------------------------------
def c1_square_s():
    p = square(20.0, 64, pairing=0, t=0.5, n_angles=32, n_energies=16, kappa=0.0)
    return p, noisy_delta(p, BULK_GUESS[("s", 0.5)], 0.05, seed=1), None


def c2_diamond_d(n=256, n_angles=128):
    t = 0.1
    p = diamond(50.0, n, pairing=1, t=t, n_angles=n_angles, n_energies=n_energies_for_cutoff(t),
                flux_quanta=0.5, kappa=80.0)
    return p, noisy_delta(p, BULK_GUESS[("dx2y2", 0.1)], 0.05, seed=2), None


def c4_disc_d(n=128, n_angles=64, seed=4):
    t = 0.2
    rng = np.random.default_rng(seed)
    r = 15.0 * math.sqrt(rng.uniform())
    th = rng.uniform(0, 2 * math.pi)
    p = disc(25.0, n, pairing=1, t=t, n_angles=n_angles, n_energies=n_energies_for_cutoff(t),
             kappa=0.0)
    d = vortex_delta(p, BULK_GUESS[("dx2y2", 0.2)], [(r * math.cos(th), r * math.sin(th))], [-1])
    return p, d, None


def c5_square_d(n=1024, n_angles=256, seed=5, n_vortex=20):
    t = 0.05
    p = square(200.0, n, pairing=1, t=t, n_angles=n_angles, n_energies=n_energies_for_cutoff(t),
               flux_quanta=20.0, kappa=80.0)
    rng = np.random.default_rng(seed)
    centers = []
    while len(centers) < n_vortex:
        c = rng.uniform(-85, 85, size=2)
        if all(math.hypot(c[0] - q[0], c[1] - q[1]) >= 15.0 for q in centers):
            centers.append((float(c[0]), float(c[1])))
    d = vortex_delta(p, BULK_GUESS[("dx2y2", 0.05)], centers, [-1] * n_vortex)
    return p, d, None


def annulus_d(n=256, n_angles=128, flux=0.5, seed=6):
    """The annulus of Sec. 5.1 (outer radius 25, inner 10) with d_{x2-y2}
    pairing at t = 0.1, in the solenoid gauge (Eq. solenoid_gauge)."""
    t = 0.1
    p = annulus(25.0, 10.0, n, pairing=1, t=t, n_angles=n_angles, n_energies=n_energies_for_cutoff(t),
                gauge="solenoid", flux_quanta=flux, kappa=0.0)
    return p, noisy_delta(p, BULK_GUESS[("dx2y2", 0.1)], 0.05, seed=seed), None


def random_convex_polygon(rng, radius, n_vert):
    ang = np.sort(rng.uniform(0, 2 * math.pi, n_vert))
    rad = radius * (1.0 + rng.uniform(-0.2, 0.2, n_vert))
    return list(rad * np.cos(ang)), list(rad * np.sin(ang))


def c3_batch(n_grains=64, seed=3, h=0.2, radius_range=(10.0, 40.0)):
    """Batched workload: seeded discs and convex polygons of uneven size,
    pairing, temperature, field and angle count."""
    rng = np.random.default_rng(seed)
    grains = []
    for g in range(n_grains):
        R = float(rng.uniform(*radius_range))
        pairing = int(rng.integers(0, 2))
        t = float(rng.uniform(0.05, 0.8))
        alpha = float(rng.uniform(0, 5))
        n_ang = int(rng.choice([64, 128, 192, 256]))
        ne = n_energies_for_cutoff(t)
        kw = dict(pairing=pairing, t=t, n_angles=n_ang, n_energies=ne, flux_quanta=alpha,
                  kappa=0.0)
        if rng.uniform() < 0.5:
            n = int(math.ceil(2 * R / h))
            p = disc(R, n, **kw)
        else:
            while True:
                vx, vy = random_convex_polygon(rng, R, int(rng.integers(3, 11)))
                # keep strictly convex, counter-clockwise polygons with a sane area
                cross = [(vx[(i + 1) % len(vx)] - vx[i]) * (vy[(i + 2) % len(vx)] - vy[(i + 1) % len(vx)])
                         - (vy[(i + 1) % len(vx)] - vy[i]) * (vx[(i + 2) % len(vx)] - vx[(i + 1) % len(vx)])
                         for i in range(len(vx))]
                if min(cross) > 1e-3 * R * R:
                    break
            p = polygon(vx, vy, h, **kw)
        guess = 0.27 if pairing == 0 else 0.24
        amp = guess * math.sqrt(max(1.0 - t, 0.05))
        grains.append((p, noisy_delta(p, amp, 0.05, seed=1000 + g), None))
    return grains
