"""ctypes front end of the plain FP64 C oracle.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product package never
imports this module, and this module imports nothing from the product.

Parameters are plain dicts with the keys of the ``or_params`` struct (the same
keys the product's ``sc_params`` uses), so a test can hand one dict to both.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_last_error.restype = ctypes.c_char_p
        L.or_geom_create.restype = ctypes.c_void_p
        L.or_geom_create.argtypes = [ctypes.c_void_p]
        L.or_geom_free.argtypes = [ctypes.c_void_p]
        L.or_geom_area.restype = ctypes.c_double
        L.or_geom_area.argtypes = [ctypes.c_void_p]
        for name in ("or_geom_info", "or_geom_mask", "or_geom_ghost", "or_geom_lines",
                     "or_geom_links", "or_geom_chords", "or_external_a", "or_geom_quadrature", "or_sample_fields", "or_sweep",
                     "or_rotate_back", "or_outputs", "or_vector_potential", "or_sweep_subset"):
            getattr(L, name).restype = ctypes.c_int
        L.or_norm_D.restype = ctypes.c_double
        L.or_norm_D.argtypes = [ctypes.c_double, ctypes.c_int]
        L.or_greens.restype = ctypes.c_double
        L.or_greens.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.or_bulk_gap.restype = ctypes.c_double
        L.or_bulk_gap.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.or_quad_weight.restype = ctypes.c_double
        L.or_quad_weight.argtypes = [ctypes.c_int, ctypes.c_int]
        L.or_geom_set_energy_weights.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        _lib = L
    return _lib


class _Part(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("add", ctypes.c_int32),
        ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("r", ctypes.c_double),
        ("n_vert", ctypes.c_int32),
        ("vx", ctypes.POINTER(ctypes.c_double)), ("vy", ctypes.POINTER(ctypes.c_double)),
    ]


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("h", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
        ("shape_kind", ctypes.c_int32),
        ("disc_cx", ctypes.c_double), ("disc_cy", ctypes.c_double), ("disc_r", ctypes.c_double),
        ("n_vert", ctypes.c_int32),
        ("vx", ctypes.POINTER(ctypes.c_double)), ("vy", ctypes.POINTER(ctypes.c_double)),
        ("pairing", ctypes.c_int32), ("crystal_rotation", ctypes.c_double),
        ("t", ctypes.c_double), ("flux_quanta", ctypes.c_double),
        ("gauge_cx", ctypes.c_double), ("gauge_cy", ctypes.c_double),
        ("kappa", ctypes.c_double), ("charge_sign", ctypes.c_int32),
        ("n_angles", ctypes.c_int32), ("n_energies", ctypes.c_int32),
        ("lattice_ox", ctypes.c_double), ("lattice_oy", ctypes.c_double),
        ("stepper", ctypes.c_int32),
        ("n_components", ctypes.c_int32), ("pairings", ctypes.c_int32 * 4), ("tc_ratios", ctypes.c_double * 4),
        ("n_parts", ctypes.c_int32), ("parts", ctypes.POINTER(_Part)),
        ("gauge", ctypes.c_int32),
    ]


GAUGES = {"symmetric": 0, "landau": 1, "solenoid": 2}
PART_KINDS = {"disc": 0, "polygon": 1}


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _cplx_to_f64(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)


def matsubara(t, n_e):
    """Positive Matsubara energies i*eps_n, eps_n = pi T (2n+1) = t (n + 1/2)
    in units of 2 pi kB Tc (Sec. 2, below Eq. symmetries)."""
    return 1j * t * (np.arange(n_e) + 0.5)


def norm_D(t, n_e):
    return lib().or_norm_D(float(t), int(n_e))


def greens(m, n, h):
    return lib().or_greens(int(m), int(n), float(h))


def bulk_gap(pairing, t, n_e, n_angles):
    return lib().or_bulk_gap(int(pairing), float(t), int(n_e), int(n_angles))


def quad_weight(k, n):
    return lib().or_quad_weight(int(k), int(n))


STEPPERS = {"closed": 0, "midpoint": 1}


def ozaki_poles(n):
    """Ozaki's continued-fraction poles of the Fermi function (Ozaki, PRB 75,
    035123 (2007); the energy sum of Sec. 3.1): the 2n x 2n symmetric
    tridiagonal matrix with zero diagonal and off-diagonal 1/(2 sqrt((2m-1)(2m+1)))
    has eigenvalues +-b_p; z_p = 1/b_p and R_p = v_p[0]^2/(4 b_p^2) give
    1/(1 + e^x) = 1/2 - sum_p R_p [1/(x - i z_p) + 1/(x + i z_p)].
    Returns z (ascending) and R."""
    M = 2 * n
    B = np.zeros((M, M))
    m = np.arange(1, M)
    off = 1.0 / (2.0 * np.sqrt((2 * m - 1.0) * (2 * m + 1.0)))
    B[m - 1, m] = off
    B[m, m - 1] = off
    w, v = np.linalg.eigh(B)
    pos = w > 0
    b = w[pos]
    z = 1.0 / b
    R = v[0, pos] ** 2 / (4.0 * b * b)
    o = np.argsort(z)
    return z[o], R[o]


def ozaki_energies(t, n):
    """Positive energies (units of 2 pi kB Tc) and weights of the Ozaki sum:
    T sum_n F(i eps_n) -> sum_p R_p T F(i T z_p) (+ the mirrored pole), so
    eps_p = t z_p / (2 pi)."""
    z, R = ozaki_poles(n)
    return t * z / (2.0 * math.pi), R


def step_midpoint(P, Q, R, ell, ga):
    """Implicit midpoint step (App. C, Eq. riccati_midpoint) of
    d gamma/ds = i (P gamma^2 + 2 Q gamma + R) over a length ell."""
    L = lib()
    arr = [np.array([complex(v).real, complex(v).imag]) for v in (P, Q, R, ga)]
    out = np.zeros(2)
    L.or_step_midpoint(_p(arr[0]), _p(arr[1]), _p(arr[2]), ctypes.c_double(ell), _p(arr[3]), _p(out))
    return complex(out[0], out[1])


def step(P, Q, R, ell, ga):
    L = lib()
    arr = [np.array([complex(v).real, complex(v).imag]) for v in (P, Q, R, ga)]
    out = np.zeros(2)
    L.or_step(_p(arr[0]), _p(arr[1]), _p(arr[2]), ctypes.c_double(ell), _p(arr[3]), _p(out))
    return complex(out[0], out[1])


class OracleGeom:
    """Geometry, lattices and boundary links of one grain, plus the sweep."""

    def __init__(self, prm):
        self.prm = dict(prm)
        L = lib()
        vx = np.ascontiguousarray(prm.get("vx", [0.0]), dtype=np.float64)
        vy = np.ascontiguousarray(prm.get("vy", [0.0]), dtype=np.float64)
        self._vx, self._vy = vx, vy
        s = _Params()
        for name, _ in _Params._fields_:
            if name in ("vx", "vy"):
                continue
            if name == "n_vert":
                s.n_vert = len(prm.get("vx", [])) if prm.get("shape_kind", 0) == 1 else 0
                continue
            if name == "stepper":
                s.stepper = STEPPERS[prm.get("stepper", "closed")]
                continue
            if name in ("n_components", "pairings", "tc_ratios", "n_parts", "parts"):
                continue
            if name == "gauge":
                s.gauge = GAUGES[prm.get("gauge", "symmetric")]
                continue
            if name == "pairing" and prm.get("components"):
                s.pairing = int(prm["components"][0][0])
                continue
            setattr(s, name, prm[name])
        s.vx = vx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s.vy = vy.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        comps = prm.get("components") or [(prm["pairing"], 1.0)]
        s.n_components = len(comps)
        for c, (pairing, tcr) in enumerate(comps):
            s.pairings[c] = int(pairing)
            s.tc_ratios[c] = float(tcr)
        self.C = len(comps)
        parts = prm.get("parts") or []
        self._parts = (_Part * max(1, len(parts)))()
        self._part_arrays = []
        for k, q in enumerate(parts):
            P = self._parts[k]
            P.kind = PART_KINDS[q["kind"]]
            P.add = 1 if q.get("add", True) else 0
            if q["kind"] == "disc":
                P.cx, P.cy, P.r = float(q["cx"]), float(q["cy"]), float(q["r"])
            else:
                ax = np.ascontiguousarray(q["vx"], np.float64)
                ay = np.ascontiguousarray(q["vy"], np.float64)
                self._part_arrays += [ax, ay]
                P.n_vert = len(ax)
                P.vx = ax.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                P.vy = ay.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s.n_parts = len(parts)
        s.parts = ctypes.cast(self._parts, ctypes.POINTER(_Part))
        self._s = s
        h = L.or_geom_create(ctypes.byref(s))
        if not h:
            raise ValueError("oracle geometry: " + L.or_last_error().decode())
        self._h = ctypes.c_void_p(h)
        info = np.zeros(6, np.int64)
        L.or_geom_info(self._h, _p(info))
        self.n_pairs, self.n_lines, self.n_samples, self.n_in = (int(v) for v in info[:4])
        self.n_lines_all, self.n_samples_all = int(info[4]), int(info[5])
        self.nx, self.ny = prm["nx"], prm["ny"]
        self.N = prm["n_angles"]
        self.n_e = prm["n_energies"]
        self.energy_sum = prm.get("energy_sum", "matsubara")
        if self.energy_sum == "ozaki":
            eps, w = ozaki_energies(prm["t"], self.n_e)
            self._eps = eps
            self._ewt = np.ascontiguousarray(w)
            D = math.log(prm["t"]) + prm["t"] * float(np.sum(w / eps))
            L.or_geom_set_energy_weights(self._h, _p(self._ewt), self.n_e, ctypes.c_double(D))
            self.normD = D
        elif self.energy_sum != "matsubara":
            raise ValueError("energy_sum must be 'matsubara' or 'ozaki'")

    def __del__(self):
        try:
            lib().or_geom_free(self._h)
        except Exception:
            pass

    # ---- geometry dumps -------------------------------------------------
    @property
    def area(self):
        return lib().or_geom_area(self._h)

    def mask(self):
        m = np.zeros(self.nx * self.ny, np.uint8)
        lib().or_geom_mask(self._h, _p(m))
        return m.reshape(self.ny, self.nx)

    def ghost(self):
        g = np.zeros((self.nx + 2) * (self.ny + 2), np.int32)
        lib().or_geom_ghost(self._h, _p(g))
        return g.reshape(self.ny + 2, self.nx + 2)

    def lines(self):
        np_ = self.n_pairs
        l_lo = np.zeros(np_, np.int32)
        l_hi = np.zeros(np_, np.int32)
        n = self.n_lines
        smin, smax = np.zeros(n), np.zeros(n)
        m0, m1 = np.zeros(n, np.int32), np.zeros(n, np.int32)
        lib().or_geom_lines(self._h, _p(l_lo), _p(l_hi), _p(smin), _p(smax), _p(m0), _p(m1))
        pair, l = np.zeros(n, np.int32), np.zeros(n, np.int32)
        lib().or_geom_chords(self._h, _p(pair), _p(l))
        return dict(l_lo=l_lo, l_hi=l_hi, smin=smin, smax=smax, m0=m0, m1=m1, pair=pair, l=l)

    def chords_per_pair(self):
        return np.bincount(self.lines()["pair"], minlength=self.n_pairs)

    def samples_per_pair(self):
        L = self.lines()
        ns = np.maximum(L["m1"] - L["m0"] + 1, 0)
        return np.bincount(L["pair"], weights=ns, minlength=self.n_pairs).astype(np.int64)

    def links(self):
        """Entry links of gamma, [angle][chord][4]: tap angle, lattice line l of
        the tapped chord, the tapped chord's index within its pair, weight."""
        n = 4 * self.n_lines_all
        ta, tl, tc, tw = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n)
        lib().or_geom_links(self._h, _p(ta), _p(tl), _p(tc), _p(tw))
        return dict(angle=ta.reshape(-1, 4), line=tl.reshape(-1, 4), chord=tc.reshape(-1, 4),
                    w=tw.reshape(-1, 4))

    def external_a(self, x, y):
        """External vector potential of the gauge at the points (x, y)."""
        xy = np.ascontiguousarray(np.stack([np.ravel(x), np.ravel(y)], axis=1), np.float64)
        A = np.zeros_like(xy)
        if lib().or_external_a(self._h, len(xy), _p(xy), _p(A)):
            raise RuntimeError(lib().or_last_error().decode())
        return A.reshape(np.shape(x) + (2,))

    def quadrature(self):
        w, vh, eta = np.zeros(self.N), np.zeros(2 * self.N), np.zeros(self.N)
        lib().or_geom_quadrature(self._h, _p(w), _p(vh), _p(eta))
        return w, vh.reshape(-1, 2), eta

    def sample_fields(self, delta, aind, pair):
        d = _cplx_to_f64(delta)
        a = None if aind is None else np.ascontiguousarray(aind, np.float64)
        ns = int(self.samples_per_pair()[pair])
        ds = np.zeros(2 * max(ns, 1))
        av = np.zeros(2 * max(ns, 1))
        rc = lib().or_sample_fields(self._h, _p(d), _p(a), int(pair), _p(ds), _p(av))
        if rc:
            raise RuntimeError(lib().or_last_error().decode())
        return ds[:2 * ns].view(np.complex128), av[:2 * ns].reshape(-1, 2)

    # ---- sweep ----------------------------------------------------------
    def sweep(self, delta, aind, z, mode=0, exit_in=None, want_gammas=False):
        """One sweep at complex energies z (no vector-potential term).
        Returns (images, exit_out[, gammas])."""
        d = _cplx_to_f64(delta)
        a = None if aind is None else np.ascontiguousarray(aind, np.float64)
        zz = _cplx_to_f64(np.asarray(z))
        n_e = len(z)
        ex_out = np.zeros(2 * 2 * self.n_lines_all * n_e)
        ex_in = None if exit_in is None else _cplx_to_f64(exit_in)
        nv = 4 if mode == 0 else n_e
        images = np.zeros(self.n_samples_all * nv)
        gam = np.zeros(2 * 2 * self.n_samples_all * n_e) if want_gammas else None
        rc = lib().or_sweep(self._h, _p(d), _p(a), _p(zz), int(n_e), int(mode), _p(ex_in),
                            _p(ex_out), _p(images), _p(gam))
        if rc:
            raise RuntimeError(lib().or_last_error().decode())
        ex = ex_out.view(np.complex128).reshape(2, self.n_lines_all, n_e)
        im = images.reshape(self.n_samples_all, nv)
        if want_gammas:
            return im, ex, gam.view(np.complex128).reshape(2, self.n_samples_all, n_e)
        return im, ex

    def sweep_subset(self, delta, aind, angles):
        """First-sweep energy sums of the listed angles only (Matsubara);
        returns a list of [samples][4] arrays, one per angle."""
        d = _cplx_to_f64(delta)
        a = None if aind is None else np.ascontiguousarray(aind, np.float64)
        z = _cplx_to_f64(self.matsubara())
        ang = np.ascontiguousarray(angles, np.int32)
        per_pair = [int(v) for v in self.samples_per_pair()]
        sizes = [per_pair[k % self.n_pairs] for k in angles]
        out = np.zeros(4 * sum(sizes))
        rc = lib().or_sweep_subset(self._h, _p(d), _p(a), _p(z), int(self.n_e), _p(ang), len(ang), _p(out))
        if rc:
            raise RuntimeError(lib().or_last_error().decode())
        res, o = [], 0
        for sz in sizes:
            res.append(out[4 * o:4 * (o + sz)].reshape(sz, 4))
            o += sz
        return res

    def rotate_back(self, images, mode=0, n_e=None):
        n_e = n_e if n_e is not None else self.n_e
        nout = 3 + 2 * self.C if mode == 0 else n_e
        acc = np.zeros(nout * self.nx * self.ny)
        im = np.ascontiguousarray(images, np.float64)
        lib().or_rotate_back(self._h, _p(im), int(mode), int(n_e), _p(acc))
        return acc.reshape(nout, self.ny, self.nx)

    def outputs(self, acc, delta, aind):
        """Delta_new (per component: [C, ny, nx] when C > 1), j, F(R), F_total, eps_G."""
        d = _cplx_to_f64(delta)
        a = None if aind is None else np.ascontiguousarray(aind, np.float64)
        npts = self.nx * self.ny
        dn = np.zeros(2 * npts * self.C)
        j = np.zeros(2 * npts)
        F = np.zeros(npts)
        sc = np.zeros(2)
        accf = np.ascontiguousarray(acc, np.float64)
        lib().or_outputs(self._h, _p(accf), _p(d), _p(a), _p(dn), _p(j), _p(F), _p(sc))
        shape = (self.C, self.ny, self.nx) if self.C > 1 else (self.ny, self.nx)
        return dict(delta_new=dn.view(np.complex128).reshape(shape),
                    j=j.reshape(self.ny, self.nx, 2), F=F.reshape(self.ny, self.nx),
                    F_total=float(sc[0]), eps_G=float(sc[1]))

    def vector_potential(self, j):
        jj = np.ascontiguousarray(j, np.float64)
        a = np.zeros(2 * self.nx * self.ny)
        lib().or_vector_potential(self._h, _p(jj), _p(a))
        return a.reshape(self.ny, self.nx, 2)

    # ---- composed steps -------------------------------------------------
    def matsubara(self):
        """The positive energies of the energy sums, times i: Matsubara
        energies or Ozaki's poles."""
        if self.energy_sum == "ozaki":
            return 1j * self._eps
        return matsubara(self.prm["t"], self.n_e)

    def full_sweep(self, delta, aind=None, exit_in=None):
        """Sweep at the positive Matsubara energies + outputs (Algorithm 1 body)."""
        im, ex = self.sweep(delta, aind, self.matsubara(), 0, exit_in)
        acc = self.rotate_back(im, 0)
        out = self.outputs(acc, delta, aind)
        out["exit"] = ex
        out["acc"] = acc
        out["images"] = im
        return out

    def picard(self, delta0, n_iter, aind0=None, update_a=True):
        """Fixed-point iteration of Algorithm 1 with the Picard step (alpha = 1):
        Delta <- Delta_new, A_ind <- from j, boundary values carried over."""
        delta = np.array(delta0, dtype=np.complex128)
        aind = None if aind0 is None else np.array(aind0, np.float64)
        kappa = self.prm["kappa"]
        use_a = update_a and kappa > 0 and math.isfinite(kappa)
        if use_a and aind is None:
            aind = np.zeros((self.ny, self.nx, 2))
        exit_in = None
        hist = []
        out = None
        for _ in range(n_iter):
            out = self.full_sweep(delta, aind, exit_in)
            hist.append(out["eps_G"])
            exit_in = out["exit"]
            delta = out["delta_new"]
            if use_a:
                aind = self.vector_potential(out["j"])
        return dict(delta=delta, aind=aind, history=np.array(hist), last=out, exit=exit_in)

    def self_consistency(self, delta0, n_iter, params, aind0=None):
        """Algorithm 1 with an accelerator of App. E (oracle/accel.py): each
        iteration sweeps with the current (Delta, A_ind), forms g(x) =
        (Delta_new, kappa^2 A from j) and takes the accelerator's step; boundary
        values are carried over."""
        from . import accel
        kappa = self.prm["kappa"]
        use_a = kappa > 0 and math.isfinite(kappa)
        delta = np.array(delta0, dtype=np.complex128)
        aind = np.zeros((self.ny, self.nx, 2)) if use_a and aind0 is None else (
            None if aind0 is None else np.array(aind0, np.float64))
        m = self.mask().astype(bool)
        acc = accel.Accelerator(params)
        ex = None
        hist = []
        for _ in range(n_iter):
            out = self.full_sweep(delta, aind, ex)
            ex = out["exit"]
            hist.append(out["eps_G"])
            a_new = self.vector_potential(out["j"]) if use_a else None
            x = accel.pack(delta, aind, m, kappa)
            g = accel.pack(out["delta_new"], a_new, m, kappa)
            delta, aind = accel.unpack(acc.step(x, g), delta, aind, m, kappa)
        return dict(delta=delta, aind=aind, history=np.array(hist), exit=ex, accelerator=acc)

    def ldos(self, delta, aind, energies, broadening, n_burnin=20, tol=1e-10):
        """LDOS N(R, eps)/N_F = -<Im g^R>/pi (Sec. 2) at eps + i*broadening,
        boundary values burnt in with Delta, A frozen."""
        z = np.asarray(energies, np.float64) + 1j * broadening
        ex = None
        for it in range(max(1, n_burnin)):
            im, ex2 = self.sweep(delta, aind, z, 1, ex)
            done = ex is not None and np.max(np.abs(ex2 - ex)) < tol
            ex = ex2
            if done:
                break
        acc = self.rotate_back(im, 1, len(z))
        return acc, ex
