"""Self-consistency accelerators of App. E, plain numpy -- test infrastructure
only (tests/, smoke(), bench.py's CPU-baseline leg).

The unknowns are concatenated into x = (Re Delta, Im Delta, kappa^2 A_x,
kappa^2 A_y) (Eq. x_concat): Delta over the grain's grid points, A_ind over the
whole grid (only with a finite kappa > 0), g(x) is one sweep's (Delta_new, kappa^2 A_new) and
d = g(x) - x (Eq. difference).  Each accelerator maps (x_i, d_i) to x_{i+1}:

  Picard     x+ = x + alpha d                                   (Eq. picard)
  Polyak     v+ = (1 - beta) v + alpha d,  x+ = x + v+,  v_0 = 0  (Eq. polyak)
  BB         alpha_{i+1} = alpha_i * s_i,  s = BB1 (i odd) / BB2 (i even),
             x+ = x + alpha_{i+1} d                              (Eq. barzilai_borwein)
  CongAcc    per component c: s = cos(m_c, d_c), alpha_c <- alpha_c k^s,
             w_c kept if s >= s_min else w* with cos(w* m + (1-w*) d, d) = s_min,
             m_c <- w_c m_c + (1 - w_c) d_c,  x_c+ = x_c + alpha_c m_c   (App. E, CongAcc)

Readings where the paper is silent: BB takes alpha_1 = step_size on the first
iteration (no d_{-1}), then clamps alpha to [step_size_min, step_size_max] and
keeps it when a BB denominator vanishes; CongAcc's first iteration keeps
alpha_c = step_size and takes m_c = d_c (w_0 = 0); a component whose d_c or m_c
has zero norm keeps its alpha_c and w_c; w* is found by 60 bisection steps on
[0, 1]; alpha_c is clamped like BB's.
"""
import math

import numpy as np

PICARD, POLYAK, BARZILAI_BORWEIN, CONGACC = 0, 1, 2, 3
NAMES = {"picard": PICARD, "polyak": POLYAK, "barzilai-borwein": BARZILAI_BORWEIN, "congacc": CONGACC}


def default_params(kind):
    """The defaults printed in the paper's listings for each accelerator."""
    kind = NAMES.get(kind, kind)
    p = dict(kind=kind, step_size=1.0, drag=0.5, step_size_factor=1.234, cos_similarity_min=0.7,
             step_size_max=100.0, step_size_min=0.001)
    if kind == POLYAK:
        p["step_size"] = 2.0
    elif kind == CONGACC:
        p["step_size"] = 0.5
    return p


def cos_sim(a, b):
    na, nb = math.sqrt(float(a @ a)), math.sqrt(float(b @ b))
    if na == 0.0 or nb == 0.0:
        return None
    return float(a @ b) / (na * nb)


class Accelerator:
    """State of one accelerator over a sequence of iterations; x and g are
    lists of the component vectors (1-D float64 arrays)."""

    def __init__(self, params):
        self.p = dict(params)
        self.i = 0
        self.v = None        # Polyak velocity
        self.d_prev = None   # BB: d_{i-1}
        self.alpha = self.p["step_size"]
        self.alpha_c = None  # CongAcc per component
        self.w_c = None
        self.m_c = None

    def _clamp(self, a):
        return min(max(a, self.p["step_size_min"]), self.p["step_size_max"])

    def step(self, x, g):
        p = self.p
        d = [gi - xi for xi, gi in zip(x, g)]
        kind = p["kind"]
        if kind == PICARD:
            xn = [xi + p["step_size"] * di for xi, di in zip(x, d)]
        elif kind == POLYAK:
            if self.v is None:
                self.v = [np.zeros_like(di) for di in d]
            self.v = [(1.0 - p["drag"]) * vi + p["step_size"] * di for vi, di in zip(self.v, d)]
            xn = [xi + vi for xi, vi in zip(x, self.v)]
        elif kind == BARZILAI_BORWEIN:
            if self.i >= 1:
                dc = np.concatenate(d)
                dp = np.concatenate(self.d_prev)
                dd = dc - dp
                q = abs(float(dp @ dd))
                if self.i % 2 == 1:  # BB1
                    den, num = q, float(dp @ dp)
                else:                # BB2
                    den, num = float(dd @ dd), q
                if den > 0.0:
                    self.alpha = self._clamp(self.alpha * num / den)
            self.d_prev = [di.copy() for di in d]
            xn = [xi + self.alpha * di for xi, di in zip(x, d)]
        elif kind == CONGACC:
            nc = len(d)
            if self.alpha_c is None:
                self.alpha_c = [p["step_size"]] * nc
                self.w_c = [0.0] * nc
                self.m_c = [np.zeros_like(di) for di in d]
            xn = []
            for c in range(nc):
                m, dc = self.m_c[c], d[c]
                if self.i >= 1:
                    s = cos_sim(m, dc)
                    if s is not None:
                        self.alpha_c[c] = self._clamp(self.alpha_c[c] * p["step_size_factor"] ** s)
                        if s < p["cos_similarity_min"]:
                            self.w_c[c] = self._similarity_weight(m, dc, p["cos_similarity_min"])
                w = self.w_c[c]
                self.m_c[c] = w * m + (1.0 - w) * dc
                xn.append(x[c] + self.alpha_c[c] * self.m_c[c])
        else:
            raise ValueError(kind)
        self.i += 1
        return xn

    @staticmethod
    def _similarity_weight(m, d, s_min):
        """w in [0, 1] with cos(w m + (1 - w) d, d) = s_min, by bisection
        (cos is 1 at w = 0 and below s_min at w = 1)."""
        lo, hi = 0.0, 1.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if cos_sim(mid * m + (1.0 - mid) * d, d) >= s_min:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)


def pack(delta, aind, mask, kappa):
    """x from the grid fields: Delta over the grain points (Re and Im of each
    order-parameter component), kappa^2 A_ind over the whole grid (the induced
    potential is a field on every grid point)."""
    m = mask.astype(bool)
    comps = delta if np.ndim(delta) == 3 else [delta]
    x = []
    for dc in comps:
        x += [np.ascontiguousarray(dc[m].real), np.ascontiguousarray(dc[m].imag)]
    if aind is not None and kappa > 0 and math.isfinite(kappa):
        x += [kappa ** 2 * aind[..., 0].ravel(), kappa ** 2 * aind[..., 1].ravel()]
    return x


def unpack(x, delta_like, aind_like, mask, kappa):
    """Grid fields from x; Delta outside the grain keeps its old values (the
    sweep never reads them: bilinear stencils there take the nearest grain
    point)."""
    m = mask.astype(bool)
    delta = np.array(delta_like, dtype=np.complex128)
    nc = delta.shape[0] if delta.ndim == 3 else 1
    for c in range(nc):
        dc = delta[c] if delta.ndim == 3 else delta
        dc[m] = x[2 * c] + 1j * x[2 * c + 1]
    aind = None if aind_like is None else np.array(aind_like, dtype=np.float64)
    if len(x) == 2 * nc + 2:
        aind[..., 0] = (x[2 * nc] / kappa ** 2).reshape(aind.shape[:2])
        aind[..., 1] = (x[2 * nc + 1] / kappa ** 2).reshape(aind.shape[:2])
    return delta, aind
