"""The allocation-free line sweep (sc_sweep_lines_noalloc) against the regular
context sweep (sc_riccati_sweep).

sc_sweep_lines_noalloc exists for callers that cannot allocate device memory
when they run a sweep (their device heap belongs to another allocator, or
they cannot afford cudaMalloc's implicit synchronisation).  It takes every
buffer from the caller and keeps its scratch in a static array inside the
library.  Here it gets the lattice samples of a grain, built from the
oracle's FP64 sample fields (and, for lines without samples, the field at the
chord midpoint), and must reproduce the context's FP32 sweeps (images and
exit values of every line) within the FP32 tolerances of the other GPU tests:
the first sweep from the homogeneous start, on two calls in a row since every
call reuses the same array; the second sweep from entry values gathered
through the context's boundary links; lines longer than the stated maximum
are skipped with NaN exits and leave every other line unchanged; and a call
after the first one does not take device memory, whatever its energy layout.

This file is named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_IMG = 1e-5   # relative to the largest image value
TOL_EXIT = 2e-5  # absolute, |gamma| <= 1


def _grain(name):
    if name == "disc_vortex":
        p = W.disc(5.0, 40, pairing=1, t=0.25, n_angles=18, n_energies=13, flux_quanta=1.0)
        d = W.vortex_delta(p, 0.22, [(1.0, -0.5)], [-1], seed=13, rel_noise=0.05)
        return p, d
    # has two lines without samples and a single longest line
    p = W.diamond(12.0, 48, pairing=1, t=0.3, n_angles=16, n_energies=40, flux_quanta=0.5)
    return p, W.noisy_delta(p, 0.23, 0.1, seed=12)


def _bilinear(p, ghost, f, x, y):
    """Bilinear value of the grid field f at (x, y), stencil points outside the
    grain replaced through the ghost map (the sampling reading of the sweep)."""
    h = p["h"]
    gx, gy = (x - p["x0"]) / h - 0.5, (y - p["y0"]) / h - 0.5
    i0, j0 = math.floor(gx), math.floor(gy)
    fx, fy = gx - i0, gy - j0
    v = 0.0
    flat = f.reshape(-1)
    for b in (0, 1):
        for a in (0, 1):
            w = (fx if a else 1 - fx) * (fy if b else 1 - fy)
            src = ghost[j0 + b + 1, i0 + a + 1]
            if w != 0.0:
                v += w * flat[src]
    return v


def _line_inputs(p, delta):
    """Samples and line table in the library's slot order (pairs, then lines,
    then samples), from the oracle's fields at the lattice samples; a line
    without samples holds its chord-midpoint value in its one slot."""
    g = oracle.OracleGeom(p)
    w, vh, eta = g.quadrature()
    L = g.lines()
    ghost = g.ghost()
    h = p["h"]
    O = np.array([p["x0"] + 0.5 * p["nx"] * h + p["lattice_ox"] * h,
                  p["y0"] + 0.5 * p["ny"] * h + p["lattice_oy"] * h])
    samples, slot0, ns_l, lens = [], [], [], []
    off = 0
    line = 0
    for q in range(g.n_pairs):
        ds, av = g.sample_fields(delta, None, q)
        a = p["charge_sign"] * (av @ vh[q])
        s = 0
        for l in range(L["l_lo"][q], L["l_hi"][q] + 1):
            m0, m1 = int(L["m0"][line]), int(L["m1"][line])
            smin, smax = L["smin"][line], L["smax"][line]
            ns = max(0, m1 - m0 + 1)
            slot0.append(off)
            ns_l.append(ns)
            if ns > 0:
                for k in range(ns):
                    samples.append([eta[q] * ds[s + k].real, eta[q] * ds[s + k].imag, a[s + k], 0.0])
                lens.append([max(0.0, m0 * h - smin), max(0.0, smax - m1 * h)])
                s += ns
                off += ns
            else:
                e_par, e_perp = vh[q], np.array([-vh[q][1], vh[q][0]])
                P = O + l * h * e_perp + 0.5 * (smin + smax) * e_par
                dm = _bilinear(p, ghost, np.asarray(delta, np.complex128), P[0], P[1])
                am = p["charge_sign"] * float(g.external_a(np.array([P[0]]), np.array([P[1]]))[0] @ vh[q])
                samples.append([eta[q] * dm.real, eta[q] * dm.imag, am, 0.0])
                lens.append([smax - smin, smax - smin])
                off += 1
            line += 1
    return (np.array(samples, np.float32), np.array(slot0, np.int32), np.array(ns_l, np.int32),
            np.array(lens, np.float32))


class _Call:
    """Device copies of a grain's line inputs and one call of the entry point."""

    def __init__(self, p, delta):
        import torch
        self.p = p
        self.samples, self.slot0, self.ns, self.lens = _line_inputs(p, delta)
        self.n_lines = len(self.slot0)
        dev = torch.device("cuda")
        self.d = [torch.from_numpy(a).to(dev) for a in (self.samples, self.slot0, self.ns, self.lens)]
        self.rows = np.concatenate([self.slot0[i] + np.arange(self.ns[i])
                                    for i in range(self.n_lines) if self.ns[i] > 0])
        n_e = p["n_energies"]
        self.images = torch.empty((len(self.samples), 4), dtype=torch.float32, device=dev)
        self.exits = torch.empty((2, self.n_lines, n_e, 2), dtype=torch.float32, device=dev)

    def __call__(self, entry=None, max_ns=None, n_e=None):
        import torch
        from paper_2205_15000_b300 import sc
        self.images.fill_(float("nan"))
        self.exits.fill_(float("nan"))
        p = self.p
        sc.sc_sweep_lines_noalloc(*self.d, entry, self.n_lines,
                                  int(self.ns.max()) if max_ns is None else max_ns,
                                  p["n_energies"] if n_e is None else n_e, p["t"], p["h"],
                                  self.images, self.exits)
        torch.cuda.synchronize()
        ex = self.exits.cpu().numpy()
        return self.images.cpu().numpy(), ex[..., 0] + 1j * ex[..., 1]


def _check(call, img, ex, ref_img, ref_ex, what):
    scale = np.max(np.abs(ref_img))
    assert np.max(np.abs(img[call.rows] - ref_img)) <= TOL_IMG * scale, what
    assert np.all(np.isfinite(ex)), what
    assert np.max(np.abs(ex - ref_ex)) <= TOL_EXIT, what


def _gathered_entries(ctx, n_e):
    """Entry values of the next sweep: the context's exits gathered through its
    boundary links (4 taps per line and direction), [2][n_lines][n_e]."""
    nl = ctx.info.n_lines
    ex = ctx.exits().reshape(2, nl, n_e)
    lk = ctx.links()
    L = ctx.lines()
    P = ctx.info.n_pairs
    line0 = np.concatenate([[0], np.cumsum(np.bincount(L["pair"], minlength=P))])
    ta, tc, tw = (lk[k].reshape(2, nl, 4) for k in ("angle", "chord", "w"))
    d = (ta >= P).astype(int)
    src = line0[ta % P] + tc
    return np.einsum("dlq,dlqe->dle", tw, ex[d, src])


@pytest.mark.parametrize("name", ["disc_vortex", "diamond"])
def test_noalloc_sweep_matches_context_sweeps(name):
    import torch
    from paper_2205_15000_b300 import sc

    p, delta = _grain(name)
    n_e = p["n_energies"]
    ctx = sc.Context(p, precision="fp32")
    ctx.set_fields(delta)
    ctx.sweep()
    ref_img = ctx.images()
    ref_ex = ctx.exits().reshape(2, ctx.info.n_lines, n_e)
    call = _Call(p, delta)
    assert call.n_lines == ctx.info.n_lines
    # first sweep (homogeneous start), twice in a row on the shared array
    for k in range(2):
        img, ex = call()
        _check(call, img, ex, ref_img, ref_ex, f"first sweep, call {k}")
    # second sweep: entry values gathered from the first sweep's exits
    entry = _gathered_entries(ctx, n_e)
    d_entry = torch.from_numpy(np.stack([entry.real, entry.imag], axis=-1).astype(np.float32)).cuda()
    ctx.sweep()
    img, ex = call(entry=d_entry)
    _check(call, img, ex, ctx.images(), ctx.exits().reshape(2, ctx.info.n_lines, n_e), "second sweep")


def test_noalloc_skips_lines_longer_than_max_ns():
    """A line with more samples than max_ns is not swept: its exit values are
    NaN, its image slots are left alone, and every other line comes out bit for
    bit as in a call whose max_ns covers all lines (the kernel checks a line's
    length before it reads any sample)."""
    p, delta = _grain("diamond")
    call = _Call(p, delta)
    full_img, full_ex = call()
    longest = int(call.ns.max())
    over = call.ns > longest - 1
    assert 0 < over.sum() < call.n_lines
    img, ex = call(max_ns=longest - 1)
    assert np.all(np.isnan(ex[:, over]))
    np.testing.assert_array_equal(ex[:, ~over], full_ex[:, ~over])
    keep = np.concatenate([call.slot0[i] + np.arange(max(call.ns[i], 1)) for i in range(call.n_lines) if not over[i]])
    skip = np.concatenate([call.slot0[i] + np.arange(call.ns[i]) for i in range(call.n_lines) if over[i]])
    np.testing.assert_array_equal(img[keep], full_img[keep])
    assert np.all(np.isnan(img[skip]))


def test_noalloc_later_calls_take_no_device_memory():
    """After the first call on a device (which looks up the static array and
    loads the kernels of every energy layout), a call with another energy
    layout leaves the device's free memory unchanged."""
    import torch

    p, delta = _grain("diamond")
    call = _Call(p, delta)
    call(n_e=13)  # one energy per lane
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n_e in (40, 13, 40):  # two energies per lane, then back
        call(n_e=n_e)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0


def test_noalloc_rejects_sizes_beyond_limit():
    import torch
    from paper_2205_15000_b300 import sc

    dev = torch.device("cuda")
    f = torch.zeros(64, dtype=torch.float32, device=dev)
    i = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(sc.ScError) as ei:
        sc.sc_sweep_lines_noalloc(f, i, i, f, None, 1, 4, 300, 0.5, 0.2, f, f)
    assert ei.value.status == sc.SC_EINVAL and "256" in str(ei.value)
    with pytest.raises(sc.ScError) as ei:
        sc.sc_sweep_lines_noalloc(f, i, i, f, None, 1, 1 << 20, 64, 0.5, 0.2, f, f)
    assert ei.value.status == sc.SC_EINVAL and "static scratch" in str(ei.value)
