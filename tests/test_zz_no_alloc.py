"""The allocation-free line sweep (sc_sweep_lines_noalloc) against the regular
context sweep (sc_riccati_sweep).

sc_sweep_lines_noalloc exists for callers that cannot allocate device memory
when they run a sweep (their device heap belongs to another allocator, or
they cannot afford cudaMalloc's implicit synchronisation).  It takes every
buffer from the caller and keeps its scratch in a static array inside the
library.  Here it gets the lattice samples of a grain, built from the
oracle's FP64 sample fields, and must reproduce the context sweep's first
FP32 sweep (images and exit values) within the FP32 tolerances of the other
GPU tests -- on two calls in a row, since every call reuses the same array.
"""
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
    p = W.diamond(12.0, 48, pairing=1, t=0.3, n_angles=16, n_energies=40, flux_quanta=0.5)
    return p, W.noisy_delta(p, 0.23, 0.1, seed=12)


def _line_inputs(p, delta):
    """Samples and line table in the library's slot order (pairs, then lines,
    then samples), from the oracle's fields at the lattice samples."""
    g = oracle.OracleGeom(p)
    w, vh, eta = g.quadrature()
    L = g.lines()
    h = p["h"]
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
                # a line without samples: its chord-midpoint value is not compared here
                samples.append([0.2, 0.0, 0.0, 0.0])
                lens.append([smax - smin, smax - smin])
                off += 1
            line += 1
    return (np.array(samples, np.float32), np.array(slot0, np.int32), np.array(ns_l, np.int32),
            np.array(lens, np.float32))


@pytest.mark.parametrize("name", ["disc_vortex", "diamond"])
def test_noalloc_sweep_matches_context_sweep_twice(name):
    import torch
    from paper_2205_15000_b300 import sc

    p, delta = _grain(name)
    ctx = sc.Context(p, precision="fp32")
    ctx.set_fields(delta)
    ctx.sweep()
    ref_img = ctx.images()
    ref_ex = ctx.exits().reshape(2, ctx.info.n_lines, p["n_energies"])

    samples, slot0, ns, lens = _line_inputs(p, delta)
    n_lines = len(slot0)
    assert n_lines == ctx.info.n_lines
    n_e = p["n_energies"]
    dev = torch.device("cuda")
    d_samples = torch.from_numpy(samples).to(dev)
    d_slot0 = torch.from_numpy(slot0).to(dev)
    d_ns = torch.from_numpy(ns).to(dev)
    d_len = torch.from_numpy(lens).to(dev)
    has = ns > 0
    rows = np.concatenate([slot0[i] + np.arange(ns[i]) for i in range(n_lines) if ns[i] > 0])
    for call in range(2):
        images = torch.full((len(samples), 4), float("nan"), dtype=torch.float32, device=dev)
        exits = torch.full((2, n_lines, n_e, 2), float("nan"), dtype=torch.float32, device=dev)
        sc.sc_sweep_lines_noalloc(d_samples, d_slot0, d_ns, d_len, None, n_lines, int(ns.max()), n_e,
                                  p["t"], p["h"], images, exits)
        torch.cuda.synchronize()
        img = images.cpu().numpy()[rows]
        ex = exits.cpu().numpy()
        ex = ex[..., 0] + 1j * ex[..., 1]
        scale = np.max(np.abs(ref_img))
        assert np.max(np.abs(img - ref_img)) <= TOL_IMG * scale, call
        assert np.max(np.abs(ex[:, has] - ref_ex[:, has])) <= TOL_EXIT, call


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
