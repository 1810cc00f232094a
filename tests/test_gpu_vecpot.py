"""The induced vector potential (App. D) computed by zero-padded FFT
convolution on the device against the oracle's direct double sum of the same
cell-integrated Green's function, on the current of a sweep: FP64 to 1e-10 of
the field's maximum, on square and non-square grids."""
import numpy as np
import pytest

import oracle
from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _grains():
    p = W.disc(5.0, 40, pairing=0, t=0.5, n_angles=16, n_energies=6, flux_quanta=1.5, kappa=3.0)
    yield p, W.vortex_delta(p, 0.25, [(0.5, 0.0)], [-1], seed=91, rel_noise=0.05)
    # a rectangle on a 64 x 40 grid: padded 128 x 128, unequal extents
    q = W.base_params(nx=64, ny=40, h=0.25, x0=-8.0, y0=-5.0, shape_kind=1, vx=[-7.5, 7.5, 7.5, -7.5],
                      vy=[-4.5, -4.5, 4.5, 4.5], pairing=1, t=0.3, n_angles=12, n_energies=8, flux_quanta=2.0,
                      kappa=5.0)
    yield q, W.vortex_delta(q, 0.22, [(2.0, 1.0)], [-1], seed=92, rel_noise=0.05)
    # a composite grain with a hole on a 100 x 100 grid (padded 256 x 256)
    r = W.annulus(6.0, 2.0, 100, margin=0.3, pairing=0, t=0.5, n_angles=16, n_energies=6, flux_quanta=1.0,
                  kappa=4.0)
    yield r, W.noisy_delta(r, 0.26, 0.1, seed=93)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_fft_vector_potential_matches_direct_sum(k):
    from paper_2205_15000_b300 import sc
    import torch
    p, d = list(_grains())[k]
    g = oracle.OracleGeom(p)
    o = g.full_sweep(d)
    ref = g.vector_potential(o["j"])
    ctx = sc.Context(p, precision="fp64")
    ctx.set_fields(d)
    ctx.sweep()
    sc.sc_update_vector_potential(ctx.h)
    _, a = ctx.fields()
    torch.cuda.synchronize()
    a = a.cpu().numpy()
    scale = np.max(np.abs(ref))
    assert scale > 0
    assert np.max(np.abs(a - ref)) <= 1e-10 * scale, np.max(np.abs(a - ref)) / scale
