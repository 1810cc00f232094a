"""Adjoint sweep at the large workload's size: d_{x2-y2} square of side 200 xi0
on a 1024 x 1024 grid, 256 Fermi angles, t = 0.05 (160 Matsubara energies),
20 vortices.

Central differences of the oracle are out of reach at this size (each
evaluation is 4.3e10 steps), so the FP32 adjoint -- with the forward gamma
parked at every sample and kept every 32 samples -- is compared with the FP64
adjoint of the same sweep, which the oracle's central differences fix at the
adjoint workload's size.  The sweep starts from fresh boundary values (the
same entry values in both precisions).  Bound: 1e-3 of the largest FP64
gradient component, the FP32 bound of the adjoint's parity.
"""
import numpy as np
import pytest

from paper_2205_15000_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _gradients(p, d, precision, ckpt=0):
    import torch
    from paper_2205_15000_b300 import sc
    ctx = sc.Context(dict(p, adjoint_checkpoint=ckpt), precision=precision)
    ctx.set_fields(d)
    ctx.sweep()
    gd, ga = ctx.adjoint(g_Ftotal=1.0)
    out = gd.cpu().numpy(), ga.cpu().numpy()
    ctx.close()
    torch.cuda.empty_cache()
    return out


def test_c5_fp32_adjoint_against_fp64_adjoint():
    p, d, _ = W.c5_square_d()
    gd64, ga64 = _gradients(p, d, "fp64")
    s_d, s_a = np.max(np.abs(gd64)), np.max(np.abs(ga64))
    assert s_d > 0 and s_a > 0
    for ckpt in (0, 32):
        gd32, ga32 = _gradients(p, d, "fp32", ckpt)
        ed = np.max(np.abs(gd32 - gd64)) / s_d
        ea = np.max(np.abs(ga32 - ga64)) / s_a
        print(f"c5 adjoint, FP32 (checkpoint {ckpt}) against FP64: dDelta {ed:.3e}, dA {ea:.3e}")
        assert ed <= 1e-3 and ea <= 1e-3, (ckpt, ed, ea)
