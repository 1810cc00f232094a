"""The self-consistent s-wave annulus in the symmetric gauge with screening
against the analytic London-Maxwell solution of Sec. 5.1.2 (Eqs. LMeqRing,
Aring, Bring): the whole loop -- sweep, gap equation, current, induced vector
potential by FFT convolution (App. D), Barzilai-Borwein steps (App. E) --
converged on the GPU, and the magnetic field B = B_ext + curl A_ind compared
with B(R) = Phi0 [a I0(R/lambda) - b K0(R/lambda)] in the annulus and the
uniform field beta Phi0 / A_h in the hole, with 1/lambda^2 = Y(T) / lambda0^2
(Y the Yosida function of the converged gap, lambda0 = kappa xi0)."""
import math

import numpy as np
import pytest
from scipy.special import iv, kv

from paper_2205_15000_b300 import workloads as W

R_OUT, R_IN = 25.0, 10.0


def london_maxwell_B(alpha, n, lam):
    """B(R) in units B0 = Phi0/(pi xi0^2): the annulus profile and the hole's
    uniform field, from the constants (a, b, beta) of Eq. Aring."""
    A = math.pi * (R_OUT ** 2 - R_IN ** 2)
    Ah = math.pi * R_IN ** 2
    I = lambda mu, r: iv(mu, r / lam)  # noqa: E731
    K = lambda mu, r: kv(mu, r / lam)  # noqa: E731
    M = I(0, R_OUT) * K(2, R_IN) - I(2, R_IN) * K(0, R_OUT)
    a = (K(2, R_IN) / A * alpha + K(0, R_OUT) / Ah * n) / M
    b = (I(2, R_IN) / A * alpha + I(0, R_OUT) / Ah * n) / M
    beta = (2 * math.pi * lam ** 2 / A * alpha - (I(0, R_OUT) * K(0, R_IN) - I(0, R_IN) * K(0, R_OUT)) * n) / M
    return (lambda r: math.pi * (a * I(0, r) - b * K(0, r))), math.pi * beta / Ah


def test_london_maxwell_solution_limits():
    """The transcription of Eq. Aring: continuity of B at R> with B_ext, and no
    screening as lambda grows (B -> B_ext everywhere)."""
    A = math.pi * (R_OUT ** 2 - R_IN ** 2)
    B, Bh = london_maxwell_B(1.3, 0, 1e4)
    assert abs(B(R_OUT) - math.pi * 1.3 / A) < 1e-12
    assert abs(B(R_IN) / (math.pi * 1.3 / A) - 1) < 1e-5 and abs(Bh / (math.pi * 1.3 / A) - 1) < 1e-5
    B, Bh = london_maxwell_B(0.0, -1, 10.0)
    assert abs(B(R_OUT)) < 1e-15 and abs(B(R_IN) - Bh) < 1e-15 and Bh > 0


@pytest.mark.gpu
@pytest.mark.parametrize("alpha,n", [(1.0, 0), (0.0, -1)])
def test_screened_annulus_matches_london_maxwell(alpha, n):
    import torch
    from paper_2205_15000_b300 import sc
    t, ne, kappa = 0.5, 16, 10.0
    p = W.annulus(R_OUT, R_IN, 200, pairing=0, t=t, n_angles=32, n_energies=ne, flux_quanta=alpha, kappa=kappa,
                  charge_sign=-1)
    X, Y = W.grid_xy(p)
    ctx = sc.Context(p, precision="fp32")
    ctx.set_fields(0.26 * np.exp(1j * n * np.arctan2(Y, X)), np.zeros((p["ny"], p["nx"], 2)))
    prm = sc.accel_params("barzilai-borwein")
    for it in range(400):
        ctx.sweep()
        eps = ctx.outputs()["eps_G"]
        ctx.accelerate(prm)
        if eps < 1e-6 and it > 20:
            break
    assert eps < 1e-5
    d, a = ctx.fields()
    torch.cuda.synchronize()
    d, a = d.cpu().numpy(), a.cpu().numpy()
    m = ctx.mask().astype(bool)
    r = np.hypot(X, Y)
    # Yosida function of the converged gap (uniform in the bulk of the s-wave annulus)
    dg = float(np.median(np.abs(d[m & (r > 14) & (r < 21)])))
    e = t * (np.arange(ne) + 0.5)
    yos = t * float(np.sum(dg * dg / (e * e + dg * dg) ** 1.5))
    lam = kappa / math.sqrt(yos)
    h = p["h"]
    Bind = np.zeros_like(r)
    Bind[1:-1, 1:-1] = ((a[1:-1, 2:, 1] - a[1:-1, :-2, 1]) - (a[2:, 1:-1, 0] - a[:-2, 1:-1, 0])) / (2 * h)
    Btot = math.pi * alpha / (math.pi * (R_OUT ** 2 - R_IN ** 2)) + Bind
    Bf, Bh = london_maxwell_B(alpha, n, lam)
    scale = max(abs(Bf(R_OUT) - Bh), abs(Bh), abs(Bf(R_IN)))
    for lo, hi in [(2.0, 8.0), (11.0, 13.0), (15.0, 17.0), (19.0, 21.0), (23.0, 24.0)]:
        sel = (r >= lo) & (r < hi)
        rm = float(np.mean(r[sel]))
        ref = Bh if hi <= R_IN else Bf(rm)
        print(f"alpha {alpha} n {n} lambda {lam:.3f} R {rm:5.2f}: B {float(np.mean(Btot[sel])):.6e} "
              f"analytic {ref:.6e} (deviation {abs(float(np.mean(Btot[sel])) - ref) / scale:.4f} of the scale)")
        assert abs(float(np.mean(Btot[sel])) - ref) < 0.03 * scale, (lo, hi, float(np.mean(Btot[sel])), ref, scale)
