"""Cases for the bounds-checked build (libsc_checked.so, every table index of
the kernels compared with its table's size): the same computations run once
with each library, so that the results can be compared bit for bit.  Run as a
script it writes the results of the library that SC_LIBRARY selects to an
.npz file, with the kernels' violation count.  Not collected by pytest."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2205_15000_b300 import workloads as W  # noqa: E402


def grains():
    g = {}
    p = W.disc(5.0, 40, pairing=1, t=0.25, n_angles=18, n_energies=13, flux_quanta=1.0)
    g["disc_vortex"] = (p, W.vortex_delta(p, 0.22, [(1.0, -0.5)], [-1], seed=13, rel_noise=0.05))
    p = W.diamond(12.0, 48, pairing=1, t=0.3, n_angles=16, n_energies=40, flux_quanta=0.5)
    g["diamond"] = (p, W.noisy_delta(p, 0.23, 0.1, seed=12))
    p = W.annulus(6.0, 2.5, 48, margin=0.3, pairing=0, t=0.5, n_angles=16, n_energies=10, gauge="solenoid",
                  flux_quanta=0.5)
    g["annulus"] = (p, W.noisy_delta(p, 0.26, 0.05, seed=14))
    p = W.disc(3.0, 24, pairing=1, t=0.02, n_angles=8, n_energies=700, flux_quanta=0.4)
    g["blocked_700"] = (p, W.vortex_delta(p, 0.24, [(0.5, -0.3)], [-1], seed=61, rel_noise=0.05))
    return g


def run():
    """Every case with the loaded library: {name: array}."""
    import torch
    from paper_2205_15000_b300 import sc
    out = {}
    gr = grains()
    for name, (p, d) in gr.items():
        for prec in ("fp64", "fp32"):
            ctx = sc.Context(p, precision=prec)
            ctx.set_fields(d)
            for k in range(2):
                ctx.sweep()
                o = ctx.outputs()
                out[f"{name}_{prec}_{k}_images"] = ctx.images()
                out[f"{name}_{prec}_{k}_exits"] = ctx.exits()
                for key in ("delta_new", "j", "F"):
                    out[f"{name}_{prec}_{k}_{key}"] = o[key].cpu().numpy()
            if name != "blocked_700":
                gd, ga = ctx.adjoint(g_Ftotal=1.0)
                out[f"adj_{name}_{prec}_delta"] = gd.cpu().numpy()
                out[f"adj_{name}_{prec}_a"] = ga.cpu().numpy()
                out[f"ldos_{name}_{prec}"] = ctx.ldos(np.linspace(-0.3, 0.3, 6), 0.05, 30).cpu().numpy()
            ctx.close()
    b = sc.Batch([gr[k][0] for k in ("disc_vortex", "diamond", "annulus")], precision="fp32")
    for m, k in zip(b.members, ("disc_vortex", "diamond", "annulus")):
        m.set_fields(gr[k][1])
    b.run(3, True)
    for m, k in zip(b.members, ("disc_vortex", "diamond", "annulus")):
        o = m.outputs()
        for key in ("delta_new", "j", "F"):
            out[f"batch_{k}_{key}"] = o[key].cpu().numpy()
    b.close()
    # a member in two energy parts (132 energies: 2 x 10 and 16 x 7 lanes x energies)
    p132 = W.disc(3.0, 24, pairing=1, t=0.06, n_angles=16, n_energies=132, flux_quanta=0.4)
    d132 = W.vortex_delta(p132, 0.24, [(0.5, -0.3)], [-1], seed=35, rel_noise=0.05)
    b = sc.Batch([p132, gr["diamond"][0]], precision="fp32", energies_per_lane=10)
    sc.sc_batch_set_energy_parts(b.h, True)
    assert b.info().split_members >= 1
    for m, d in zip(b.members, (d132, gr["diamond"][1])):
        m.set_fields(d)
    b.run(3, True)
    for m, k in zip(b.members, ("disc_132", "diamond")):
        o = m.outputs()
        for key in ("delta_new", "j", "F"):
            out[f"parts_{k}_{key}"] = o[key].cpu().numpy()
    b.close()
    torch.cuda.synchronize()
    v, checked = sc.sc_debug_bounds()
    return out, v, checked


if __name__ == "__main__":
    res, v, checked = run()
    np.savez(sys.argv[1], violations=np.array(v), checked=np.array(int(checked)), **res)
