"""torch.autograd.Function wrappers of the sweep and of the LDOS.

Forward runs the library's sweep (or LDOS sweeps) through the C ABI; backward
calls the library's adjoint sweep.  The boundary coherence functions are
treated as constants: the gradient is that of the sweep at fixed entry
values (converge them first, e.g. with sc_burnin).  Nothing here computes
physics; tensors are only handed to and from the library.
"""
import torch

from . import sc


class RiccatiSweep(torch.autograd.Function):
    """(Delta, A_ind) -> (Delta_new, j, F(R), F_total) for one context."""

    @staticmethod
    def forward(fctx, context, delta, aind):
        context.set_fields(delta.detach(), None if aind is None else aind.detach())
        context.sweep()
        out = context.outputs()
        fctx.context = context
        fctx.sweep_id = context.sweep_count
        fctx.has_a = aind is not None
        F_total = torch.tensor(out["F_total"], dtype=torch.float64, device=delta.device)
        return out["delta_new"], out["j"], out["F"], F_total

    @staticmethod
    def backward(fctx, g_dn, g_j, g_F, g_Ft):
        context = fctx.context
        if context.sweep_count != fctx.sweep_id:
            raise RuntimeError("the context swept again after this forward; its adjoint is gone")
        gd, ga = context.adjoint(g_delta_new=g_dn, g_j=g_j, g_F=g_F,
                                 g_Ftotal=0.0 if g_Ft is None else float(g_Ft))
        return None, gd, (ga if fctx.has_a else None)


class LdosMap(torch.autograd.Function):
    """(Delta, A_ind) -> N(R, eps)/N_F at the given (symmetric) energies."""

    @staticmethod
    def forward(fctx, context, delta, aind, energies, broadening, n_burnin):
        context.set_fields(delta.detach(), None if aind is None else aind.detach())
        N = context.ldos(energies, broadening, n_burnin)
        fctx.context = context
        fctx.args = (list(energies), float(broadening), int(n_burnin))
        fctx.has_a = aind is not None
        fctx.fields = (delta.detach(), None if aind is None else aind.detach())
        return N

    @staticmethod
    def backward(fctx, g_N):
        context = fctx.context
        context.set_fields(*fctx.fields)
        energies, broadening, n_burnin = fctx.args
        gd, ga = context.ldos_adjoint(energies, broadening, g_N.contiguous(), n_burnin)
        return None, gd, (ga if fctx.has_a else None), None, None, None


def riccati_sweep(context, delta, aind=None):
    return RiccatiSweep.apply(context, delta, aind)


def ldos_map(context, delta, energies, broadening, aind=None, n_burnin=40):
    return LdosMap.apply(context, delta, aind, energies, broadening, n_burnin)
